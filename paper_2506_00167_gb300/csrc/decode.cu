// Layered offset-min-sum decoding of QC-LDPC code blocks on sm_103a.
//
// Algorithm (the paper's receiver decodes with a toolbox LDPC decoder and
// states no algorithm, Sec. VI-D "UE"; this library fixes layered offset min-sum):
// every iteration runs base rows l = 0 .. m_eff-1 in order.  Lifted check
// (l, k) reaches, through base edge j (column c_j, shift s_j = V mod Z),
// variable v_j = c_j * Z + (k + s_j) mod Z, and updates
//   Q_j = L[v_j] - R_j,  R'_j = (-1)^{XOR_{i!=j} [Q_i < 0]} max(min_{i!=j}|Q_i| - beta, 0),
//   L[v_j] = Q_j + R'_j.
// After an iteration the hard decision [L < 0] is checked against the m_eff
// rows; with early termination a block stops at the first zero syndrome.
//
// GB300 mapping:
// * one group of Z threads per code block, thread k owns lifted check k of
//   every layer; a block holds G groups of one shape (G * Z threads);
// * the circulant shift is the shared-memory address (k + s_j) mod Z: each
//   block of Z posteriors is one contiguous run, so a warp's 32 reads hit 32
//   distinct banks (Z a multiple of 32);
// * the launch's edge tables and every group's channel LLRs are staged into
//   shared memory by bulk (TMA-engine) copies completing on one mbarrier;
// * the edges of a row are read two at a time (one 128-bit load: two column
//   bases, two shifts); the table pads rows to an even degree with an edge
//   on a per-group dummy slot whose value can never be a row minimum, which
//   the paired INT8 kernel processes (cheaper than a run-time tail there) and
//   this kernel skips (an odd row's last edge runs after its whole chunks);
// * check-to-variable messages are stored compressed per check: the two
//   smallest offset magnitudes, the argmin edge and one sign bit per edge
//   (12 bytes FP32, 6 bytes INT8, 8 bytes INT16 per check) -- in shared
//   memory, or in a global scratch slot per resident group when the shape
//   does not fit (RGLOBAL);
// * the update is written for the SM's ALU pipe, which runs min/max,
//   compare, select and logic at half the FMA rate and bounds this kernel:
//   signs are applied as one bitwise op on the float's sign bit, the parity
//   is an XOR of the float bit patterns, the argmin is found in the second
//   pass by comparing against the minimum (ties are value-invariant), and in
//   the integer modes the minimum and argmin are tracked together as one
//   exact key (magnitude * 32 + edge);
// * layers are separated by a named barrier per group (a warp sync for
//   Z <= 32); after each iteration the hard decisions are packed by warp
//   ballot into a bitmap, the syndrome is a funnel-shift XOR of rotated bitmap
//   words, and bar.red.or combines it; the information bits are the first
//   kb columns of that bitmap, copied out coalesced.
#include "decode_core.cuh"

namespace ldpcgb {

namespace {

using namespace core;

template <typename LT, typename MT, bool SAT, bool RGLOBAL, bool CRC>
__global__ void __launch_bounds__(kDecodeMaxBlock, 2) oms_decode_kernel(const DecodeArgs a) {
  extern __shared__ __align__(128) uint8_t smem[];
  uint32_t* s_tab = reinterpret_cast<uint32_t*>(smem);
  uint64_t* s_bar = reinterpret_cast<uint64_t*>(smem + a.hdr_bytes - 16);
  int* s_item = reinterpret_cast<int*>(smem + a.hdr_bytes - 8);
  uint8_t* regions = smem + a.hdr_bytes;

  const int tid = threadIdx.x;
  const int lane = tid & 31;

  if (tid == 0) {
    mbar_init(s_bar, 1);
    fence_proxy_async_smem();
  }
  __syncthreads();
  uint32_t phase = 0;

  // items come from the work queue (largest first) or, without one, by stride
  for (int next = blockIdx.x;; next += gridDim.x) {
    if (tid == 0) *s_item = a.queue ? static_cast<int>(atomicAdd(a.queue, 1u)) : next;
    __syncthreads();
    const int item_i = *s_item;
    if (item_i >= a.n_items) break;
    const DecodeItem item = a.items[item_i];
    const ShapeDev sh = a.shapes[item.shape];
    const int Z = item.Z;
    const int g = tid / Z;
    const int k = tid - g * Z;
    const uint32_t wmask = (Z >= 32) ? 0xFFFFFFFFu : (((1u << Z) - 1u) << (lane & ~(Z - 1)));

    // ---- stage the shape table and each group's LLRs (bulk copies)
    if (tid == 0) {
      fence_proxy_async_smem();  // earlier generic smem accesses before async writes
      uint32_t bytes = static_cast<uint32_t>(sh.tab_words) * 4u;
      for (int gg = 0; gg < item.count; ++gg) {
        const CbDev cb = a.cbs[a.item_cbs[item.first + gg]];
        bytes += static_cast<uint32_t>(cb.n_eff * Z) * sizeof(LT);
      }
      mbar_arrive_expect_tx(s_bar, bytes);
      bulk_g2s(s_tab, a.tabs + sh.tab_off, static_cast<uint32_t>(sh.tab_words) * 4u, s_bar);
      for (int gg = 0; gg < item.count; ++gg) {
        const CbDev cb = a.cbs[a.item_cbs[item.first + gg]];
        const LT* src = static_cast<const LT*>(a.llr) + cb.llr_off;
        bulk_g2s(regions + gg * item.region_bytes, src, static_cast<uint32_t>(cb.n_eff * Z) * sizeof(LT), s_bar);
      }
    }

    const bool active = g < item.count;
    CbDev cb{};
    int cbi = 0;
    LT* L = reinterpret_cast<LT*>(regions + g * item.region_bytes);
    MT *mag1, *mag2;
    uint32_t* meta;
    if (RGLOBAL) {
      uint8_t* base = a.rscratch + (static_cast<int64_t>(blockIdx.x) * a.G + g) * a.rscratch_group;
      mag1 = reinterpret_cast<MT*>(base);
      mag2 = mag1 + item.rec_cap;
      meta = reinterpret_cast<uint32_t*>(base + 2 * ((item.rec_cap * sizeof(MT) + 15) & ~15));
    } else {
      uint8_t* base = regions + g * item.region_bytes + item.L_bytes + item.hb_bytes;
      mag1 = reinterpret_cast<MT*>(base);
      mag2 = mag1 + item.rec_cap;
      meta = reinterpret_cast<uint32_t*>(base + 2 * ((item.rec_cap * sizeof(MT) + 15) & ~15));
    }
    if (active) {
      cbi = a.item_cbs[item.first + g];
      cb = a.cbs[cbi];
      // R = 0 before the first iteration, and this thread's dummy slot (both
      // overlap the copies in flight: neither region is a copy target)
      zero_records(mag1, mag2, meta, cb.m_eff * Z, k, Z);
      if constexpr (SAT)
        st_val(L, item.dummy_base + k, a.post_sat);
      else
        L[item.dummy_base + k] = LT(kBigF);
    }

    const bool got = mbar_wait_bounded(s_bar, phase, 1u << 22);
    phase ^= 1u;
    if (!__syncthreads_and(got)) {
      if (tid == 0) atomicOr(a.err, LDPC_DEVERR_TMA_TIMEOUT);
      // give the copies still in flight a bounded chance to land before exiting
      mbar_wait_bounded(s_bar, phase ^ 1u, 1u << 20);
      return;
    }

    if (active) {
      const uint32_t* rows = s_tab + sh.row_off;
      uint32_t* hb = reinterpret_cast<uint32_t*>(regions + g * item.region_bytes + item.L_bytes);
      const int m = cb.m_eff;
      const bool wide = (Z & 31) == 0;
      if constexpr (!SAT) {
        // -0.0 in a caller's LLRs would carry a sign bit while not being < 0;
        // adding +0.0 turns it into +0.0 and leaves every other value alone
        for (int i = k; i < cb.n_eff * Z; i += Z) L[i] = L[i] + LT(0);
        group_sync(Z, g, wmask);
      }
      int it = 1;
      bool ok = false, crc_ok = false;
      const bool has_crc = CRC && (cb.flags & LDPC_CB_CRC24B) != 0;
      RowIn<kChunk> row = load_row<kChunk>(s_tab, rows[0], mag1, mag2, meta, k);
      for (;; ++it) {
        for (int l = 0; l < m; ++l) {
          check_update_exact<LT, MT, SAT, true, kChunk>(row, k, Z, L, mag1, mag2, meta, l * Z + k,
                                                        item.dummy_base + k, a.beta, a.msg_sat, a.post_sat);
          // the next row's table and record are ready before the barrier
          const int ln = l + 1 < m ? l + 1 : 0;
          row = load_row<kChunk>(s_tab, rows[ln], mag1, mag2, meta, ln * Z + k);
          group_sync(Z, g, wmask);
        }
        if (a.early_term || it == a.max_iter) {
          bool bad;
          uint32_t cr = 0;
          const uint32_t* ptab = a.cbcrc + a.shapes[item.shape].crc_off;
          if (wide) {
            hard_bitmap(L, hb, cb.n_eff, k, Z);
            group_sync(Z, g, wmask);
            bad = syndrome_bitmap<kChunk>(s_tab, rows, hb, m, k, Z);
            if (has_crc) cr = cb_crc_part_hb(hb, ptab, cb.kb, k, Z);
          } else {
            bad = syndrome_direct<kChunk>(s_tab, rows, m, k, Z, L);
            if (has_crc) cr = cb_crc_part(L, ptab, cb.kb, k, Z);
          }
          ok = !group_any(Z, g, wmask, bad);
          // after that barrier the bitmap's parity words are free: scratch for the CRC's XOR
          if (has_crc) crc_ok = group_xor_zero(Z, g, wmask, cr, hb + cb.kb * (Z >> 5), k);
          if ((ok || crc_ok) && a.early_term) break;
          if (it == a.max_iter) break;
        }
      }
      // ---- the kb information columns, packed
      const int kb = cb.kb;
      uint32_t* out = a.bits + cb.bits_off;
      if (wide) {  // the bitmap already holds them: a coalesced copy
        const int nw = kb * (Z >> 5);
        for (int i = k; i < nw; i += Z) out[i] = hb[i];
      } else {  // Z == 16: two columns per word, half a warp per block
        const int sh16 = lane & 16;
        for (int c = 0; c < kb; c += 2) {
          const uint32_t b0 = __ballot_sync(wmask, L[c * Z + k] < LT(0)) >> sh16;
          const uint32_t b1 = __ballot_sync(wmask, L[(c + 1) * Z + k] < LT(0)) >> sh16;
          if (k == 0) out[c >> 1] = (b0 & 0xFFFFu) | (b1 << 16);
        }
      }
      if (k == 0) a.status[cbi] = it | (ok ? (1 << 16) : 0) | (crc_ok ? (1 << 17) : 0);
    }
    __syncthreads();  // the next item's copies overwrite this item's shared memory
  }
}

// INT8, two code blocks per thread group (see decode_core.cuh): items list
// up to 2G code blocks of one shape, largest first, paired in order, so the
// first block of a pair has at least as many decoded rows as the second.  A
// pair runs the first block's rows; for the second block the extra rows only
// touch its never-sent parity columns (LLR 0) and leave every other variable
// unchanged, and its syndrome covers its own rows only.
//
// RGLOBAL: the three message words per check live in a global scratch slot
// per resident group, and the int8 LLRs are read straight from global memory
// (one 32-bit load per four variables of each block) instead of being staged.
template <bool RGLOBAL, bool CRC>
__global__ void __launch_bounds__(kDecodeMaxBlock, 2) oms_decode_i8x2_kernel(const DecodeArgs a) {
  extern __shared__ __align__(128) uint8_t smem[];
  uint32_t* s_tab = reinterpret_cast<uint32_t*>(smem);
  uint64_t* s_bar = reinterpret_cast<uint64_t*>(smem + a.hdr_bytes - 16);
  int* s_item = reinterpret_cast<int*>(smem + a.hdr_bytes - 8);
  uint8_t* regions = smem + a.hdr_bytes;
  const int tid = threadIdx.x;
  const __half2 beta = __float2half2_rn(a.beta);
  const __half2 msg = __float2half2_rn(a.msg_sat);
  const __half2 post = __float2half2_rn(a.post_sat);

  if (tid == 0) {
    mbar_init(s_bar, 1);
    fence_proxy_async_smem();
  }
  __syncthreads();
  uint32_t phase = 0;

  for (int next = blockIdx.x;; next += gridDim.x) {
    if (tid == 0) *s_item = a.queue ? static_cast<int>(atomicAdd(a.queue, 1u)) : next;
    __syncthreads();
    const int item_i = *s_item;
    if (item_i >= a.n_items) break;
    const DecodeItem item = a.items[item_i];
    const ShapeDev sh = a.shapes[item.shape];
    const int Z = item.Z;
    const int g = tid / Z;
    const int k = tid - g * Z;
    const int pairs = (item.count + 1) >> 1;
    uint8_t* reg = regions + g * item.region_bytes;
    uint32_t* L = reinterpret_cast<uint32_t*>(reg);
    uint32_t* hbA = reinterpret_cast<uint32_t*>(reg + item.L_bytes);
    uint32_t* hbB = reinterpret_cast<uint32_t*>(reg + item.L_bytes + item.hb_bytes);
    uint8_t* recs = reg + item.L_bytes + 2 * item.hb_bytes;
    if (RGLOBAL) recs = a.rscratch + (static_cast<int64_t>(blockIdx.x) * a.G + g) * a.rscratch_group;
    // per check: (magnitudes, s1) as one 8-byte pair, then s2
    uint2* ms = reinterpret_cast<uint2*>(recs);
    uint32_t* sg2 = reinterpret_cast<uint32_t*>(recs) + 2 * item.rec_cap;

    // ---- stage the table and (shared-message form) each pair's int8 LLRs
    // into its message area
    if (tid == 0) {
      fence_proxy_async_smem();
      uint32_t bytes = static_cast<uint32_t>(sh.tab_words) * 4u;
      if (!RGLOBAL)
        for (int c = 0; c < item.count; ++c)
          bytes += static_cast<uint32_t>(a.cbs[a.item_cbs[item.first + c]].n_eff * Z);
      mbar_arrive_expect_tx(s_bar, bytes);
      bulk_g2s(s_tab, a.tabs + sh.tab_off, static_cast<uint32_t>(sh.tab_words) * 4u, s_bar);
      for (int pp = 0; pp < (RGLOBAL ? 0 : pairs); ++pp) {
        uint8_t* st = regions + pp * item.region_bytes + item.L_bytes + 2 * item.hb_bytes;
        const CbDev ca = a.cbs[a.item_cbs[item.first + 2 * pp]];
        const uint32_t na = static_cast<uint32_t>(ca.n_eff * Z);
        bulk_g2s(st, static_cast<const int8_t*>(a.llr) + ca.llr_off, na, s_bar);
        if (2 * pp + 1 < item.count) {
          const CbDev cbb = a.cbs[a.item_cbs[item.first + 2 * pp + 1]];
          bulk_g2s(st + ((na + 15u) & ~15u), static_cast<const int8_t*>(a.llr) + cbb.llr_off,
                   static_cast<uint32_t>(cbb.n_eff * Z), s_bar);
        }
      }
    }
    const bool active = g < pairs;
    const bool hasB = 2 * g + 1 < item.count;
    CbDev A{}, Bc{};
    int ia = 0, ib = 0;
    if (active) {
      ia = a.item_cbs[item.first + 2 * g];
      A = a.cbs[ia];
      if (hasB) {
        ib = a.item_cbs[item.first + 2 * g + 1];
        Bc = a.cbs[ib];
      }
    }
    const bool got = mbar_wait_bounded(s_bar, phase, 1u << 22);
    phase ^= 1u;
    if (!__syncthreads_and(got)) {
      if (tid == 0) atomicOr(a.err, LDPC_DEVERR_TMA_TIMEOUT);
      mbar_wait_bounded(s_bar, phase ^ 1u, 1u << 20);
      return;
    }
    if (active) {
      const int nA = A.n_eff * Z, nB = hasB ? Bc.n_eff * Z : 0;
      const __half2 h1536 = __float2half2_rn(1536.0f);
      if (RGLOBAL) {
        // n_eff * Z is a multiple of 32 and the LLR offsets of 16: four
        // variables per 32-bit load, written as one 16-byte store
        const uint32_t* gA = reinterpret_cast<const uint32_t*>(static_cast<const int8_t*>(a.llr) + A.llr_off);
        const uint32_t* gB = reinterpret_cast<const uint32_t*>(static_cast<const int8_t*>(a.llr) + Bc.llr_off);
        for (int p4 = k; p4 < (nA >> 2); p4 += Z) {
          const uint32_t wa = __ldg(gA + p4);
          const uint32_t wb = 4 * p4 < nB ? __ldg(gB + p4) : 0u;
          uint32_t o[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const uint32_t va = (0x6600u + static_cast<uint32_t>(static_cast<int8_t>(wa >> (8 * i)))) & 0xFFFFu;
            const uint32_t vb = (0x6600u + static_cast<uint32_t>(static_cast<int8_t>(wb >> (8 * i)))) & 0xFFFFu;
            o[i] = as_u32(__hsub2(as_h2(va | (vb << 16)), h1536));
          }
          reinterpret_cast<uint4*>(L)[p4] = make_uint4(o[0], o[1], o[2], o[3]);
        }
      } else {
        const int8_t* stA = reinterpret_cast<const int8_t*>(recs);
        const int8_t* stB = stA + ((nA + 15) & ~15);
        for (int p = k; p < nA; p += Z) {
          const uint32_t va = static_cast<uint32_t>(0x6600 + stA[p]) & 0xFFFFu;
          const uint32_t vb = static_cast<uint32_t>(0x6600 + (p < nB ? stB[p] : 0)) & 0xFFFFu;
          L[p] = as_u32(__hsub2(as_h2(va | (vb << 16)), h1536));
        }
      }
      group_sync(Z, g, 0xFFFFFFFFu);
      for (int r = k; r < A.m_eff * Z; r += Z) {
        ms[r] = make_uint2(0u, 0u);
        sg2[r] = 0u;
      }
      group_sync(Z, g, 0xFFFFFFFFu);

      const uint32_t* rows = s_tab + sh.row_off;
      const int mA = A.m_eff, mB = hasB ? Bc.m_eff : 0;
      bool doneA = false, doneB = !hasB;
      PairIn prow = load_pair_row(s_tab, rows[0], ms, sg2, k);
      for (int it = 1;; ++it) {
        for (int l = 0; l < mA; ++l) {
          check_update_x2_by_degree(prow, k, Z, L, ms, sg2, l * Z + k, item.dummy_base + k, beta, msg, post);
          // the next row's table entry and message words are loaded before the barrier
          const int ln = l + 1 < mA ? l + 1 : 0;
          prow = load_pair_row(s_tab, rows[ln], ms, sg2, ln * Z + k);
          group_sync(Z, g, 0xFFFFFFFFu);
        }
        if (a.early_term || it == a.max_iter) {
          hard_bitmap_x2(L, hbA, hbB, A.n_eff, k, Z);
          group_sync(Z, g, 0xFFFFFFFFu);
          const bool badA = !doneA && syndrome_bitmap<kChunk>(s_tab, rows, hbA, mA, k, Z);
          const bool badB = !doneB && syndrome_bitmap<kChunk>(s_tab, rows, hbB, mB, k, Z);
          const bool crcA = CRC && !doneA && (A.flags & LDPC_CB_CRC24B) != 0;
          const bool crcB = CRC && !doneB && (Bc.flags & LDPC_CB_CRC24B) != 0;
          uint32_t rA = 0, rB = 0;
          if (crcA || crcB) {
            const uint32_t* ptab = a.cbcrc + sh.crc_off;
            if (crcA) rA = cb_crc_part_hb(hbA, ptab, A.kb, k, Z);
            if (crcB) rB = cb_crc_part_hb(hbB, ptab, A.kb, k, Z);
          }
          const bool okA = !group_any(Z, g, 0xFFFFFFFFu, badA);
          const bool okB = !group_any(Z, g, 0xFFFFFFFFu, badB);
          bool cA = false, cB = false;
          if (crcA || crcB) {  // both blocks' XORs meet in their bitmaps' (now free) parity words
            const bool zA = group_xor_zero2(Z, g, rA, rB, hbA + A.kb * (Z >> 5), hbB + A.kb * (Z >> 5), k, &cB);
            cA = crcA && zA;
            cB = crcB && cB;
          }
          const bool last = it == a.max_iter;
          const int nw = A.kb * (Z >> 5);
          if (!doneA && (((okA || cA) && a.early_term) || last)) {
            uint32_t* out = a.bits + A.bits_off;
            for (int i = k; i < nw; i += Z) out[i] = hbA[i];
            if (k == 0) a.status[ia] = it | (okA ? (1 << 16) : 0) | (cA ? (1 << 17) : 0);
            doneA = true;
          }
          if (!doneB && (((okB || cB) && a.early_term) || last)) {
            uint32_t* out = a.bits + Bc.bits_off;
            for (int i = k; i < nw; i += Z) out[i] = hbB[i];
            if (k == 0) a.status[ib] = it | (okB ? (1 << 16) : 0) | (cB ? (1 << 17) : 0);
            doneB = true;
          }
          if (doneA && doneB) break;
        }
      }
    }
    __syncthreads();
  }
}

template <bool RG, bool CRC>
const void* decode_kernel_ptr(int mode) {
  switch (mode) {
    case LDPC_F32: return reinterpret_cast<const void*>(&oms_decode_kernel<float, float, false, RG, CRC>);
    case LDPC_I8: return reinterpret_cast<const void*>(&oms_decode_kernel<int8_t, uint8_t, true, RG, CRC>);
    default: return reinterpret_cast<const void*>(&oms_decode_kernel<int16_t, uint16_t, true, RG, CRC>);
  }
}

template <bool CRC>
const void* kernel_for(int mode, int base) {
  if (base == kKindPairI8) return reinterpret_cast<const void*>(&oms_decode_i8x2_kernel<false, CRC>);
  if (base == kKindPairI8Global) return reinterpret_cast<const void*>(&oms_decode_i8x2_kernel<true, CRC>);
  return base == kKindGlobal ? decode_kernel_ptr<true, CRC>(mode) : decode_kernel_ptr<false, CRC>(mode);
}

}  // namespace

// kind = base kind | kKindCrc: the variant with the code-block CRC exit is
// launched only for launches holding a block with LDPC_CB_CRC24B; without
// it the kernel is the plain decoder, register allocation included.
const void* kernel_kind(int mode, int kind) {
  const int base = kind & ~kKindCrc;
  return (kind & kKindCrc) ? kernel_for<true>(mode, base) : kernel_for<false>(mode, base);
}

cudaError_t read_check_log_decode(uint32_t* out4) { return cudaMemcpyFromSymbol(out4, g_check_log, 16); }

cudaError_t decode_prepare(int mode) {
  for (int kind = 0; kind < 2 * kKindCrc; ++kind) {
    if (kind_is_pair(kind) && mode != LDPC_I8) continue;
    cudaError_t e = cudaFuncSetAttribute(kernel_kind(mode, kind), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kMaxSmem);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t decode_occupancy(int mode, int kind, int block, int smem, int* blocks_per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, kernel_kind(mode, kind), block, smem);
}

cudaError_t launch_decode(int mode, int kind, dim3 grid, dim3 block, int smem, cudaStream_t st,
                          const DecodeArgs& a) {
  void* args[] = {const_cast<DecodeArgs*>(&a)};
  return cudaLaunchKernel(kernel_kind(mode, kind), grid, block, args, static_cast<size_t>(smem), st);
}

}  // namespace ldpcgb
