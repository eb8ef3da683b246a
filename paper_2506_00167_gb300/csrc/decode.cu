// Layered offset-min-sum decoding of QC-LDPC code blocks on sm_103a.
//
// Algorithm (the paper's receiver decodes with a toolbox LDPC decoder and
// states no algorithm, Sec. IV "UE"; this library fixes layered offset min-sum):
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
//   distinct banks (Z a multiple of 32) and the shift costs no instruction
//   beyond the address add;
// * the shape's edge table and every group's channel LLRs are staged into
//   shared memory by bulk (TMA-engine) copies completing on one mbarrier;
// * check-to-variable messages are stored compressed per check: the two
//   smallest offset magnitudes, the argmin edge and one sign bit per edge
//   (12 bytes FP32, 6 bytes INT8, 8 bytes INT16 per check) -- in shared
//   memory, or in a global scratch slot per resident group when the shape
//   does not fit (RGLOBAL);
// * layers are separated by a named barrier per group (a warp sync for
//   Z <= 32); the syndrome test ORs every thread's parity with bar.red.or;
// * the information bits are packed by warp ballot straight from shared
//   memory into the caller's output words.
#include "internal.cuh"

namespace ldpcgb {

namespace {

template <typename LT>
__device__ __forceinline__ float load_l(const LT* L, int i) {
  return static_cast<float>(L[i]);
}

template <typename LT>
__device__ __forceinline__ void store_l(LT* L, int i, float v) {
  if constexpr (sizeof(LT) == 4)
    L[i] = v;
  else
    L[i] = static_cast<LT>(__float2int_rn(v));  // v is an exact integer
}

template <typename MT>
__device__ __forceinline__ void store_m(MT* M, int i, float v) {
  if constexpr (sizeof(MT) == 4)
    M[i] = v;
  else
    M[i] = static_cast<MT>(__float2int_rn(v));
}

// Group-wide barrier: a warp-level sync for Z <= 32, else named barrier 1 + g.
__device__ __forceinline__ void group_sync(int Z, int g, uint32_t wmask) {
  if (Z <= 32)
    __syncwarp(wmask);
  else
    named_bar_sync(1 + g, Z);
}

__device__ __forceinline__ bool group_any(int Z, int g, uint32_t wmask, bool pred) {
  if (Z <= 32) {
    __syncwarp(wmask);
    return __any_sync(wmask, pred);
  }
  return named_bar_or(1 + g, Z, pred);
}

// One lifted check (l, k): read the compressed messages, run both passes,
// write the posteriors and the new compressed messages.
template <typename LT, typename MT, bool SAT>
__device__ __forceinline__ void check_update(const uint32_t* __restrict__ tab, int e0, int deg, int k, int Z,
                                             LT* __restrict__ L, MT* __restrict__ mag1, MT* __restrict__ mag2,
                                             uint32_t* __restrict__ meta, int rec, float beta, float msg_sat,
                                             float post_sat) {
  const float r1 = static_cast<float>(mag1[rec]);
  const float r2 = static_cast<float>(mag2[rec]);
  const uint32_t mo = meta[rec];
  const int idx_o = static_cast<int>(mo >> 27);

  float q[kMaxDeg];
  int addr[kMaxDeg];
  float min1 = 3.0e38f, min2 = 3.0e38f;
  int idx = 0;
  uint32_t sg = 0;
#pragma unroll
  for (int j = 0; j < kMaxDeg; ++j) {
    if (j < deg) {
      const uint32_t e = tab[e0 + j];
      int t = k + static_cast<int>(e >> 16);
      t = (t >= Z) ? t - Z : t;
      addr[j] = static_cast<int>(e & 0xFFFFu) + t;
      float r = (j == idx_o) ? r2 : r1;
      r = ((mo >> j) & 1u) ? -r : r;
      float Q = load_l(L, addr[j]) - r;
      if (SAT) Q = fminf(fmaxf(Q, -post_sat), post_sat);
      q[j] = Q;
      float a = fabsf(Q);
      if (SAT) a = fminf(a, msg_sat);
      sg |= (Q < 0.0f ? 1u : 0u) << j;
      idx = (a < min1) ? j : idx;
      min2 = fminf(min2, fmaxf(min1, a));
      min1 = fminf(min1, a);
    }
  }
  const uint32_t par = __popc(sg) & 1u;
  const float n1 = fmaxf(min1 - beta, 0.0f);
  const float n2 = fmaxf(min2 - beta, 0.0f);
  const uint32_t rs = par ? ~sg : sg;  // bit j set: R'_j negative
#pragma unroll
  for (int j = 0; j < kMaxDeg; ++j) {
    if (j < deg) {
      float r = (j == idx) ? n2 : n1;
      r = ((rs >> j) & 1u) ? -r : r;
      float v = q[j] + r;
      if (SAT) v = fminf(fmaxf(v, -post_sat), post_sat);
      store_l(L, addr[j], v);
    }
  }
  store_m(mag1, rec, n1);
  store_m(mag2, rec, n2);
  meta[rec] = (rs & 0x07FFFFFFu) | (static_cast<uint32_t>(idx) << 27);
}

// Parity of this thread's checks in every decoded row: true if any is odd.
template <typename LT>
__device__ __forceinline__ bool syndrome_bad(const uint32_t* __restrict__ tab, const uint32_t* __restrict__ rows,
                                             int m_eff, int k, int Z, const LT* __restrict__ L) {
  uint32_t bad = 0;
  for (int l = 0; l < m_eff; ++l) {
    const int e0 = static_cast<int>(rows[l]);
    const int e1 = static_cast<int>(rows[l + 1]);
    uint32_t p = 0;
    for (int e = e0; e < e1; ++e) {
      const uint32_t w = tab[e];
      int t = k + static_cast<int>(w >> 16);
      t = (t >= Z) ? t - Z : t;
      p ^= (L[static_cast<int>(w & 0xFFFFu) + t] < LT(0)) ? 1u : 0u;
    }
    bad |= p;
  }
  return bad != 0;
}

template <typename LT, typename MT, bool SAT, bool RGLOBAL>
__global__ void __launch_bounds__(512) oms_decode_kernel(const DecodeArgs a) {
  extern __shared__ __align__(128) uint8_t smem[];
  uint32_t* s_tab = reinterpret_cast<uint32_t*>(smem);
  uint64_t* s_bar = reinterpret_cast<uint64_t*>(smem + a.hdr_bytes - 16);
  uint8_t* regions = smem + a.hdr_bytes;

  const int tid = threadIdx.x;
  const int Z = a.Z;
  const int g = tid / Z;
  const int k = tid - g * Z;
  const int lane = tid & 31;
  const uint32_t wmask = (Z >= 32) ? 0xFFFFFFFFu : (((1u << Z) - 1u) << (lane & ~(Z - 1)));

  if (tid == 0) {
    mbar_init(s_bar, 1);
    fence_proxy_async_smem();
  }
  __syncthreads();
  uint32_t phase = 0;

  for (int item_i = blockIdx.x; item_i < a.n_items; item_i += gridDim.x) {
    const DecodeItem item = a.items[item_i];
    const ShapeDev sh = a.shapes[item.shape];

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
        bulk_g2s(regions + gg * a.region_bytes, src, static_cast<uint32_t>(cb.n_eff * Z) * sizeof(LT), s_bar);
      }
    }

    const bool active = g < item.count;
    CbDev cb{};
    int cbi = 0;
    LT* L = reinterpret_cast<LT*>(regions + g * a.region_bytes);
    MT *mag1, *mag2;
    uint32_t* meta;
    if (RGLOBAL) {
      uint8_t* base = a.rscratch + (static_cast<int64_t>(blockIdx.x) * a.G + g) * a.rscratch_group;
      mag1 = reinterpret_cast<MT*>(base);
      mag2 = mag1 + a.rec_cap;
      meta = reinterpret_cast<uint32_t*>(base + 2 * ((a.rec_cap * sizeof(MT) + 15) & ~15));
    } else {
      uint8_t* base = regions + g * a.region_bytes + a.L_bytes;
      mag1 = reinterpret_cast<MT*>(base);
      mag2 = mag1 + a.rec_cap;
      meta = reinterpret_cast<uint32_t*>(base + 2 * ((a.rec_cap * sizeof(MT) + 15) & ~15));
    }
    if (active) {
      cbi = a.item_cbs[item.first + g];
      cb = a.cbs[cbi];
      // R = 0 before the first iteration (overlaps the copies in flight)
      for (int r = k; r < cb.m_eff * Z; r += Z) {
        mag1[r] = MT(0);
        mag2[r] = MT(0);
        meta[r] = 0u;
      }
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
      const uint32_t* tab = s_tab;
      const uint32_t* rows = s_tab + sh.row_off;
      const int m = cb.m_eff;
      int it = 1;
      bool ok = false;
      for (;; ++it) {
        for (int l = 0; l < m; ++l) {
          const int e0 = static_cast<int>(rows[l]);
          const int deg = static_cast<int>(rows[l + 1]) - e0;
          check_update<LT, MT, SAT>(tab, e0, deg, k, Z, L, mag1, mag2, meta, l * Z + k, a.beta, a.msg_sat,
                                    a.post_sat);
          group_sync(Z, g, wmask);
        }
        if (a.early_term || it == a.max_iter) {
          const bool bad = syndrome_bad(tab, rows, m, k, Z, L);
          ok = !group_any(Z, g, wmask, bad);
          if (ok && a.early_term) break;
          if (it == a.max_iter) break;
        }
      }
      // ---- hard decision of the kb information columns, packed by ballot
      const int kb = cb.kb;
      uint32_t* out = a.bits + cb.bits_off;
      if (Z >= 32) {
        const int wz = Z >> 5;
        const int w = k >> 5;
        for (int c = 0; c < kb; ++c) {
          const uint32_t b = __ballot_sync(0xFFFFFFFFu, L[c * Z + k] < LT(0));
          if (lane == 0) out[c * wz + w] = b;
        }
      } else {  // Z == 16: two columns per word, half a warp per block
        const int sh16 = lane & 16;
        for (int c = 0; c < kb; c += 2) {
          const uint32_t b0 = __ballot_sync(wmask, L[c * Z + k] < LT(0)) >> sh16;
          const uint32_t b1 = __ballot_sync(wmask, L[(c + 1) * Z + k] < LT(0)) >> sh16;
          if (k == 0) out[c >> 1] = (b0 & 0xFFFFu) | (b1 << 16);
        }
      }
      if (k == 0) a.status[cbi] = it | (ok ? (1 << 16) : 0);
    }
    __syncthreads();  // the next item's copies overwrite this item's shared memory
  }
}

template <bool RG>
const void* decode_kernel_ptr(int mode) {
  switch (mode) {
    case LDPC_F32: return reinterpret_cast<const void*>(&oms_decode_kernel<float, float, false, RG>);
    case LDPC_I8: return reinterpret_cast<const void*>(&oms_decode_kernel<int8_t, uint8_t, true, RG>);
    default: return reinterpret_cast<const void*>(&oms_decode_kernel<int16_t, uint16_t, true, RG>);
  }
}

const void* kernel_for(int mode, bool rglobal) {
  return rglobal ? decode_kernel_ptr<true>(mode) : decode_kernel_ptr<false>(mode);
}

}  // namespace

cudaError_t decode_prepare(int mode) {
  for (int rg = 0; rg < 2; ++rg) {
    cudaError_t e = cudaFuncSetAttribute(kernel_for(mode, rg != 0), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kMaxSmem);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t decode_occupancy(int mode, bool rglobal, int block, int smem, int* blocks_per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, kernel_for(mode, rglobal), block, smem);
}

cudaError_t launch_decode(int mode, bool rglobal, dim3 grid, dim3 block, int smem, cudaStream_t st,
                          const DecodeArgs& a) {
  void* args[] = {const_cast<DecodeArgs*>(&a)};
  return cudaLaunchKernel(kernel_for(mode, rglobal), grid, block, args, static_cast<size_t>(smem), st);
}

}  // namespace ldpcgb
