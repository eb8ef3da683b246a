// Transport-block CRC-24 check, goodput and reward on sm_103a.
//
// d_e = 1 iff the TB's decoded (A + 24) bits are a multiple of g(x) (register
// from 0, first bit = highest degree): the same test as comparing the CRC
// recomputed from the received payload with the received CRC (paper Sec. VI-D
// "UE Feedback").  Per slot: goodput_sc = sum_e d_e n_e (Sec. III-B, eq. 1),
// reward = (1/N) sum_e (d_e - 1) n_e (Sec. V-A, eq. 2), and the delivered
// payload bits.
//
// A segmented TB (every block with LDPC_CB_CRC24B) runs its CRC over each
// block's first K - 24 bits only, and each block's K bits must also be a
// multiple of g_B(x): d_e needs every check to pass.
//
// One block per slot, one warp per TB.  The TB's blocks' words, back to
// back, are split into 32 runs of whole words; each lane runs the TB bytes of
// its run (all four of a word, one of a segmented block's last word) through
// a byte-table LFSR from state 0, giving seg(x) * x^24 mod g, shifts it into
// place -- times x^(8 * TB bytes after the run) mod g: one GF(2) multiply by
// x^(32 m) from a per-batch table, then a zero byte per remaining byte -- and
// the warp xor-reduces.  A block's own CRC is the same over its K / 32 words
// with g_B's tables.  No atomics: the block reduces the slot's sums in shared
// memory, so results are deterministic.
#include "crc_core.cuh"

namespace ldpcgb {

namespace {

using namespace crccore;

// TB bytes carried by one code block.
__device__ __forceinline__ int tb_bytes_of(const CbDev& c, int seg) { return ((c.kb * c.Z) >> 3) - 3 * seg; }

__device__ __forceinline__ uint32_t warp_xor(uint32_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v ^= __shfl_xor_sync(0xFFFFFFFFu, v, o);
  return v;
}

__global__ void __launch_bounds__(kCrcBlock) tb_crc_goodput_kernel(const CrcArgs a) {
  __shared__ uint32_t s_tab[256];
  __shared__ uint32_t s_tab_b[256];
  __shared__ unsigned long long s_gb[kCrcBlock / 32];
  __shared__ uint32_t s_gs[kCrcBlock / 32];
  __shared__ uint32_t s_fail[kCrcBlock / 32];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) {
    s_tab[i] = a.crc_table[i];
    s_tab_b[i] = a.crc_table_b[i];
  }
  __syncthreads();

  const int slot = blockIdx.x;
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int t0 = a.slot_start[slot];
  const int t1 = a.slot_start[slot + 1];
  unsigned long long gb = 0;
  uint32_t gs = 0, fail = 0;

  for (int i = t0 + warp; i < t1; i += kCrcBlock / 32) {
    const TbDev tb = a.tbs[a.slot_tbs[i]];
    // the TB's blocks' words back to back, W in all; the last word of a block
    // with its own CRC holds one TB byte (its other three are that CRC)
    int W = 0;
    for (int c = tb.first_cb; c < tb.first_cb + tb.n_cb; ++c) W += (a.cbs[c].kb * a.cbs[c].Z) >> 5;
    const int per = (W + 31) >> 5;
    const int w0 = min(W, lane * per);
    const int w1 = min(W, w0 + per);
    uint32_t state = 0;
    int after = 0;  // TB bytes after this lane's words
    {
      int cbi = tb.first_cb;
      int cb_first = 0;
      int cb_words = (a.cbs[cbi].kb * a.cbs[cbi].Z) >> 5;
      while (w0 >= cb_first + cb_words && cbi + 1 < tb.first_cb + tb.n_cb) {
        cb_first += cb_words;
        ++cbi;
        cb_words = (a.cbs[cbi].kb * a.cbs[cbi].Z) >> 5;
      }
      const uint32_t* src = a.bits + a.cbs[cbi].bits_off;
      for (int w = w0; w < w1; ++w) {
        if (w >= cb_first + cb_words) {
          cb_first += cb_words;
          ++cbi;
          cb_words = (a.cbs[cbi].kb * a.cbs[cbi].Z) >> 5;
          src = a.bits + a.cbs[cbi].bits_off;
        }
        const uint32_t v = src[w - cb_first];
        const int nbytes = (tb.seg && w == cb_first + cb_words - 1) ? 1 : 4;
        for (int j = 0; j < nbytes; ++j) state = crc_byte_step(state, msb_first_byte(v, j), s_tab);
      }
      // TB bytes after word w1: the rest of block cbi, then whole blocks
      if (w1 < cb_first + cb_words) after = 4 * (cb_first + cb_words - w1) - 3 * tb.seg;
      for (int c = cbi + 1; c < tb.first_cb + tb.n_cb; ++c) after += tb_bytes_of(a.cbs[c], tb.seg);
    }
    if (w0 < w1) {
      // times x^(8 * after): x^(32 * (after / 4)) by table, then one zero byte per remaining byte
      state = gf2_mulmod(state, a.xpow32[after >> 2]);
      for (int j = 0; j < (after & 3); ++j) state = crc_byte_step(state, 0u, s_tab);
    }
    uint32_t d = warp_xor(state) == 0u ? 1u : 0u;
    if (tb.seg) {
      for (int c = tb.first_cb; c < tb.first_cb + tb.n_cb; ++c) {
        const CbDev cb = a.cbs[c];
        const int Wc = (cb.kb * cb.Z) >> 5;
        const int pc = (Wc + 31) >> 5;
        const int v0 = min(Wc, lane * pc);
        const int v1 = min(Wc, v0 + pc);
        const uint32_t* src = a.bits + cb.bits_off;
        uint32_t st = 0;
        for (int w = v0; w < v1; ++w) {
          const uint32_t v = src[w];
#pragma unroll
          for (int j = 0; j < 4; ++j) st = crc_byte_step(st, msb_first_byte(v, j), s_tab_b);
        }
        if (v0 < v1) st = gf2_mulmod(st, a.xpow32_b[Wc - v1], kPolyFullB);
        if (warp_xor(st) != 0u) d = 0u;
      }
    }
    if (lane == 0) {
      a.d[a.slot_tbs[i]] = static_cast<uint8_t>(d);
      gb += d * static_cast<unsigned long long>(tb.payload_bits);
      gs += d * static_cast<uint32_t>(tb.n_sc);
      fail += (1u - d) * static_cast<uint32_t>(tb.n_sc);
    }
  }
  if (lane == 0) {
    s_gb[warp] = gb;
    s_gs[warp] = gs;
    s_fail[warp] = fail;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long tgb = 0;
    uint32_t tgs = 0, tf = 0;
    for (int w = 0; w < kCrcBlock / 32; ++w) {
      tgb += s_gb[w];
      tgs += s_gs[w];
      tf += s_fail[w];
    }
    a.goodput_bits[slot] = tgb;
    a.goodput_sc[slot] = tgs;
    a.reward[slot] = -static_cast<float>(tf) / static_cast<float>(a.slot_N[slot]);
  }
}

}  // namespace

cudaError_t launch_crc(int n_slots, cudaStream_t st, const CrcArgs& a) {
  if (n_slots == 0) return cudaSuccess;
  void* args[] = {const_cast<CrcArgs*>(&a)};
  return cudaLaunchKernel(reinterpret_cast<const void*>(&tb_crc_goodput_kernel), dim3(n_slots), dim3(kCrcBlock),
                          args, 0, st);
}

}  // namespace ldpcgb
