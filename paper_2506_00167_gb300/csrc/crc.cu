// Transport-block CRC-24 check, goodput and reward on sm_103a.
//
// d_e = 1 iff the TB's decoded (A + 24) bits are a multiple of g(x) (register
// from 0, first bit = highest degree): the same test as comparing the CRC
// recomputed from the received payload with the received CRC (paper Sec. VI-D
// "UE Feedback").  Per slot: goodput_sc = sum_e d_e n_e (Sec. III-B, eq. 1),
// reward = (1/N) sum_e (d_e - 1) n_e (Sec. V-A, eq. 2), and the delivered
// payload bits.
//
// One block per slot, one warp per TB.  A TB of W words is split into 32
// contiguous segments; each lane runs its segment through a byte-table LFSR
// from state 0, giving seg(x) * x^24 mod g, then shifts it into place by one
// GF(2) multiply with x^(32 * words after the segment) mod g (a per-batch
// table) and the warp xor-reduces.  No atomics: the block reduces the slot's
// sums in shared memory, so results are deterministic.
#include "crc_core.cuh"

namespace ldpcgb {

namespace {

using namespace crccore;

__global__ void __launch_bounds__(kCrcBlock) tb_crc_goodput_kernel(const CrcArgs a) {
  __shared__ uint32_t s_tab[256];
  __shared__ unsigned long long s_gb[kCrcBlock / 32];
  __shared__ uint32_t s_gs[kCrcBlock / 32];
  __shared__ uint32_t s_fail[kCrcBlock / 32];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) s_tab[i] = a.crc_table[i];
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
    const int W = tb.words;
    const int per = (W + 31) >> 5;
    const int w0 = min(W, lane * per);
    const int w1 = min(W, w0 + per);
    uint32_t state = 0;
    if (w0 < w1) {
      // find the code block holding TB word w0
      int cbi = tb.first_cb;
      int cb_first = 0;
      int cb_words = (a.cbs[cbi].kb * a.cbs[cbi].Z) >> 5;
      while (w0 >= cb_first + cb_words) {
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
        const uint32_t v = __brev(src[w - cb_first]);  // bit 31 = first bit in time
#pragma unroll
        for (int b = 3; b >= 0; --b) {
          const uint32_t byte = (v >> (8 * b)) & 0xFFu;
          state = ((state << 8) & 0xFFFFFFu) ^ s_tab[((state >> 16) ^ byte) & 0xFFu];
        }
      }
      state = gf2_mulmod(state, a.xpow32[W - w1]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) state ^= __shfl_xor_sync(0xFFFFFFFFu, state, o);
    const uint32_t d = state == 0u ? 1u : 0u;
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
