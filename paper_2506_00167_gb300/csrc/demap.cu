// Puncture flushing + max-log soft demapping + rate dematching on sm_103a.
//
// The receiver sets the LLRs of bits carried by URLLC-punctured resource
// elements to 0 after soft demodulation (paper Sec. VI-D "UE"); the
// demodulator itself is unstated there and this library uses max-log over
// NR-style Gray QAM.  Max-log is separable per axis for this constellation:
// the Q part of |y - s|^2 cancels in the difference for an I bit, so each
// LLR is a minimum over the 2^(Qm/2) PAM levels of one axis.
//
// A block covers a tile of kDemapTile resource elements of one code block,
// each thread kDemapPerThread of them, kDemapBlock apart: all of a thread's
// symbol and mask-word loads are issued before any arithmetic, so enough
// bytes are in flight per SM to keep HBM busy.  Each resource element gives
// Qm LLRs, written to its interleaved codeword position t0 + i * (E/Qm) + r
// (offset by the redundancy version's start k0, modulo the buffer) -- for a
// fixed bit plane i consecutive threads write consecutive positions, so every
// store is coalesced but at the buffer's wrap point.  The first tile of each
// code block also zero-fills the positions never transmitted.  When rate
// matching repeats the circular buffer (E > Ncb), this kernel writes the
// first pass and demap_repeat_kernel then rewrites the repeated positions
// with the sum of their two LLRs.
#include "demap_core.cuh"

namespace ldpcgb {

namespace {

using namespace demapcore;

template <typename LT>
__global__ void __launch_bounds__(kDemapBlock) demap_kernel(const DemapArgs a) {
  const DemapTile tile = a.tiles[blockIdx.x];
  const CbDev cb = a.cbs[tile.cb];
  float2 y[kDemapPerThread];
  uint32_t mw[kDemapPerThread];
#pragma unroll
  for (int u = 0; u < kDemapPerThread; ++u) {
    const int r = tile.re_start + u * kDemapBlock + static_cast<int>(threadIdx.x);
    if (r < cb.n_re) {
      y[u] = __ldcs(a.sym + cb.re_off + r);  // read once: streaming
      mw[u] = __ldg(a.mask + cb.mask_off + (r >> 5));
    }
  }
#pragma unroll
  for (int u = 0; u < kDemapPerThread; ++u) {
    const int r = tile.re_start + u * kDemapBlock + static_cast<int>(threadIdx.x);
    if (r < cb.n_re) {
      switch (cb.Qm) {
        case 2: demap_re<LT, 2>(a, cb, r, y[u], mw[u]); break;
        case 4: demap_re<LT, 4>(a, cb, r, y[u], mw[u]); break;
        case 6: demap_re<LT, 6>(a, cb, r, y[u], mw[u]); break;
        default: demap_re<LT, 8>(a, cb, r, y[u], mw[u]); break;
      }
    }
  }
  if (tile.re_start == 0) {  // positions never transmitted hold LLR 0
    LT* out = static_cast<LT*>(a.llr) + cb.llr_off;
    for (int p = threadIdx.x; p < cb.t0; p += blockDim.x) out[p] = LT(0);
    // buffer offsets k0 + j (mod Ncb) for j from E to Ncb: those the version does not reach
    const int ncb = cb.n_eff * cb.Z - cb.t0;
    for (int j = min(cb.E, ncb) + threadIdx.x; j < ncb; j += blockDim.x) {
      const int q = cb.k0 + j;
      out[cb.t0 + (q >= ncb ? q - ncb : q)] = LT(0);
    }
  }
}

// Repeated bits e2 in [Ncb, E) of a block whose rate matching wraps: buffer
// offset (k0 + e2) mod Ncb gets lambda(e2 - Ncb) + lambda(e2), one thread per
// repeated bit, after demap_kernel has written the first pass.
template <typename LT>
__global__ void __launch_bounds__(kDemapBlock) demap_repeat_kernel(const DemapArgs a) {
  const DemapTile tile = a.tiles[blockIdx.x];
  const CbDev cb = a.cbs[tile.cb];
  const int e2 = tile.re_start + static_cast<int>(threadIdx.x);
  if (e2 >= cb.E) return;
  const int ncb = cb.n_eff * cb.Z - cb.t0;
  const float2* sym = a.sym + cb.re_off;
  const uint32_t* msk = a.mask + cb.mask_off;
  auto ls = [&](int i) { return __ldg(sym + i); };
  auto lm = [&](int r) { return ((__ldg(msk + (r >> 5)) >> (r & 31)) & 1u) != 0u; };
  float v;
  switch (cb.Qm) {
    case 2: v = bit_llr<2>(e2 - ncb, cb.n_re, a.interleave, cb.inv_sigma2, ls, lm) +
                bit_llr<2>(e2, cb.n_re, a.interleave, cb.inv_sigma2, ls, lm); break;
    case 4: v = bit_llr<4>(e2 - ncb, cb.n_re, a.interleave, cb.inv_sigma2, ls, lm) +
                bit_llr<4>(e2, cb.n_re, a.interleave, cb.inv_sigma2, ls, lm); break;
    case 6: v = bit_llr<6>(e2 - ncb, cb.n_re, a.interleave, cb.inv_sigma2, ls, lm) +
                bit_llr<6>(e2, cb.n_re, a.interleave, cb.inv_sigma2, ls, lm); break;
    default: v = bit_llr<8>(e2 - ncb, cb.n_re, a.interleave, cb.inv_sigma2, ls, lm) +
                 bit_llr<8>(e2, cb.n_re, a.interleave, cb.inv_sigma2, ls, lm); break;
  }
  const int q = cb.k0 + e2 - ncb;  // the buffer offset both bits land on
  static_cast<LT*>(a.llr)[cb.llr_off + cb.t0 + (q >= ncb ? q - ncb : q)] = to_llr<LT>(v, a.q_scale, a.llr_sat);
}

}  // namespace

cudaError_t launch_demap_repeat(int mode, int n_tiles, cudaStream_t st, const DemapArgs& a) {
  if (n_tiles == 0) return cudaSuccess;
  void* args[] = {const_cast<DemapArgs*>(&a)};
  const void* fn = mode == LDPC_F32  ? reinterpret_cast<const void*>(&demap_repeat_kernel<float>)
                   : mode == LDPC_I8 ? reinterpret_cast<const void*>(&demap_repeat_kernel<int8_t>)
                                     : reinterpret_cast<const void*>(&demap_repeat_kernel<int16_t>);
  return cudaLaunchKernel(fn, dim3(n_tiles), dim3(kDemapBlock), args, 0, st);
}

cudaError_t launch_demap(int mode, int n_tiles, cudaStream_t st, const DemapArgs& a) {
  if (n_tiles == 0) return cudaSuccess;
  void* args[] = {const_cast<DemapArgs*>(&a)};
  const void* fn = mode == LDPC_F32  ? reinterpret_cast<const void*>(&demap_kernel<float>)
                   : mode == LDPC_I8 ? reinterpret_cast<const void*>(&demap_kernel<int8_t>)
                                     : reinterpret_cast<const void*>(&demap_kernel<int16_t>);
  return cudaLaunchKernel(fn, dim3(n_tiles), dim3(kDemapBlock), args, 0, st);
}

}  // namespace ldpcgb
