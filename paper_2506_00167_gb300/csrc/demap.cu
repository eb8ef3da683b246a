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
// Qm LLRs, written to its interleaved codeword position t0 + i * (E/Qm) + r --
// for a fixed bit plane i consecutive threads write consecutive positions, so
// every store is coalesced.  The first tile of each code block also
// zero-fills the positions never transmitted.
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
    const int tail0 = cb.t0 + cb.E;
    const int n = cb.n_eff * cb.Z;
    for (int p = tail0 + threadIdx.x; p < n; p += blockDim.x) out[p] = LT(0);
  }
}

}  // namespace

cudaError_t launch_demap(int mode, int n_tiles, cudaStream_t st, const DemapArgs& a) {
  if (n_tiles == 0) return cudaSuccess;
  void* args[] = {const_cast<DemapArgs*>(&a)};
  const void* fn = mode == LDPC_F32  ? reinterpret_cast<const void*>(&demap_kernel<float>)
                   : mode == LDPC_I8 ? reinterpret_cast<const void*>(&demap_kernel<int8_t>)
                                     : reinterpret_cast<const void*>(&demap_kernel<int16_t>);
  return cudaLaunchKernel(fn, dim3(n_tiles), dim3(kDemapBlock), args, 0, st);
}

}  // namespace ldpcgb
