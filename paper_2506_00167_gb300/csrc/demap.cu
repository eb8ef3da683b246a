// Puncture flushing + max-log soft demapping + rate dematching on sm_103a.
//
// The receiver sets the LLRs of bits carried by URLLC-punctured resource
// elements to 0 after soft demodulation (paper Sec. IV "UE"); the
// demodulator itself is unstated there and this library uses max-log over
// NR-style Gray QAM.  Max-log is separable per axis for this constellation:
// the Q part of |y - s|^2 cancels in the difference for an I bit, so each
// LLR is a minimum over the 2^(Qm/2) PAM levels of one axis.
//
// One thread per resource element: one 8-byte symbol load, Qm LLRs, each
// written to its interleaved codeword position t0 + i * (E/Qm) + r -- for a
// fixed bit plane i consecutive threads write consecutive positions, so every
// store is coalesced.  The first tile of each block also zero-fills the
// positions never transmitted.
#include "internal.cuh"

namespace ldpcgb {

namespace {

// Unnormalised recursive Gray PAM amplitude of per-axis label c (q bits, the
// first label bit is the most significant bit of c).
constexpr int pam_amp(int c, int q) {
  int sign = ((c >> (q - 1)) & 1) ? -1 : 1;
  if (q == 1) return sign;
  return sign * ((1 << (q - 1)) - pam_amp(c & ((1 << (q - 1)) - 1), q - 1));
}

struct PamTable {
  float v[5][16];
};

constexpr PamTable make_pam() {
  PamTable t{};
  const float norm[5] = {0.f, 1.4142135623730951f, 3.1622776601683795f, 6.48074069840786f, 13.038404810405298f};
  for (int q = 1; q <= 4; ++q)
    for (int c = 0; c < (1 << q); ++c) t.v[q][c] = static_cast<float>(pam_amp(c, q)) / norm[q];
  return t;
}

__constant__ PamTable kPam = make_pam();

// Max-log LLRs of the q bits of one axis, written to out[2t + off].
template <int q>
__device__ __forceinline__ void axis_llr(float y, float inv_s2, float* out, int off) {
  float m0[q], m1[q];
#pragma unroll
  for (int t = 0; t < q; ++t) {
    m0[t] = 3.0e38f;
    m1[t] = 3.0e38f;
  }
#pragma unroll
  for (int c = 0; c < (1 << q); ++c) {
    const float d = y - kPam.v[q][c];
    const float d2 = d * d;
#pragma unroll
    for (int t = 0; t < q; ++t) {
      if ((c >> (q - 1 - t)) & 1)
        m1[t] = fminf(m1[t], d2);
      else
        m0[t] = fminf(m0[t], d2);
    }
  }
#pragma unroll
  for (int t = 0; t < q; ++t) out[2 * t + off] = (m1[t] - m0[t]) * inv_s2;
}

template <typename LT>
__device__ __forceinline__ LT to_llr(float lam, float q_scale, float sat) {
  if constexpr (sizeof(LT) == 4) {
    return lam;
  } else {
    float x = roundf(lam * q_scale);  // round half away from zero
    x = fminf(fmaxf(x, -sat), sat);
    return static_cast<LT>(__float2int_rn(x));
  }
}

template <typename LT, int Qm>
__device__ __forceinline__ void demap_re(const DemapArgs& a, const CbDev& cb, int r) {
  const float2 y = a.sym[cb.re_off + r];
  const bool punct = (a.mask[cb.mask_off + (r >> 5)] >> (r & 31)) & 1u;
  float lam[Qm];
  axis_llr<Qm / 2>(y.x, cb.inv_sigma2, lam, 0);
  axis_llr<Qm / 2>(y.y, cb.inv_sigma2, lam, 1);
  LT* out = static_cast<LT*>(a.llr) + cb.llr_off + cb.t0;
#pragma unroll
  for (int i = 0; i < Qm; ++i) {
    const LT v = punct ? LT(0) : to_llr<LT>(lam[i], a.q_scale, a.llr_sat);
    const int pos = a.interleave ? i * cb.n_re + r : r * Qm + i;
    out[pos] = v;
  }
}

template <typename LT>
__global__ void __launch_bounds__(kDemapBlock) demap_kernel(const DemapArgs a) {
  const DemapTile tile = a.tiles[blockIdx.x];
  const CbDev cb = a.cbs[tile.cb];
  const int r = tile.re_start + threadIdx.x;
  if (r < cb.n_re) {
    switch (cb.Qm) {
      case 2: demap_re<LT, 2>(a, cb, r); break;
      case 4: demap_re<LT, 4>(a, cb, r); break;
      case 6: demap_re<LT, 6>(a, cb, r); break;
      default: demap_re<LT, 8>(a, cb, r); break;
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
