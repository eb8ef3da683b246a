// Device building blocks of the max-log demapper, shared by the batch
// demapper (demap.cu) and the serving loop's fused prologue (serve.cu).
#pragma once

#include "internal.cuh"

namespace ldpcgb {
namespace demapcore {

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

// Q: quantise (the integer modes); a float LT with Q holds the quantised
// integer as a float.
template <typename LT, bool Q = (sizeof(LT) < 4)>
__device__ __forceinline__ LT to_llr(float lam, float q_scale, float sat) {
  if constexpr (!Q) {
    return lam;
  } else {
    float x = roundf(lam * q_scale);  // round half away from zero
    x = fminf(fmaxf(x, -sat), sat);
    if constexpr (sizeof(LT) == 4)
      return x;
    else
      return static_cast<LT>(__float2int_rn(x));
  }
}

// Rate matching reads a circular buffer of the Ncb = nb * Z - t0 codeword
// positions from t0: rate-matched bit e lands on position
// t0 + ((k0 + e) mod Ncb), k0 the start of the redundancy version, so when
// E > Ncb the buffer repeats and the two LLRs of a position are added (LLR
// combining; E <= 2 Ncb).  The serving loop sends redundancy version 0 only
// (k0 = 0): there the thread that owns bit e < Ncb writes the position, adding
// the LLR of bit e + Ncb when it was sent; it demaps that bit's resource
// element itself, so each position is written once and the sum is always
// taken in the same order.

// Max-log LLR of rate-matched bit e (0 for a punctured resource element);
// ld_sym(r) loads the code block's symbol r, punct(r) tells whether resource
// element r is punctured.
template <int Qm, typename LoadSym, typename Punct>
__device__ __noinline__ float bit_llr(int e, int n_re, int interleave, float inv_sigma2, LoadSym ld_sym,
                                     Punct punct) {
  const int r = interleave ? e % n_re : e / Qm;
  const int i = interleave ? e / n_re : e % Qm;
  if (punct(r)) return 0.0f;
  const float2 y = ld_sym(r);
  float lam[Qm];
  axis_llr<Qm / 2>(y.x, inv_sigma2, lam, 0);
  axis_llr<Qm / 2>(y.y, inv_sigma2, lam, 1);
  float v = lam[0];
#pragma unroll
  for (int t = 1; t < Qm; ++t)
    if (t == i) v = lam[t];
  return v;
}

// Resource element r of a code block (symbol y, punctured or not) into its
// codeword positions, `out` pointing at the block's position t0: bit e of the
// rate-matched stream lands on buffer offset (k0 + e) mod Ncb, and a bit
// repeated at e + Ncb (E > Ncb) is added there by the owner of e.
// `out` is an LT* or any type whose out[e] takes an LT.
template <typename LT, int Qm, bool Q = (sizeof(LT) < 4), typename Out, typename LoadSym, typename Punct>
__device__ __forceinline__ void demap_re_into(float2 y, bool punct, float inv_sigma2, Out out, int r, int n_re,
                                              int E, int ncb, int k0, int interleave, float q_scale,
                                              float llr_sat, LoadSym ld_sym, Punct punct_of) {
  float lam[Qm];
  axis_llr<Qm / 2>(y.x, inv_sigma2, lam, 0);
  axis_llr<Qm / 2>(y.y, inv_sigma2, lam, 1);
#pragma unroll
  for (int i = 0; i < Qm; ++i) {
    const int e = interleave ? i * n_re + r : r * Qm + i;
    if (e >= ncb) continue;  // a repetition: added by the owner of e - ncb
    float v = punct ? 0.0f : lam[i];
    if (e + ncb < E) v += bit_llr<Qm>(e + ncb, n_re, interleave, inv_sigma2, ld_sym, punct_of);
    const int q = k0 + e;  // the redundancy version's buffer offset
    out[q >= ncb ? q - ncb : q] = to_llr<LT, Q>(v, q_scale, llr_sat);
  }
}

// Batch form: writes the first pass over the circular buffer only; the
// positions that also received a repetition are rewritten with the combined
// LLR by a second kernel (demap.cu), so this hot loop carries no repetition
// work.  Bit e < Ncb lands on buffer offset (k0 + e) mod Ncb: k0 is the start
// of the redundancy version.  Here Ncb is taken as n_eff * Z - t0, which is
// the buffer's length whenever the bits sent wrap it and otherwise covers
// every offset sent, so the offsets agree.
template <typename LT, int Qm>
__device__ __forceinline__ void demap_re(const DemapArgs& a, const CbDev& cb, int r, float2 y, uint32_t mask_word) {
  const bool punct = (mask_word >> (r & 31)) & 1u;
  float lam[Qm];
  axis_llr<Qm / 2>(y.x, cb.inv_sigma2, lam, 0);
  axis_llr<Qm / 2>(y.y, cb.inv_sigma2, lam, 1);
  LT* out = static_cast<LT*>(a.llr) + cb.llr_off + cb.t0;
  const int ncb = cb.n_eff * cb.Z - cb.t0;
#pragma unroll
  for (int i = 0; i < Qm; ++i) {
    const int e = a.interleave ? i * cb.n_re + r : r * Qm + i;
    int q = cb.k0 + e;
    q = q >= ncb ? q - ncb : q;
    if (e < ncb) out[q] = punct ? LT(0) : to_llr<LT>(lam[i], a.q_scale, a.llr_sat);
  }
}

}  // namespace demapcore
}  // namespace ldpcgb
