// Device building blocks of the layered offset-min-sum decoder, shared by
// the batch decoder (decode.cu) and the serving loop (serve.cu).  See
// decode.cu for the algorithm and its mapping onto the SM.
#pragma once

#include "internal.cuh"

namespace ldpcgb {
namespace core {

// Small integers move between int8/int16/uint8/uint16 storage and float
// registers by adding the bit pattern of 1.5 * 2^23 (exact for |x| < 2^22):
// two full-rate ALU/FMA ops instead of a conversion-unit round trip.
constexpr float kMagicF = 12582912.0f;  // 1.5 * 2^23
constexpr int kMagicI = 0x4B400000;     // its bit pattern
constexpr float kBigF = 1.0e30f;        // FP32 dummy posterior: never a minimum

template <typename T>
__device__ __forceinline__ float ld_val(const T* p, int i) {
  if constexpr (sizeof(T) == 4) {
    return static_cast<float>(p[i]);
  } else {
    return __int_as_float(static_cast<int>(p[i]) + kMagicI) - kMagicF;
  }
}

__device__ __forceinline__ int f2i_exact(float v) { return __float_as_int(v + kMagicF) - kMagicI; }

template <typename T>
__device__ __forceinline__ void st_val(T* p, int i, float v) {
  if constexpr (sizeof(T) == 4) {
    p[i] = v;
  } else {
    p[i] = static_cast<T>(f2i_exact(v));  // v is an exact integer
  }
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

// (k + s) mod Z for 0 <= k, s < Z: the unsigned minimum of k + s and k + s - Z.
__device__ __forceinline__ int rot(int k, uint32_t s, int Z) {
  const uint32_t t = static_cast<uint32_t>(k) + s;
  return static_cast<int>(umin(t, t - static_cast<uint32_t>(Z)));
}

// One lifted check (l, k) of a row with `deg` edges, chunk c's column bases
// at tab[8c .. 8c+3] and shifts at tab[8c+4 .. 8c+7].  Reads the compressed
// messages, runs both passes, writes the posteriors and new messages.
// Stored sign bits: edge j at bit deg-1-j; argmin edge in bits 27..31.
template <typename LT, typename MT, bool SAT>
__device__ __forceinline__ void check_update(const uint32_t* __restrict__ tab, int deg, int k, int Z,
                                             LT* __restrict__ L, MT* __restrict__ mag1, MT* __restrict__ mag2,
                                             uint32_t* __restrict__ meta, int rec, int dummy, float beta,
                                             float msg_sat, float post_sat) {
  // integer modes: the dummy slot is reset to +post_sat so a padding edge's
  // |Q| saturates at msg_sat and (edge index larger) never beats a real edge;
  // float: 1e30 absorbs every update and needs no reset
  if constexpr (SAT) st_val(L, dummy, post_sat);
  const float r1 = ld_val(mag1, rec);
  const float r2 = ld_val(mag2, rec);
  const uint32_t mo = meta[rec];
  const int idx_o = static_cast<int>(mo >> 27);
  // edge 0's sign at bit 31; positions past deg read as negative, so padding
  // edges see Q = dummy + |R| (large and positive)
  uint32_t sgn = (mo << (32 - deg)) | ((1u << (32 - deg)) - 1u);
  const int nch = (deg + 3) >> 2;

  float q[kMaxChunks * 4];
  int addr[kMaxChunks * 4];
  float min1 = 3.0e38f, min2 = 3.0e38f;  // SAT modes: keys |Q| * 32 + j
  uint32_t par = 0;
#pragma unroll
  for (int c = 0; c < kMaxChunks; ++c) {
    if (c >= nch) break;
    const uint4 B = *reinterpret_cast<const uint4*>(tab + 8 * c);
    const uint4 S = *reinterpret_cast<const uint4*>(tab + 8 * c + 4);
    addr[4 * c + 0] = static_cast<int>(B.x) + rot(k, S.x, Z);
    addr[4 * c + 1] = static_cast<int>(B.y) + rot(k, S.y, Z);
    addr[4 * c + 2] = static_cast<int>(B.z) + rot(k, S.z, Z);
    addr[4 * c + 3] = static_cast<int>(B.w) + rot(k, S.w, Z);
    float lv[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) lv[i] = ld_val(L, addr[4 * c + i]);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int j = 4 * c + i;
      const float m = (j == idx_o) ? r2 : r1;
      const float r = __uint_as_float(__float_as_uint(m) | (sgn & 0x80000000u));
      sgn <<= 1;
      float Q = lv[i] - r;
      if (SAT) Q = fminf(fmaxf(Q, -post_sat), post_sat);
      q[j] = Q;
      par ^= __float_as_uint(Q);
      float a = fabsf(Q);
      if (SAT) a = fmaf(fminf(a, msg_sat), 32.0f, static_cast<float>(j));
      min2 = fminf(min2, fmaxf(min1, a));
      min1 = fminf(min1, a);
    }
  }
  float n1, n2;
  int idx = 0;
  if (SAT) {
    const int k1 = f2i_exact(min1);
    idx = k1 & 31;
    n1 = fmaxf(static_cast<float>(k1 >> 5) - beta, 0.0f);
    n2 = fmaxf(static_cast<float>(f2i_exact(min2) >> 5) - beta, 0.0f);
  } else {
    n1 = fmaxf(min1 - beta, 0.0f);
    n2 = fmaxf(min2 - beta, 0.0f);
  }
  const uint32_t pm = par & 0x80000000u;
  uint32_t rs = 0;
#pragma unroll
  for (int c = 0; c < kMaxChunks; ++c) {
    if (c >= nch) break;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int j = 4 * c + i;
      bool is_min;
      if (SAT) {
        is_min = (j == idx);
      } else {
        is_min = (fabsf(q[j]) == min1);
        idx = is_min ? j : idx;
      }
      const float m = is_min ? n2 : n1;
      // sign of R'_j = parity of the other edges' signs = parity ^ sign(Q_j)
      const uint32_t rb = __float_as_uint(m) | ((__float_as_uint(q[j]) ^ pm) & 0x80000000u);
      float v = q[j] + __uint_as_float(rb);
      if (SAT) v = fminf(fmaxf(v, -post_sat), post_sat);
      st_val(L, addr[j], v);  // padding edges write the dummy slot
      rs = __funnelshift_l(rb, rs, 1);
    }
  }
  rs >>= 4 * nch - deg;  // drop the padding edges' bits
  st_val(mag1, rec, n1);
  st_val(mag2, rec, n2);
  meta[rec] = rs | (static_cast<uint32_t>(idx) << 27);
}

// Edge e of a row whose chunks start at `tab`: (column base, shift).
__device__ __forceinline__ uint2 edge_at(const uint32_t* tab, int e) {
  const int c = e >> 2, i = e & 3;
  return make_uint2(tab[8 * c + i], tab[8 * c + 4 + i]);
}

// Z % 32 == 0: hard decisions of all n_eff columns into the bitmap hb
// (column c, word w holds checks 32w..32w+31), one ballot per warp and column.
template <typename LT>
__device__ __forceinline__ void hard_bitmap(const LT* __restrict__ L, uint32_t* __restrict__ hb, int n_eff, int k,
                                            int Z) {
  const int W = Z >> 5;
  const int w = k >> 5;
  const bool lane0 = (k & 31) == 0;
  for (int c = 0; c < n_eff; ++c) {
    const uint32_t b = __ballot_sync(0xFFFFFFFFu, L[c * Z + k] < LT(0));
    if (lane0) hb[c * W + w] = b;
  }
}

// Z % 32 == 0: is any of this thread's (row, word) syndrome words nonzero?
// Row l's syndrome is XOR_j rot(hb[c_j], s_j); word ww of rot(B, s) is the
// funnel shift of words ww + s/32 and ww + s/32 + 1 (mod Z/32) by s % 32.
__device__ __forceinline__ bool syndrome_bitmap(const uint32_t* __restrict__ tab, const uint32_t* __restrict__ rows,
                                                const uint32_t* __restrict__ hb, int m_eff, int k, int Z) {
  const int W = Z >> 5;
  uint32_t bad = 0;
  for (int task = k; task < m_eff * W; task += Z) {
    const int l = task / W;
    const int ww = task - l * W;
    const uint32_t info = rows[l];
    const uint32_t* rt = tab + (info & 0xFFFFu);
    const int deg = static_cast<int>(info >> 16);
    uint32_t x = 0;
    for (int e = 0; e < deg; ++e) {
      const uint2 bs = edge_at(rt, e);
      const int s = static_cast<int>(bs.y);
      const uint32_t* col = hb + (bs.x >> 5);
      int i0 = ww + (s >> 5);
      i0 = (i0 >= W) ? i0 - W : i0;
      const int i1 = (i0 + 1 == W) ? 0 : i0 + 1;
      x ^= __funnelshift_r(col[i0], col[i1], s & 31);
    }
    bad |= x;
  }
  return bad != 0;
}

// Z < 32 (Z = 16): parity of this thread's check in every decoded row.
template <typename LT>
__device__ __forceinline__ bool syndrome_direct(const uint32_t* __restrict__ tab, const uint32_t* __restrict__ rows,
                                                int m_eff, int k, int Z, const LT* __restrict__ L) {
  uint32_t bad = 0;
  for (int l = 0; l < m_eff; ++l) {
    const uint32_t info = rows[l];
    const uint32_t* rt = tab + (info & 0xFFFFu);
    const int deg = static_cast<int>(info >> 16);
    uint32_t p = 0;
    for (int e = 0; e < deg; ++e) {
      const uint2 bs = edge_at(rt, e);
      p ^= (L[static_cast<int>(bs.x) + rot(k, bs.y, Z)] < LT(0)) ? 1u : 0u;
    }
    bad |= p;
  }
  return bad != 0;
}

}  // namespace core
}  // namespace ldpcgb
