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

// (k + s) mod Z for 0 <= k, s < Z: the unsigned minimum of k + s and k + s - Z
// (k + s - Z wraps around when k + s < Z), as one fused add-and-minimum (DPX)
// on the sum.
__device__ __forceinline__ int rot(int k, uint32_t s, int Z) {
  const uint32_t t = static_cast<uint32_t>(k) + s;
  return static_cast<int>(__viaddmin_u32(t, 0u - static_cast<uint32_t>(Z), t));
}

// What a check update needs before it touches the posteriors: the row's edge
// table and degree, its first chunk of column bases and shifts, and this
// thread's compressed message record.  None of it is written by other threads
// during a layer, so the next row's copy is loaded before the layer barrier
// and only the posterior loads wait for it.
template <int CH>
struct Chunk {
  static_assert(CH == 2 || CH == 4, "edge-table chunks of 2 or 4 edges");
  uint32_t b[CH], s[CH];  // column bases, shifts
};

template <int CH>
__device__ __forceinline__ Chunk<CH> load_chunk(const uint32_t* tab, int c) {
  Chunk<CH> ch;
  if constexpr (CH == 2) {
    const uint4 v = *reinterpret_cast<const uint4*>(tab + 4 * c);
    ch.b[0] = v.x;
    ch.b[1] = v.y;
    ch.s[0] = v.z;
    ch.s[1] = v.w;
  } else {
    const uint4 B = *reinterpret_cast<const uint4*>(tab + 8 * c);
    const uint4 S = *reinterpret_cast<const uint4*>(tab + 8 * c + 4);
    ch.b[0] = B.x, ch.b[1] = B.y, ch.b[2] = B.z, ch.b[3] = B.w;
    ch.s[0] = S.x, ch.s[1] = S.y, ch.s[2] = S.z, ch.s[3] = S.w;
  }
  return ch;
}

template <int CH>
struct RowIn {
  const uint32_t* tab;
  int deg;
  Chunk<CH> c0;
  float r1, r2;
  uint32_t mo;
};

template <int CH, typename MT>
__device__ __forceinline__ RowIn<CH> load_row(const uint32_t* __restrict__ s_tab, uint32_t info,
                                              const MT* __restrict__ mag1, const MT* __restrict__ mag2,
                                              const uint32_t* __restrict__ meta, int rec) {
  RowIn<CH> r;
  r.tab = s_tab + (info & 0xFFFFu);
  r.deg = static_cast<int>(info >> 16);
  r.c0 = load_chunk<CH>(r.tab, 0);
  if constexpr (sizeof(MT) == 4) {  // float: both magnitudes in one 8-byte record
    const float2 rr = reinterpret_cast<const float2*>(mag1)[rec];
    r.r1 = rr.x;
    r.r2 = rr.y;
  } else {
    r.r1 = ld_val(mag1, rec);
    r.r2 = ld_val(mag2, rec);
  }
  r.mo = meta[rec];
  return r;
}

// Pass 1 for edge j at posterior slot a (value lv): Q_j = L - R_j, its sign
// into qs, |Q_j| (integer modes: the key |Q_j| * 32 + j) into the two minima.
template <typename LT, bool SAT, bool LEAN>
__device__ __forceinline__ float pass1_edge(LT* __restrict__ L, int a, float lv, int j, int idx_o, float r1,
                                            float r2, uint32_t& sgn, float& min1, float& min2, uint32_t& qs,
                                            float msg_sat, float post_sat) {
  const float m = (j == idx_o) ? r2 : r1;
  const float r = __uint_as_float(__float_as_uint(m) | (sgn & 0x80000000u));
  sgn <<= 1;
  float Q = lv - r;
  if (SAT) Q = fminf(fmaxf(Q, -post_sat), post_sat);
  if constexpr (LEAN) st_val(L, a, Q);  // Q waits in the posterior's slot for pass 2
  qs = __funnelshift_l(__float_as_uint(Q), qs, 1);
  float v = fabsf(Q);
  if (SAT) v = fmaf(fminf(v, msg_sat), 32.0f, static_cast<float>(j));
  min2 = fminf(min2, fmaxf(min1, v));
  min1 = fminf(min1, v);
  return Q;
}

// A posterior written into another CTA's replica (cluster decoder): `a` is a
// shared::cluster address from mapa.
template <typename LT>
__device__ __forceinline__ void st_cluster(uint32_t a, float v) {
  if constexpr (sizeof(LT) == 4) {
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
  } else if constexpr (sizeof(LT) == 2) {
    asm volatile("st.shared::cluster.b16 [%0], %1;" ::"r"(a), "h"(static_cast<unsigned short>(f2i_exact(v)))
                 : "memory");
  } else {
    asm volatile("st.shared::cluster.b8 [%0], %1;" ::"r"(a), "r"(f2i_exact(v)) : "memory");
  }
}

// Pass 2 for edge j: L = Q_j + R'_j, R'_j the other edges' minimum carrying
// the parity and Q_j's sign.  NREP > 1 (cluster decoder): the posterior is
// also written into the NREP - 1 other CTAs' replicas, whose shared::cluster
// base addresses are rep[0 .. NREP-2].
template <typename LT, bool SAT, int NREP = 1>
__device__ __forceinline__ void pass2_edge(LT* __restrict__ L, int a, float qv, int j, int& idx, float min1,
                                           float n1s, float n2s, float post_sat, const uint32_t* rep = nullptr) {
  bool is_min;
  if (SAT) {
    is_min = (j == idx);
  } else {
    is_min = (fabsf(qv) == min1);
    idx = is_min ? j : idx;
  }
  const float m = is_min ? n2s : n1s;
  const uint32_t rb = __float_as_uint(m) ^ (__float_as_uint(qv) & 0x80000000u);
  float v = qv + __uint_as_float(rb);
  if (SAT) v = fminf(fmaxf(v, -post_sat), post_sat);
  st_val(L, a, v);
  if constexpr (NREP > 1) {
#pragma unroll
    for (int r = 0; r < NREP - 1; ++r) st_cluster<LT>(rep[r] + static_cast<uint32_t>(a) * sizeof(LT), v);
  }
}

// One lifted check (l, k): row data in `in` (chunk c at tab[2 CH c ..]).
// Runs both passes, writes the posteriors and the new record.  The whole
// chunks run unrolled; the deg % CH edges of a last, partial chunk run
// after them (the table's padding entries are never touched).
//
// The record keeps the signs of the stored messages R_j (edge j at bit
// deg-1-j) and the argmin edge in bits 27..31.  R'_j carries the sign
// product over i != j, i.e. sign(Q_j) XOR the parity of all Q signs: the
// update collects the Q signs in pass 1, takes their parity with one
// popcount, and stores them XOR the parity, so the next update reads R_j's
// sign as it is.
//
// LEAN: pass 1 parks each Q_j in its posterior's slot (the check owns those
// slots during the layer) and pass 2 reads it back, instead of holding the
// row's Q values in registers: one shared store and load more per edge for
// about 30 fewer registers, which lets two 384-thread blocks share an SM
// (check_update_exact parks only rows above kRegQMaxDeg).
template <typename LT, typename MT, bool SAT, bool LEAN, int CH, int DEG = -1, int NREP = 1>
__device__ __forceinline__ void check_update(const RowIn<CH>& in, int k, int Z, LT* __restrict__ L,
                                             MT* __restrict__ mag1, MT* __restrict__ mag2,
                                             uint32_t* __restrict__ meta, int rec, int dummy, float beta,
                                             float msg_sat, float post_sat, const uint32_t* rep = nullptr) {
  // checked builds: every posterior index stays inside the group's region
  // (dummy - k + Z elements: the columns, then one dummy slot per thread)
  const int lim = dummy - k + Z;
  // PAD (the register-resident form): an odd row's padding edge is processed
  // like a real one, on this thread's dummy slot (which can never be a
  // minimum), instead of a separate tail: the latency-bound single loop runs
  // faster with the uniform chunk loop.  Integer modes reset the dummy slot
  // so that the padding edge's |Q| saturates (and, with the larger index,
  // never beats a real edge).
  // DEG >= 0: the row's degree is a compile-time constant; exactly its DEG
  // edges are processed, chunk by chunk, with neither padding nor tail.
  constexpr bool EXACT = DEG >= 0;
  constexpr bool PAD = !LEAN && !EXACT;
  if constexpr (PAD && SAT) st_val(L, dummy, post_sat);
  const uint32_t* tab = in.tab;
  const int deg = EXACT ? DEG : in.deg;
  const float r1 = in.r1, r2 = in.r2;
  const uint32_t mo = in.mo;
  const int idx_o = static_cast<int>(mo >> 27);
  // signs of the R_j, edge 0's moved to bit 31 (integer modes with PAD:
  // positions past deg read as negative, so the padding edge sees
  // Q = dummy + |R|, large and positive)
  uint32_t sgn = (PAD && SAT) ? ((mo << (32 - deg)) | ((1u << (32 - deg)) - 1u)) : (mo << (32 - deg));
  const int nfull = EXACT ? (DEG + CH - 1) / CH : (PAD ? (deg + CH - 1) / CH : deg / CH);
  const int ntail = (PAD || EXACT) ? 0 : deg - CH * nfull;

  float q[LEAN ? 1 : MaxChunks<CH>::value * CH];
  int addr[MaxChunks<CH>::value * CH];
  int addr_t[CH - 1];  // the partial chunk's edges
  float min1 = 3.0e38f, min2 = 3.0e38f;  // SAT modes: keys |Q| * 32 + j
  uint32_t qs = 0;                       // Q sign bits, first edge highest
#pragma unroll
  for (int c = 0; c < MaxChunks<CH>::value; ++c) {
    if (c >= nfull) break;
    const Chunk<CH> ch = c == 0 ? in.c0 : load_chunk<CH>(tab, c);
#pragma unroll
    for (int i = 0; i < CH; ++i)
      if (!EXACT || CH * c + i < DEG)
        addr[CH * c + i] = checked(static_cast<int>(ch.b[i]) + rot(k, ch.s[i], Z), lim, dummy, 1);
    float lv[CH];
#pragma unroll
    for (int i = 0; i < CH; ++i)
      if (!EXACT || CH * c + i < DEG) lv[i] = ld_val(L, addr[CH * c + i]);
#pragma unroll
    for (int i = 0; i < CH; ++i) {
      const int j = CH * c + i;
      if (EXACT && j >= DEG) continue;
      const float Q = pass1_edge<LT, SAT, LEAN>(L, addr[j], lv[i], j, idx_o, r1, r2, sgn, min1, min2, qs, msg_sat,
                                                post_sat);
      if constexpr (!LEAN) q[j] = Q;
    }
  }
  float qt[CH - 1];
  if (ntail) {
    const Chunk<CH> ch = nfull == 0 ? in.c0 : load_chunk<CH>(tab, nfull);
#pragma unroll
    for (int i = 0; i < CH - 1; ++i) {
      if (i < ntail) {
        const int j = CH * nfull + i;
        addr_t[i] = checked(static_cast<int>(ch.b[i]) + rot(k, ch.s[i], Z), lim, dummy, 2);
        qt[i] = pass1_edge<LT, SAT, LEAN>(L, addr_t[i], ld_val(L, addr_t[i]), j, idx_o, r1, r2, sgn, min1, min2,
                                          qs, msg_sat, post_sat);
      }
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
  // magnitudes carrying the parity in their sign bit: the sign of R'_j is
  // parity ^ sign(Q_j), one xor with Q_j's sign bit
  const uint32_t pm = static_cast<uint32_t>(__popc(qs)) << 31;
  const float n1s = __uint_as_float(__float_as_uint(n1) | pm);
  const float n2s = __uint_as_float(__float_as_uint(n2) | pm);
#pragma unroll
  for (int c = 0; c < MaxChunks<CH>::value; ++c) {
    if (c >= nfull) break;
    float qv[CH];
#pragma unroll
    for (int i = 0; i < CH; ++i)
      if (!EXACT || CH * c + i < DEG) qv[i] = LEAN ? ld_val(L, addr[CH * c + i]) : q[LEAN ? 0 : CH * c + i];
#pragma unroll
    for (int i = 0; i < CH; ++i) {
      const int j = CH * c + i;
      if (EXACT && j >= DEG) continue;
      pass2_edge<LT, SAT, NREP>(L, addr[j], qv[i], j, idx, min1, n1s, n2s, post_sat, rep);
    }
  }
  if (ntail) {
#pragma unroll
    for (int i = 0; i < CH - 1; ++i)
      if (i < ntail)
        pass2_edge<LT, SAT, NREP>(L, addr_t[i], LEAN ? ld_val(L, addr_t[i]) : qt[i], CH * nfull + i, idx, min1,
                                  n1s, n2s, post_sat, rep);
  }
  if constexpr (sizeof(MT) == 4) {
    reinterpret_cast<float2*>(mag1)[rec] = make_float2(n1, n2);
  } else {
    st_val(mag1, rec, n1);
    st_val(mag2, rec, n2);
  }
  // the new R signs: the Q signs XOR the parity, on the row's deg bits
  const uint32_t pspread = static_cast<uint32_t>(static_cast<int32_t>(pm) >> 31);
  const uint32_t dmask = (1u << deg) - 1u;
  meta[rec] = ((PAD ? qs >> (CH * nfull - deg) : qs) ^ (pspread & dmask)) | (static_cast<uint32_t>(idx) << 27);
}

// The update with the row's exact degree as a compile-time constant (DEG
// from 2 to the largest degree): no padding edge and no tail.  A LEAN caller's
// rows of degree up to kRegQMaxDeg keep their Q values in registers all the
// same: one shared store and load less per edge.  With the degree fixed at
// compile time the compiler fits rows of degree 22 in the 80-register budget
// of two 384-thread blocks per SM without spilling; beyond that the Q values
// park.
constexpr int kRegQMaxDeg = 22;
//
// The degree is found by bisection of [DEG, HI]: first at 8 (most rows of the
// base graphs have degree 3-8), then by halves, so a row of degree 20 takes 6
// compares instead of the 19 of a chain from degree 2 upward.  (The paired
// INT8 update keeps its chain, check_update_x2_by_degree: there bisection
// measured slower.)
template <int LO, int HI>
constexpr int degree_split() {
  return (LO <= 8 && HI > 8) ? 8 : (LO + HI) / 2;
}

template <typename LT, typename MT, bool SAT, bool LEAN, int CH, int DEG = 2, int NREP = 1, int HI = kMaxDeg>
__device__ __forceinline__ void check_update_exact(const RowIn<CH>& in, int k, int Z, LT* __restrict__ L,
                                                   MT* __restrict__ mag1, MT* __restrict__ mag2,
                                                   uint32_t* __restrict__ meta, int rec, int dummy, float beta,
                                                   float msg_sat, float post_sat, const uint32_t* rep = nullptr) {
  if constexpr (DEG < HI) {
    constexpr int MID = degree_split<DEG, HI>();
    if (in.deg <= MID)
      check_update_exact<LT, MT, SAT, LEAN, CH, DEG, NREP, MID>(in, k, Z, L, mag1, mag2, meta, rec, dummy, beta,
                                                                msg_sat, post_sat, rep);
    else
      check_update_exact<LT, MT, SAT, LEAN, CH, MID + 1, NREP, HI>(in, k, Z, L, mag1, mag2, meta, rec, dummy, beta,
                                                                   msg_sat, post_sat, rep);
  } else {
    constexpr bool lean = LEAN && DEG > kRegQMaxDeg;
    check_update<LT, MT, SAT, lean, CH, DEG, NREP>(in, k, Z, L, mag1, mag2, meta, rec, dummy, beta, msg_sat,
                                                   post_sat, rep);
  }
}

// R = 0 for the first n check records (float: the magnitudes are one float2
// array spanning the mag1 and mag2 areas).
template <typename MT>
__device__ __forceinline__ void zero_records(MT* mag1, MT* mag2, uint32_t* meta, int n, int k, int Z) {
  for (int r = k; r < n; r += Z) {
    if constexpr (sizeof(MT) == 4) {
      reinterpret_cast<float2*>(mag1)[r] = make_float2(0.0f, 0.0f);
    } else {
      mag1[r] = MT(0);
      mag2[r] = MT(0);
    }
    meta[r] = 0u;
  }
}

// Edge e of a row whose chunks start at `tab`: (column base, shift).
template <int CH>
__device__ __forceinline__ uint2 edge_at(const uint32_t* tab, int e) {
  const int c = e / CH, i = e % CH;
  return make_uint2(tab[2 * CH * c + i], tab[2 * CH * c + CH + i]);
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
template <int CH>
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
      const uint2 bs = edge_at<CH>(rt, e);
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
template <int CH, typename LT>
__device__ __forceinline__ bool syndrome_direct(const uint32_t* __restrict__ tab, const uint32_t* __restrict__ rows,
                                                int m_eff, int k, int Z, const LT* __restrict__ L) {
  uint32_t bad = 0;
  for (int l = 0; l < m_eff; ++l) {
    const uint32_t info = rows[l];
    const uint32_t* rt = tab + (info & 0xFFFFu);
    const int deg = static_cast<int>(info >> 16);
    uint32_t p = 0;
    for (int e = 0; e < deg; ++e) {
      const uint2 bs = edge_at<CH>(rt, e);
      p ^= (L[static_cast<int>(bs.x) + rot(k, bs.y, Z)] < LT(0)) ? 1u : 0u;
    }
    bad |= p;
  }
  return bad != 0;
}

// ---- CRC-aided exit for blocks that carry their own CRC (LDPC_CB_CRC24B).
// Bit p of the K = kb * Z information bits stands for x^(K-1-p); the block
// passes iff the XOR of x^(K-1-p) mod g_B over its set bits is 0.  btab holds,
// for every byte j of the block and every byte value v, the XOR of those
// remainders over v's set bits (bit i of v = block bit 8j + i); the threads
// XOR the entries of their bytes and the group XORs the threads' sums.

// Z < 32 (Z = 16): thread k's bits c * Z + k, one entry each.
template <typename LT>
__device__ __forceinline__ uint32_t cb_crc_part(const LT* __restrict__ L, const uint32_t* __restrict__ btab,
                                                int kb, int k, int Z) {
  uint32_t r = 0;
  for (int c = 0; c < kb; ++c) {
    const int p = c * Z + k;
    const uint32_t t = __ldg(btab + (p >> 3) * 256 + (1 << (p & 7)));
    r ^= (L[p] < LT(0)) ? t : 0u;
  }
  return r;
}

// Z % 32 == 0, from the hard-decision bitmap: information word m (block bits
// 32m .. 32m+31) is bitmap word m; thread k takes words k, k + Z, ..., four
// byte entries each.
__device__ __forceinline__ uint32_t cb_crc_part_hb(const uint32_t* __restrict__ hb,
                                                   const uint32_t* __restrict__ btab, int kb, int k, int Z) {
  const int nw = kb * (Z >> 5);
  uint32_t r = 0;
  for (int m = k; m < nw; m += Z) {
    const uint32_t w = hb[m];
    const uint32_t* t = btab + m * 1024;
    r ^= __ldg(t + (w & 0xFFu)) ^ __ldg(t + 256 + ((w >> 8) & 0xFFu)) ^ __ldg(t + 512 + ((w >> 16) & 0xFFu)) ^
         __ldg(t + 768 + (w >> 24));
  }
  return r;
}

// Is the XOR of r over the group's Z threads zero?  For Z > 32 the warps
// meet in `scratch` (Z / 32 words), which no thread of the group may touch
// between the preceding group barrier and the next one after this call.
__device__ __forceinline__ bool group_xor_zero(int Z, int g, uint32_t wmask, uint32_t r, uint32_t* scratch, int k) {
  r = __reduce_xor_sync(wmask, r);
  if (Z <= 32) return r == 0u;
  if ((k & 31) == 0) scratch[k >> 5] = r;
  named_bar_sync(1 + g, Z);
  uint32_t t = 0;
  for (int w = 0; w < (Z >> 5); ++w) t ^= scratch[w];
  return t == 0u;
}

// Two XOR reductions at once (Z % 32 == 0, whole warps): returns whether rA's
// total is zero and sets *zB for rB's.
__device__ __forceinline__ bool group_xor_zero2(int Z, int g, uint32_t rA, uint32_t rB, uint32_t* scrA,
                                                uint32_t* scrB, int k, bool* zB) {
  rA = __reduce_xor_sync(0xFFFFFFFFu, rA);
  rB = __reduce_xor_sync(0xFFFFFFFFu, rB);
  if (Z > 32) {
    if ((k & 31) == 0) {
      scrA[k >> 5] = rA;
      scrB[k >> 5] = rB;
    }
    named_bar_sync(1 + g, Z);
    rA = 0;
    rB = 0;
    for (int w = 0; w < (Z >> 5); ++w) {
      rA ^= scrA[w];
      rB ^= scrB[w];
    }
  }
  *zB = rB == 0u;
  return rA == 0u;
}

}  // namespace core
}  // namespace ldpcgb

// ============================================================================
// INT8, two code blocks per thread.  Every INT8 intermediate is an integer of
// magnitude < 2048 (|Q| <= 190, keys |Q|*32 + j <= 2043), which fp16
// represents exactly, and half2 min/max/add/fma on such values are exact; so
// the pair (block A in the low half, block B in the high half) is decoded
// bit-identically to two separate INT8 decodes with one instruction stream.
// Per check the state is three words: magnitudes (m1A, m1B, m2A, m2B bytes)
// and two words of sign history and argmins (layout at check_update_x2).
#include <cuda_fp16.h>

namespace ldpcgb {
namespace core {

__device__ __forceinline__ __half2 as_h2(uint32_t u) {
  __half2 h;
  memcpy(&h, &u, 4);
  return h;
}

__device__ __forceinline__ uint32_t as_u32(__half2 h) {
  uint32_t u;
  memcpy(&u, &h, 4);
  return u;
}

// 16-bit store into shared memory
__device__ __forceinline__ void st_shared_b16(void* p, uint16_t v) {
  asm volatile("st.shared.b16 [%0], %1;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(p))), "h"(v)
               : "memory");
}

// Rows up to this degree keep their Q pairs in registers for pass 2 as well
// (beyond it the 80-register budget spills).
constexpr int kRegQ2MaxDeg = 12;

// one pair check (l, k); `dummy` is this thread's dummy slot.  Pass 1 parks
// each Q_j pair in its posterior's slot and pass 2 reads it back (the check
// owns those slots during the layer), which keeps the row's Q values out of
// registers.
// The row's table and degree and this check's three message words (mg, s1,
// s2) come from the caller, which loads the next row's before the layer
// barrier.
struct PairIn {
  const uint32_t* tab;
  int deg;
  uint32_t mg, s1, s2;
};

// The three message words of a check: (magnitudes, s1) as one 8-byte pair in
// `ms`, s2 in its own array.
__device__ __forceinline__ PairIn load_pair_row(const uint32_t* __restrict__ s_tab, uint32_t info,
                                                const uint2* __restrict__ ms, const uint32_t* __restrict__ sg2,
                                                int rec) {
  PairIn r;
  r.tab = s_tab + (info & 0xFFFFu);
  r.deg = static_cast<int>(info >> 16);
  const uint2 m = ms[rec];
  r.mg = m.x;
  r.s1 = m.y;
  r.s2 = sg2[rec];
  return r;
}

// Address of edge e of a row (tab = the row's chunks) for check k.
__device__ __forceinline__ int edge_addr(const uint32_t* tab, int e, int k, int Z) {
  const uint32_t* t = tab + 2 * kChunk * (e / kChunk) + (e % kChunk);
  return static_cast<int>(t[0]) + rot(k, t[kChunk], Z);
}

// Stored form: magnitudes as above; the signs of the stored messages R_j,
// edge j < 16 at bit j (A) and 16 + j (B) of s1, edges 16..26 at bits
// 5 + (j-16) (A) and 21 + (j-16) (B) of s2, argmins in s2 bits 0..4 / 16..20.
// R'_j carries the sign product over i != j: the update stores each block's
// Q signs XOR their parity, which it reads off bits 15 / 31 of the XOR of the
// row's Q pairs.  The magnitude word and s1 sit side by side (one 8-byte
// access), s2 in its own array.
//
// Pass 2 writes every edge with the smaller magnitude; the argmin edge of
// each block, whose message takes the second magnitude instead, is then
// rewritten from its Q, read before pass 2 (the check owns the slot).
template <int DEG = -1>
__device__ __forceinline__ void check_update_x2(const PairIn& in, int k, int Z, uint32_t* __restrict__ L,
                                                uint2* __restrict__ ms, uint32_t* __restrict__ sg2, int rec,
                                                int dummy, __half2 beta, __half2 msg, __half2 post) {
  // DEG >= 0: the row's degree is a compile-time constant and only its DEG
  // edges are processed; otherwise a padding edge completes the last chunk
  // (on this thread's dummy slot, which can never be a minimum)
  constexpr bool EXACT = DEG >= 0;
  // rows of degree up to kRegQ2MaxDeg also keep their Q pairs in registers for
  // pass 2 (the parked copies still serve the argmin rewrite)
  constexpr bool REGQ = EXACT && DEG <= kRegQ2MaxDeg;
  if constexpr (!EXACT) L[dummy] = as_u32(post);
  const uint32_t* tab = in.tab;
  const int deg = EXACT ? DEG : in.deg;
  const uint32_t mg = in.mg, s1 = in.s1, s2 = in.s2;
  const __half2 h1024 = __float2half2_rn(1024.0f);
  const uint32_t M1s = as_u32(__hsub2(as_h2(__byte_perm(mg, 0x64646464u, 0x5140)), h1024));
  const uint32_t M2s = as_u32(__hsub2(as_h2(__byte_perm(mg, 0x64646464u, 0x5342)), h1024));
  // the argmins as half2 1024 + index, compared with 1024 + j below
  const __half2 I = as_h2((s2 & 0x001F001Fu) | 0x64006400u);
  const __half2 h32 = __float2half2_rn(32.0f);
  const __half2 npost = __hneg2(post);
  const int nch = (deg + kChunk - 1) / kChunk;

  int addr[kMaxChunks * kChunk];
  uint32_t qr[REGQ ? kMaxChunks * kChunk : 1];
  __half2 min1 = __float2half2_rn(65504.0f), min2 = min1;
  uint32_t acc1 = 0, acc2 = 0;  // Q signs: each new edge enters at bits 15 / 31
  uint32_t par = 0;              // XOR of the Q pairs: bits 15 / 31 are the sign parities
#pragma unroll
  for (int c = 0; c < kMaxChunks; ++c) {
    if (c >= nch) break;
    const Chunk<kChunk> ch = load_chunk<kChunk>(tab, c);
#pragma unroll
    for (int i = 0; i < kChunk; ++i)
      if (!EXACT || kChunk * c + i < DEG)
        addr[kChunk * c + i] = checked(static_cast<int>(ch.b[i]) + rot(k, ch.s[i], Z), dummy - k + Z, dummy, 3);
    uint32_t lv[kChunk];
#pragma unroll
    for (int i = 0; i < kChunk; ++i)
      if (!EXACT || kChunk * c + i < DEG) lv[i] = L[addr[kChunk * c + i]];
#pragma unroll
    for (int i = 0; i < kChunk; ++i) {
      const int j = kChunk * c + i;
      if (EXACT && j >= DEG) continue;
      const __half2 J = __float2half2_rn(static_cast<float>(j));
      const uint32_t eq = __heq2_mask(I, __float2half2_rn(static_cast<float>(1024 + j)));
      // (edge 27 can only be padding, whose sign does not matter)
      const uint32_t sw = j < 16 ? (s1 << (15 - j)) : (j <= 26 ? (s2 << (26 - j)) : 0u);
      const uint32_t rb = ((M2s & eq) | (M1s & ~eq)) ^ (sw & 0x80008000u);
      __half2 Q = __hsub2(as_h2(lv[i]), as_h2(rb));
      Q = __hmin2(__hmax2(Q, npost), post);
      L[addr[j]] = as_u32(Q);
      if constexpr (REGQ) qr[j] = as_u32(Q);
      par ^= as_u32(Q);
      if (j < 16)
        acc1 = ((acc1 >> 1) & 0x7FFF7FFFu) | (as_u32(Q) & 0x80008000u);
      else
        acc2 = ((acc2 >> 1) & 0x7FFF7FFFu) | (as_u32(Q) & 0x80008000u);
      const __half2 key = __hfma2(__hmin2(__habs2(Q), msg), h32, J);
      min2 = __hmin2(min2, __hmax2(min1, key));
      min1 = __hmin2(min1, key);
    }
  }
  // the keys decoded in half2, exactly (integers < 2048; the division by 32
  // is a power-of-two scaling): magnitude = floor(key / 32), argmin = key - 32
  // magnitude, new magnitudes max(magnitude - beta, 0)
  const __half2 zero2 = __float2half2_rn(0.0f);
  const __half2 m1 = h2floor(__hmul2(min1, __float2half2_rn(0.03125f)));
  const __half2 m2 = h2floor(__hmul2(min2, __float2half2_rn(0.03125f)));
  const __half2 h1 = __hmax2(__hsub2(m1, beta), zero2);
  const __half2 h2 = __hmax2(__hsub2(m2, beta), zero2);
  // 1024 + x (0 <= x < 1024) holds x in its low mantissa bits
  const uint32_t iw = as_u32(__hadd2(__hfma2(m1, __float2half2_rn(-32.0f), min1), h1024)) & 0x001F001Fu;
  const uint32_t idxA = iw & 0xFFFFu, idxB = iw >> 16;
  const uint32_t mw = __byte_perm(as_u32(__hadd2(h1, h1024)), as_u32(__hadd2(h2, h1024)), 0x6420);
  const uint32_t pm = par & 0x80008000u;
  const uint32_t N1s = as_u32(h1) | pm;
  const uint32_t N2s = as_u32(h2) | pm;
  // the two argmin edges and their Q values, before pass 2 overwrites them
  const int aA = checked(edge_addr(tab, static_cast<int>(idxA), k, Z), dummy - k + Z, dummy, 4);
  const int aB = checked(edge_addr(tab, static_cast<int>(idxB), k, Z), dummy - k + Z, dummy, 4);
  const uint32_t qsel = (L[aA] & 0x0000FFFFu) | (L[aB] & 0xFFFF0000u);
#pragma unroll
  for (int c = 0; c < kMaxChunks; ++c) {
    if (c >= nch) break;
    uint32_t qv[kChunk];
#pragma unroll
    for (int i = 0; i < kChunk; ++i)
      if (!EXACT || kChunk * c + i < DEG) qv[i] = REGQ ? qr[REGQ ? kChunk * c + i : 0] : L[addr[kChunk * c + i]];
#pragma unroll
    for (int i = 0; i < kChunk; ++i) {
      if (EXACT && kChunk * c + i >= DEG) continue;
      const uint32_t rb = N1s ^ (qv[i] & 0x80008000u);
      __half2 v = __hadd2(as_h2(qv[i]), as_h2(rb));
      v = __hmin2(__hmax2(v, npost), post);
      L[addr[kChunk * c + i]] = as_u32(v);  // (without EXACT, padding edges write the dummy slot)
    }
  }
  {
    const uint32_t rb = N2s ^ (qsel & 0x80008000u);
    const uint32_t v = as_u32(__hmin2(__hmax2(__hadd2(as_h2(qsel), as_h2(rb)), npost), post));
    // block A's half of slot aA, block B's half of slot aB: one 16-bit store
    // each (inline stores with a memory clobber, ordered after pass 2's)
    st_shared_b16(reinterpret_cast<uint8_t*>(L + aA), static_cast<uint16_t>(v & 0xFFFFu));
    st_shared_b16(reinterpret_cast<uint8_t*>(L + aB) + 2, static_cast<uint16_t>(v >> 16));
  }
  const int n_all = EXACT ? DEG : kChunk * nch;
  const int n1 = n_all < 16 ? n_all : 16;
  const int n2 = n_all - 16;
  // the new R signs: each block's Q signs XOR its parity (bit 15 / 31 of pm
  // spread over its half); bits past the row's degree are never read
  const uint32_t spread = (pm >> 15) * 0xFFFFu;  // (bit 0, bit 16) = (A, B) parity, times 0xFFFF
  ms[rec] = make_uint2(mw, (acc1 ^ spread) >> (16 - n1));
  const uint32_t a2 = n2 <= 0 ? 0u : (n2 <= 11 ? (acc2 ^ spread) >> (11 - n2) : (acc2 ^ spread) << (n2 - 11));
  sg2[rec] = (a2 & 0xFFE0FFE0u) | iw;
}

// check_update_x2 with the row's degree as a compile-time constant (no padding
// edge, straight-line passes).
template <int DEG = 2>
__device__ __forceinline__ void check_update_x2_by_degree(const PairIn& in, int k, int Z, uint32_t* __restrict__ L,
                                                          uint2* __restrict__ ms, uint32_t* __restrict__ sg2, int rec,
                                                          int dummy, __half2 beta, __half2 msg, __half2 post) {
  if constexpr (DEG < kMaxDeg) {
    if (in.deg != DEG) {
      check_update_x2_by_degree<DEG + 1>(in, k, Z, L, ms, sg2, rec, dummy, beta, msg, post);
      return;
    }
  }
  check_update_x2<DEG>(in, k, Z, L, ms, sg2, rec, dummy, beta, msg, post);
}

// hard decisions of both blocks of a pair into their bitmaps
__device__ __forceinline__ void hard_bitmap_x2(const uint32_t* __restrict__ L, uint32_t* __restrict__ hbA,
                                               uint32_t* __restrict__ hbB, int n_eff, int k, int Z) {
  const int W = Z >> 5;
  const int w = k >> 5;
  const bool lane0 = (k & 31) == 0;
  for (int c = 0; c < n_eff; ++c) {
    const uint32_t v = L[c * Z + k];
    const uint32_t a = __ballot_sync(0xFFFFFFFFu, (v & 0x8000u) != 0u);
    const uint32_t b = __ballot_sync(0xFFFFFFFFu, (v & 0x80000000u) != 0u);
    if (lane0) {
      hbA[c * W + w] = a;
      hbB[c * W + w] = b;
    }
  }
}

}  // namespace core
}  // namespace ldpcgb
