// URLLC puncturing allocations on sm_103a: the two benchmark policies of the
// paper's evaluation (Sec. VII-A), the feasibility enforcer of its RT O-DU
// (Sec. V-B, eq. 6 and eq. 7) and the per-subcarrier puncture masks they
// imply.  A problem is a handful of users (at most 32): one warp solves one
// problem with one lane per user, so a single problem (the RT O-DU's
// per-TTI step) takes a few dependent operations per lane rather than a
// serial loop, and a batch is many warps side by side.
//
// Rounding ("Huntington-Hill"): every value starts at its floor and may go
// to its ceiling (never above its cap); the units left go to the values of
// largest priority q_e / sqrt(a_e (a_e + 1)) (a_e the floor; infinite for
// a_e = 0), equal priorities to the lower index.  A value can take at most
// one unit, so handing units out one at a time by priority is the same as
// giving them to the `left` highest-ranked values.  Arithmetic is float32 (the
// paper fixes no precision; the policy network's output is float32), every
// step an explicitly rounded operation in a fixed order (no fused
// multiply-adds), so a CPU implementation taking the same steps agrees bit
// for bit and the integer decisions match.
#include <cmath>
#include <string>

#include "internal.cuh"

namespace ldpcgb {

namespace {

constexpr int kMaxUsers = 32;
constexpr int kMiniSlots = 7;     // mini-slots per slot, two OFDM symbols each
constexpr int kPolicyBlock = 128;  // four problems per block
constexpr unsigned kFull = 0xFFFFFFFFu;

__device__ __forceinline__ int warp_sum(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// Huntington-Hill rounding of lane e's quota q (lanes >= E pass active = false)
// to an integer; the lane values sum to `total`.  Returns false (on every
// lane) if no rounding within [floor, min(ceil, cap)] sums to the total.
__device__ bool hh_round_warp(float q, int cap, bool active, int total, int lane, int E, int* out) {
  int a = active ? min(static_cast<int>(floorf(q)), cap) : 0;
  const int hi = active ? min(static_cast<int>(ceilf(q)), cap) : 0;
  const int left = total - warp_sum(a);
  const int room = warp_sum(hi - a);
  if (left < 0 || left > room) return false;
  const bool elig = hi > a;
  const float p = !elig ? -1.0f
                  : a == 0 ? INFINITY
                           : __fdiv_rn(q, __fsqrt_rn(__fmul_rn(static_cast<float>(a), static_cast<float>(a + 1))));
  // rank among eligible lanes: higher priority first, lower index on ties
  int rank = 0;
  for (int f = 0; f < E; ++f) {  // E is the same on every lane
    const float pf = __shfl_sync(kFull, p, f);
    const bool ef = __shfl_sync(kFull, elig, f);
    if (ef && (pf > p || (pf == p && f < lane))) ++rank;
  }
  if (elig && rank < left) ++a;
  *out = a;
  return true;
}

// One warp per (TTI, mini-slot): SCs taken from each user for that
// mini-slot's demand.  status: 0 ok, 1 demand exceeds the allocations.
__global__ void __launch_bounds__(kPolicyBlock) alloc_kernel(int policy, int n_prob, int E, const int32_t* n,
                                                            const int32_t* demand, int32_t* m, int32_t* status) {
  const int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (p >= n_prob) return;  // whole warps leave together
  const int t = p / kMiniSlots;
  const bool active = lane < E;
  const int cap = active ? n[static_cast<int64_t>(t) * E + lane] : 0;
  const int S = warp_sum(cap);
  const int D = demand[p];
  bool ok = D <= S;
  int a = 0;
  if (ok && D > 0) {
    if (policy == LDPC_POLICY_RP) {
      const float q = __fdiv_rn(__fmul_rn(static_cast<float>(D), static_cast<float>(cap)), static_cast<float>(S));
      ok = hh_round_warp(q, cap, active, D, lane, E, &a);
    } else {  // smallest allocation first, lower index on ties: SCs of the users ranked before this one
      int before = 0;
      for (int f = 0; f < E; ++f) {  // E is the same on every lane
        const int cf = __shfl_sync(kFull, cap, f);
        if (cf < cap || (cf == cap && f < lane)) before += cf;
      }
      a = active ? max(0, min(cap, D - before)) : 0;
    }
  }
  if (active) m[static_cast<int64_t>(p) * E + lane] = ok ? a : 0;
  if (lane == 0) status[p] = ok ? 0 : 1;
}

// One warp per problem: KL projection (eq. 7) by water-filling, then
// Huntington-Hill rounding.  status: 0 ok, 1 total exceeds the allocations,
// 2 no rounding sums to the total.
__global__ void __launch_bounds__(kPolicyBlock) enforce_kernel(int n_prob, int E, const float* m_in,
                                                              const int32_t* n_in, const int32_t* total_in,
                                                              int32_t* out, int32_t* status) {
  const int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (p >= n_prob) return;
  const bool active = lane < E;
  const int64_t off = static_cast<int64_t>(p) * E + lane;
  const float me = active ? m_in[off] : 0.0f;
  const int cap = active ? n_in[off] : 0;
  const float ne = static_cast<float>(cap);
  const bool pos = active && me > 0.0f;
  const int T = total_in[p];
  const float total = static_cast<float>(T);
  // allocations are integers: their sums are exact in any order
  const int cap_all = warp_sum(cap);
  const int cap_pos = warp_sum(pos ? cap : 0);
  int st = 0;
  float x = 0.0f;
  if (T > cap_all) {
    st = 1;
  } else if (cap_pos <= T) {
    // every user with m_e > 0 is capped; the rest goes to the others by capacity
    const int cap0 = cap_all - cap_pos;
    const float rest = static_cast<float>(T - cap_pos);
    if (pos)
      x = ne;
    else if (active && rest > 0.0f && cap0 > 0)
      x = __fdiv_rn(__fmul_rn(rest, ne), static_cast<float>(cap0));
  } else {
    // water-filling: users reach their cap in order of n_e / m_e (lower index on ties)
    const float b = pos ? __fdiv_rn(ne, me) : 0.0f;
    int rank = 0;
    for (int f = 0; f < E; ++f) {  // E is the same on every lane
      const float bf = __shfl_sync(kFull, b, f);
      const bool pf = __shfl_sync(kFull, pos, f);
      if (pf && (bf < b || (bf == b && f < lane))) ++rank;
    }
    // lane k evaluates "the first k users of the order capped": c_k and whether
    // the k-th user stays below its cap
    const int npos = __popc(__ballot_sync(kFull, pos));
    const int k = lane;
    int capped = 0;
    float free_m = 0.0f, mk = 0.0f, nk = 0.0f;
    for (int f = 0; f < E; ++f) {
      const float mf = __shfl_sync(kFull, me, f);
      const int cf = __shfl_sync(kFull, cap, f);
      const bool pf = __shfl_sync(kFull, pos, f);
      const int rf = __shfl_sync(kFull, pos ? rank : -1, f);
      if (!pf) continue;
      if (rf < k)
        capped += cf;
      else
        free_m = __fadd_rn(free_m, mf);  // index order, as in the definition
      if (rf == k) {
        mk = mf;
        nk = static_cast<float>(cf);
      }
    }
    const float ck = k < npos ? __fdiv_rn(__fsub_rn(total, static_cast<float>(capped)), free_m) : 0.0f;
    const bool stop = k < npos && __fmul_rn(ck, mk) <= nk;
    const unsigned hit = __ballot_sync(kFull, stop);
    const int kstar = hit ? __ffs(hit) - 1 : npos - 1;
    const float c = __shfl_sync(kFull, ck, kstar);
    if (pos) x = fminf(ne, __fmul_rn(c, me));
  }
  int a = 0;
  if (st == 0 && !hh_round_warp(x, cap, active, T, lane, E, &a)) st = 2;
  if (active) out[off] = st == 0 ? a : 0;
  if (lane == 0) status[p] = st;
}

// One thread per (TTI, OFDM symbol, 32-SC word): bit b of word w is SC
// 32w + b; user e's band starts after users 0..e-1 and its lowest m_e SCs
// of the symbol's mini-slot are punctured.
__global__ void __launch_bounds__(kPolicyBlock) sc_mask_kernel(int n_tti, int E, int words, const int32_t* n,
                                                              const int32_t* m, uint32_t* mask) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t per_tti = static_cast<int64_t>(kMiniSlots) * 2 * words;
  if (i >= static_cast<int64_t>(n_tti) * per_tti) return;
  const int t = static_cast<int>(i / per_tti);
  const int rem = static_cast<int>(i - t * per_tti);
  const int sym = rem / words;
  const int w = rem - sym * words;
  const int32_t* nt = n + static_cast<int64_t>(t) * E;
  const int32_t* mt = m + (static_cast<int64_t>(t) * kMiniSlots + sym / 2) * E;
  const int lo = 32 * w, hi = lo + 32;
  uint32_t bits = 0;
  int start = 0;
  for (int e = 0; e < E && start < hi; ++e) {
    const int a = max(start, lo), b = min(start + mt[e], hi);  // punctured SCs of user e in this word
    if (b > a) bits |= (b - a == 32 ? 0xFFFFFFFFu : ((1u << (b - a)) - 1u)) << (a - lo);
    start += nt[e];
  }
  mask[i] = bits;
}

int grid_for(int64_t n) { return static_cast<int>((n + kPolicyBlock - 1) / kPolicyBlock); }

}  // namespace

}  // namespace ldpcgb

using namespace ldpcgb;

namespace {

int policy_fail(int code, const char* msg) {
  set_error(msg);
  return code;
}

int launch_status(cudaError_t e) {
  if (e != cudaSuccess) {
    set_error(std::string("policy kernel launch: ") + cudaGetErrorString(e));
    return LDPC_ECUDA;
  }
  return LDPC_OK;
}

}  // namespace

extern "C" {

LDPC_API int ldpc_puncture_alloc(int32_t policy, int32_t n_tti, int32_t n_users, const int32_t* alloc_dev,
                                 const int32_t* demand_dev, int32_t* punct_dev, int32_t* status_dev,
                                 void* cuda_stream) {
  if (policy != LDPC_POLICY_RP && policy != LDPC_POLICY_SEF) return policy_fail(LDPC_EINVAL, "unknown policy");
  if (n_tti < 0 || n_users < 1 || n_users > kMaxUsers) return policy_fail(LDPC_EINVAL, "n_users must be 1..32");
  if (n_tti == 0) return LDPC_OK;
  if (!alloc_dev || !demand_dev || !punct_dev || !status_dev) return policy_fail(LDPC_EINVAL, "null buffer");
  const int n_prob = n_tti * kMiniSlots;
  alloc_kernel<<<grid_for(static_cast<int64_t>(n_prob) * 32), kPolicyBlock, 0,
                 static_cast<cudaStream_t>(cuda_stream)>>>(
      policy, n_prob, n_users, alloc_dev, demand_dev, punct_dev, status_dev);
  return launch_status(cudaGetLastError());
}

LDPC_API int ldpc_feasibility_enforce(int32_t n_prob, int32_t n_users, const float* punct_real_dev,
                                      const int32_t* alloc_dev, const int32_t* total_dev, int32_t* punct_dev,
                                      int32_t* status_dev, void* cuda_stream) {
  if (n_prob < 0 || n_users < 1 || n_users > kMaxUsers) return policy_fail(LDPC_EINVAL, "n_users must be 1..32");
  if (n_prob == 0) return LDPC_OK;
  if (!punct_real_dev || !alloc_dev || !total_dev || !punct_dev || !status_dev)
    return policy_fail(LDPC_EINVAL, "null buffer");
  enforce_kernel<<<grid_for(static_cast<int64_t>(n_prob) * 32), kPolicyBlock, 0,
                  static_cast<cudaStream_t>(cuda_stream)>>>(
      n_prob, n_users, punct_real_dev, alloc_dev, total_dev, punct_dev, status_dev);
  return launch_status(cudaGetLastError());
}

LDPC_API int ldpc_sc_mask(int32_t n_tti, int32_t n_users, const int32_t* alloc_dev, const int32_t* punct_dev,
                          int32_t words_per_symbol, uint32_t* mask_dev, void* cuda_stream) {
  if (n_tti < 0 || n_users < 1 || n_users > kMaxUsers || words_per_symbol < 1)
    return policy_fail(LDPC_EINVAL, "bad sizes");
  if (n_tti == 0) return LDPC_OK;
  if (!alloc_dev || !punct_dev || !mask_dev) return policy_fail(LDPC_EINVAL, "null buffer");
  const int64_t n = static_cast<int64_t>(n_tti) * kMiniSlots * 2 * words_per_symbol;
  sc_mask_kernel<<<grid_for(n), kPolicyBlock, 0, static_cast<cudaStream_t>(cuda_stream)>>>(
      n_tti, n_users, words_per_symbol, alloc_dev, punct_dev, mask_dev);
  return launch_status(cudaGetLastError());
}

}  // extern "C"
