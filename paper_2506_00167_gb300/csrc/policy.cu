// URLLC puncturing allocations on sm_103a: the two benchmark policies of the
// paper's evaluation (Sec. VII-A), the feasibility enforcer of its RT O-DU
// (Sec. V-B, eq. 6 and eq. 7) and the per-subcarrier puncture masks they
// imply.  Each problem is a handful of users (at most 32), so one thread
// solves one problem serially and a batch is many problems side by side.
//
// Rounding ("Huntington-Hill"): start from the floors of the real quotas and
// hand the remaining units out one at a time to the largest priority
// q_e / sqrt(a_e (a_e + 1)) (infinite for a_e = 0) among values below their
// ceiling and their cap; equal priorities go to the lower index.  Every
// floating-point step is an explicitly rounded float64 operation taken in a
// fixed order (no contraction into fused multiply-adds), so a CPU
// implementation taking the same steps agrees bit for bit and the integer
// decisions match.
#include <cmath>
#include <string>

#include "internal.cuh"

namespace ldpcgb {

namespace {

constexpr int kMaxUsers = 32;
constexpr int kMiniSlots = 7;  // mini-slots per slot, two OFDM symbols each
constexpr int kPolicyBlock = 128;

// Huntington-Hill rounding of q[0..E) to integers summing to `total`, each
// within [floor(q), min(ceil(q), cap)].  Returns false if impossible.
__device__ bool hh_round(const double* q, const int* cap, int E, int total, int* a) {
  int hi[kMaxUsers];
  int sum = 0, room = 0;
  for (int e = 0; e < E; ++e) {
    const int f = static_cast<int>(floor(q[e]));
    const int c = static_cast<int>(ceil(q[e]));
    a[e] = min(f, cap[e]);
    hi[e] = min(c, cap[e]);
    sum += a[e];
    room += hi[e] - a[e];
  }
  int left = total - sum;
  if (left < 0 || left > room) return false;
  for (; left > 0; --left) {
    int best = -1;
    double best_p = -1.0;
    for (int e = 0; e < E; ++e) {
      if (a[e] >= hi[e]) continue;
      const double p =
          a[e] == 0 ? INFINITY
                    : __ddiv_rn(q[e], __dsqrt_rn(__dmul_rn(static_cast<double>(a[e]), static_cast<double>(a[e] + 1))));
      if (p > best_p) {
        best = e;
        best_p = p;
      }
    }
    ++a[best];
  }
  return true;
}

// One thread per (TTI, mini-slot): SCs taken from each user for that
// mini-slot's demand.  status: 0 ok, 1 demand exceeds the allocations.
__global__ void __launch_bounds__(kPolicyBlock) alloc_kernel(int policy, int n_prob, int E, const int32_t* n,
                                                            const int32_t* demand, int32_t* m, int32_t* status) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n_prob) return;
  const int t = p / kMiniSlots;
  const int32_t* nt = n + static_cast<int64_t>(t) * E;
  int32_t* out = m + static_cast<int64_t>(p) * E;
  const int D = demand[p];
  int cap[kMaxUsers];
  int S = 0;
  for (int e = 0; e < E; ++e) {
    cap[e] = nt[e];
    S += cap[e];
  }
  int a[kMaxUsers];
  bool ok = D <= S;
  if (ok && D == 0) {
    for (int e = 0; e < E; ++e) a[e] = 0;
  } else if (ok && policy == LDPC_POLICY_RP) {
    double q[kMaxUsers];
    for (int e = 0; e < E; ++e)
      q[e] = __ddiv_rn(__dmul_rn(static_cast<double>(D), static_cast<double>(cap[e])), static_cast<double>(S));
    ok = hh_round(q, cap, E, D, a);
  } else if (ok) {  // smallest allocation first, lower index on ties
    bool used[kMaxUsers];
    for (int e = 0; e < E; ++e) {
      used[e] = false;
      a[e] = 0;
    }
    int left = D;
    for (int k = 0; k < E && left > 0; ++k) {
      int pick = -1;
      for (int e = 0; e < E; ++e)
        if (!used[e] && (pick < 0 || cap[e] < cap[pick])) pick = e;
      used[pick] = true;
      a[pick] = min(left, cap[pick]);
      left -= a[pick];
    }
  }
  for (int e = 0; e < E; ++e) out[e] = ok ? a[e] : 0;
  status[p] = ok ? 0 : 1;
}

// One thread per problem: KL projection (eq. 7) by water-filling, then
// Huntington-Hill rounding.  status: 0 ok, 1 total exceeds the allocations,
// 2 no rounding sums to the total.
__global__ void __launch_bounds__(kPolicyBlock) enforce_kernel(int n_prob, int E, const double* m_in,
                                                              const int32_t* n_in, const int32_t* total_in,
                                                              int32_t* out, int32_t* status) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n_prob) return;
  const double* m = m_in + static_cast<int64_t>(p) * E;
  const int32_t* nn = n_in + static_cast<int64_t>(p) * E;
  int32_t* o = out + static_cast<int64_t>(p) * E;
  const int T = total_in[p];
  const double total = static_cast<double>(T);
  double n[kMaxUsers], x[kMaxUsers];
  int cap[kMaxUsers];
  double cap_all = 0.0, cap_pos = 0.0;
  for (int e = 0; e < E; ++e) {
    cap[e] = nn[e];
    n[e] = static_cast<double>(cap[e]);
    x[e] = 0.0;
    cap_all = __dadd_rn(cap_all, n[e]);
    if (m[e] > 0.0) cap_pos = __dadd_rn(cap_pos, n[e]);
  }
  int st = 0;
  if (total > cap_all) {
    st = 1;
  } else if (cap_pos <= total) {
    // every user with m_e > 0 is capped; the rest goes to the others by capacity
    double cap0 = 0.0;
    for (int e = 0; e < E; ++e) {
      if (m[e] > 0.0)
        x[e] = n[e];
      else
        cap0 = __dadd_rn(cap0, n[e]);
    }
    const double rest = __dsub_rn(total, cap_pos);
    if (rest > 0.0 && cap0 > 0.0)
      for (int e = 0; e < E; ++e)
        if (!(m[e] > 0.0)) x[e] = __ddiv_rn(__dmul_rn(rest, n[e]), cap0);
  } else {
    // water-filling: users reach their cap in order of n_e / m_e (lower index on ties)
    int order[kMaxUsers];
    double brk[kMaxUsers];
    int k = 0;
    double free_m = 0.0;
    for (int e = 0; e < E; ++e) {
      if (!(m[e] > 0.0)) continue;
      free_m = __dadd_rn(free_m, m[e]);
      const double b = __ddiv_rn(n[e], m[e]);
      int i = k++;
      while (i > 0 && brk[i - 1] > b) {  // stable insertion: equal breakpoints keep index order
        brk[i] = brk[i - 1];
        order[i] = order[i - 1];
        --i;
      }
      brk[i] = b;
      order[i] = e;
    }
    double capped = 0.0, c = 0.0;
    for (int i = 0; i < k; ++i) {
      const int e = order[i];
      c = __ddiv_rn(__dsub_rn(total, capped), free_m);
      if (__dmul_rn(c, m[e]) <= n[e]) break;
      capped = __dadd_rn(capped, n[e]);
      free_m = __dsub_rn(free_m, m[e]);
    }
    for (int e = 0; e < E; ++e)
      if (m[e] > 0.0) x[e] = fmin(n[e], __dmul_rn(c, m[e]));
  }
  int a[kMaxUsers];
  if (st == 0 && !hh_round(x, cap, E, T, a)) st = 2;
  for (int e = 0; e < E; ++e) o[e] = st == 0 ? a[e] : 0;
  status[p] = st;
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
  alloc_kernel<<<grid_for(n_prob), kPolicyBlock, 0, static_cast<cudaStream_t>(cuda_stream)>>>(
      policy, n_prob, n_users, alloc_dev, demand_dev, punct_dev, status_dev);
  return launch_status(cudaGetLastError());
}

LDPC_API int ldpc_feasibility_enforce(int32_t n_prob, int32_t n_users, const double* punct_real_dev,
                                      const int32_t* alloc_dev, const int32_t* total_dev, int32_t* punct_dev,
                                      int32_t* status_dev, void* cuda_stream) {
  if (n_prob < 0 || n_users < 1 || n_users > kMaxUsers) return policy_fail(LDPC_EINVAL, "n_users must be 1..32");
  if (n_prob == 0) return LDPC_OK;
  if (!punct_real_dev || !alloc_dev || !total_dev || !punct_dev || !status_dev)
    return policy_fail(LDPC_EINVAL, "null buffer");
  enforce_kernel<<<grid_for(n_prob), kPolicyBlock, 0, static_cast<cudaStream_t>(cuda_stream)>>>(
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
