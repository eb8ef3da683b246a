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
#include <algorithm>
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

// KL projection (eq. 7) by water-filling, then Huntington-Hill rounding, on
// one warp: lane e holds user e's real puncturing value `me` and allocation
// `cap`; writes lane e's integer result and the problem's status (0 ok, 1
// total exceeds the allocations, 2 no rounding sums to the total).
__device__ void enforce_warp(float me, int cap, bool active, int T, int lane, int E, int* a_out, int* st_out) {
  const float ne = static_cast<float>(cap);
  const bool pos = active && me > 0.0f;
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
  *a_out = st == 0 ? a : 0;
  *st_out = st;
}

// One warp per problem.
__global__ void __launch_bounds__(kPolicyBlock) enforce_kernel(int n_prob, int E, const float* m_in,
                                                              const int32_t* n_in, const int32_t* total_in,
                                                              int32_t* out, int32_t* status) {
  const int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (p >= n_prob) return;
  const bool active = lane < E;
  const int64_t off = static_cast<int64_t>(p) * E + lane;
  int a, st;
  enforce_warp(active ? m_in[off] : 0.0f, active ? n_in[off] : 0, active, total_in[p], lane, E, &a, &st);
  if (active) out[off] = a;
  if (lane == 0) status[p] = st;
}

// RT O-DU step for one TTI per block (Alg. 2): the policy network's forward
// pass for every branch j = 1 .. J on input [s(t)/N, j/J] (one ReLU hidden
// layer, outputs means and raw deviations, sigma = softplus, the
// reparameterised sample z = mu + sigma * noise, action (tanh(z) + 1) / 2 read
// as the fraction of each user's allocation), then the enforcer per branch on
// warp j-1 with total j L.  Sums start at the bias and add products in index
// order, each rounded once (no fused multiply-adds).
__global__ void rt_odu_kernel(int E, int H, int J, int L, const int32_t* alloc, const float* w1, const float* b1,
                              const float* w2, const float* b2, const float* noise, int32_t* book, float* act,
                              int32_t* status) {
  extern __shared__ float sm[];
  float* x = sm;                   // [J][E+1]
  float* h = x + J * (E + 1);      // [J][H]
  float* o = h + J * H;            // [J][2E]
  float* m = o + J * 2 * E;        // [J][E]
  __shared__ int s_alloc[kMaxUsers];
  __shared__ int s_N;
  const int t = blockIdx.x;
  const int tid = threadIdx.x;
  if (tid < E) s_alloc[tid] = alloc[static_cast<int64_t>(t) * E + tid];
  __syncthreads();
  if (tid == 0) {
    int N = 0;
    for (int e = 0; e < E; ++e) N += s_alloc[e];
    s_N = N;
  }
  __syncthreads();
  const float Nf = static_cast<float>(s_N);
  for (int i = tid; i < J * (E + 1); i += blockDim.x) {
    const int j = i / (E + 1), e = i - j * (E + 1);
    x[i] = e < E ? __fdiv_rn(static_cast<float>(s_alloc[e]), Nf)
                 : __fdiv_rn(static_cast<float>(j + 1), static_cast<float>(J));
  }
  __syncthreads();
  for (int i = tid; i < J * H; i += blockDim.x) {
    const int j = i / H, k = i - j * H;
    float acc = b1[k];
    for (int e = 0; e <= E; ++e) acc = __fadd_rn(acc, __fmul_rn(w1[k * (E + 1) + e], x[j * (E + 1) + e]));
    h[i] = acc < 0.0f ? 0.0f : acc;
  }
  __syncthreads();
  for (int i = tid; i < J * 2 * E; i += blockDim.x) {
    const int j = i / (2 * E), r = i - j * 2 * E;
    float acc = b2[r];
    for (int k = 0; k < H; ++k) acc = __fadd_rn(acc, __fmul_rn(w2[r * H + k], h[j * H + k]));
    o[i] = acc;
  }
  __syncthreads();
  for (int i = tid; i < J * E; i += blockDim.x) {
    const int j = i / E, e = i - j * E;
    const float mu = o[j * 2 * E + e], s = o[j * 2 * E + E + e];
    const float sigma = __fadd_rn(fmaxf(s, 0.0f), log1pf(expf(-fabsf(s))));
    const float z = __fadd_rn(mu, __fmul_rn(sigma, noise[(static_cast<int64_t>(t) * J + j) * E + e]));
    const float a = __fdiv_rn(__fadd_rn(tanhf(z), 1.0f), 2.0f);
    act[(static_cast<int64_t>(t) * J + j) * E + e] = a;
    m[i] = __fmul_rn(a, static_cast<float>(s_alloc[e]));
  }
  __syncthreads();
  const int warp = tid >> 5, lane = tid & 31;
  if (warp < J) {
    const bool active = lane < E;
    int a, st;
    enforce_warp(active ? m[warp * E + lane] : 0.0f, active ? s_alloc[lane] : 0, active, (warp + 1) * L, lane, E,
                 &a, &st);
    if (active) book[(static_cast<int64_t>(t) * J + warp) * E + lane] = a;
    if (lane == 0) status[static_cast<int64_t>(t) * J + warp] = st;
  }
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

LDPC_API int ldpc_rt_odu_codebook(int32_t n_tti, int32_t n_users, int32_t hidden, int32_t n_branch, int32_t L,
                                  const int32_t* alloc_dev, const float* w1_dev, const float* b1_dev,
                                  const float* w2_dev, const float* b2_dev, const float* noise_dev,
                                  int32_t* codebook_dev, float* action_dev, int32_t* status_dev, void* cuda_stream) {
  if (n_tti < 0 || n_users < 1 || n_users > kMaxUsers || hidden < 1 || hidden > 1024 || n_branch < 1 ||
      n_branch > 32 || L < 1)
    return policy_fail(LDPC_EINVAL, "bad sizes (users 1..32, hidden 1..1024, branches 1..32)");
  if (n_tti == 0) return LDPC_OK;
  if (!alloc_dev || !w1_dev || !b1_dev || !w2_dev || !b2_dev || !noise_dev || !codebook_dev || !action_dev ||
      !status_dev)
    return policy_fail(LDPC_EINVAL, "null buffer");
  const int threads = ((std::max(std::max(hidden, 32 * n_branch), 2 * n_users) + 31) / 32) * 32;
  if (threads > 1024) return policy_fail(LDPC_EINVAL, "too many threads for one block");
  const size_t smem = sizeof(float) * static_cast<size_t>(n_branch) *
                      static_cast<size_t>((n_users + 1) + hidden + 2 * n_users + n_users);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(reinterpret_cast<const void*>(&rt_odu_kernel),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return launch_status(e);
  }
  rt_odu_kernel<<<n_tti, threads, smem, static_cast<cudaStream_t>(cuda_stream)>>>(
      n_users, hidden, n_branch, L, alloc_dev, w1_dev, b1_dev, w2_dev, b2_dev, noise_dev, codebook_dev, action_dev,
      status_dev);
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
