// Continuous-batching decode service: a persistent device loop fed through
// rings in pinned host memory (see the serving section of ldpcgb.h).
//
// Host -> device: work items (up to G code blocks of one TB), code-block
// records and request records live in pinned, mapped host memory; the host
// writes them with plain stores, then publishes the new ring tail after a
// release fence.  Each thread block of the device loop claims the next
// published item with a compare-and-swap on a device head counter (so a
// block that gives up waiting never strands a claimed item), reads its
// records with system-scope loads, demaps the blocks' symbols from the host
// pool directly into shared memory, decodes them, and writes bits and status
// into the device arena.  The block that finishes a request's last item runs
// the TB CRC-24, copies the decoded bits to the host result pool and writes a
// completion record to a host ring, sequence number last after a system
// fence.  All waits are bounded by %globaltimer.
//
// INT8 items come in two forms, chosen per request at admission by load
// (host_rules.h): single (one code block per thread group, check messages in
// shared memory) or paired (two blocks per thread group in half2, messages in
// a device-memory slot per group); one loop kernel holds both bodies.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <limits>
#include <map>
#include <set>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include <sys/resource.h>

#include "arena.h"
#include "host_rules.h"
#include "crc_core.cuh"
#include "decode_core.cuh"
#include "demap_core.cuh"

namespace ldpcgb {
namespace {

constexpr int kServeBlock = 384;
constexpr int kServeStats = 11;  // entries of ldpc_serve_stats
constexpr int kMaxTbCb = 16;
constexpr int kServeXpowWords = kMaxTbCb * 8448 / 32 * 2;  // TB CRC shift table: words of the largest TB

struct ServeItem {  // host ring entry
  int32_t req, cb0, count, n_items;
  int32_t pair;  // INT8: decode the item's blocks two per thread group
  int32_t pad;
};

struct ServeReq {  // host record per request slot
  uint64_t tag;
  int32_t n_cb, words, shape;
  int32_t seg;         // 1: every code block ends in its own CRC (LDPC_CB_CRC24B)
  int64_t bits_off;    // arena word offset of the TB's decoded bits (contiguous)
  int64_t status_off;  // arena word offset of its status words
  int64_t result_off;  // byte offset into the result pool, -1 for none
  int32_t pattern;     // URLLC codebook entry puncturing the TB, -1: mask words in the host pool
  int32_t grid_sc;     // pattern >= 0: first SC of the TB's band on its slot's grid
  int32_t n_sc;        // the band's width in SCs (TB resource element i: symbol i / n_sc, SC i % n_sc)
  int32_t pad;
};

struct ServeDone {  // device -> host completion record
  uint64_t tag;
  int32_t d, max_iters, all_ok, req;
  uint32_t seq, pad;
  uint64_t t_dev;  // global timer at the write
};

struct HostCtl {  // host-written control words
  uint32_t tail;
  uint32_t stop;
  uint32_t pad[14];
};

struct DevCtl {  // device counters
  uint32_t head, done, err;
  uint32_t exits;  // blocks of the current loop launch that have left it (zeroed at each launch)
};

struct LoopCtl {  // device-written, host-mapped: lets the host see the loop end without a driver call
  uint32_t exited_epoch;  // launch number of the last loop all of whose blocks have exited
  uint32_t pad[15];
};

struct ServeShape {  // one (bg, Z) shape with its shared-memory layouts in the loop
  ShapeDev sh;   // table in four-edge chunks, for the single form
  ShapeDev shp;  // table in two-edge chunks, for the paired form (INT8)
  int32_t G, region_bytes, L_bytes, hb_bytes, rec_cap, dummy_base, feasible;
  int32_t Gp, region_p, Lp_bytes, feasible_p;  // paired form: groups, region, posterior bytes
  int32_t pad;
};

struct ServeArgs {
  const ServeShape* shapes;
  const uint32_t* tabs;
  const ServeItem* items;
  uint32_t item_cap;
  const CbDev* cbs;  // code-block records: re_off/mask_off index the host pool (elements/words),
                     // bits_off and llr_off (status index) the arena
  uint32_t cb_cap;
  const ServeReq* reqs;
  ServeDone* done;
  uint32_t done_cap;
  const HostCtl* hctl;
  DevCtl* dctl;
  LoopCtl* lctl;
  uint32_t epoch;  // this launch's number
  uint32_t* counts;  // per request slot: items finished
  uint32_t* arena;
  const uint8_t* host_pool;
  uint8_t* result_pool;
  const uint32_t* crc_table;
  const uint32_t* xpow32;
  const uint32_t* crc_table_b;  // code-block CRC: byte table, x^(32 m) mod g_B, position tables
  const uint32_t* xpow32_b;
  const uint32_t* cbcrc;
  const uint32_t* book;  // URLLC codebook: per entry 7 mini-slot bitmaps of book_wpm words
  int32_t book_wpm, book_prb, book_n;  // words per mini-slot bitmap, pattern period in PRBs, entries
  int32_t hdr_bytes, interleave, max_iter, early_term;
  float q_scale, llr_sat, beta, msg_sat, post_sat;
  uint64_t idle_ns;
  uint8_t* rscratch;       // device-memory messages (paired form; FP32 single form): one slot per (loop block, group)
  int64_t rscratch_group;  // bytes per group slot
  int32_t groups;          // message slots per loop block (the most groups of any shape with device-memory messages)
  // sizes the checked build tests indices against
  int32_t n_shapes, n_req;
  int64_t arena_words, pool_f2, pool_words;
};

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t ld_acquire_sys(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

template <typename T>
__device__ __forceinline__ T ld_sys(const T* p) {
  return *const_cast<const volatile T*>(p);
}

// Request inputs are written by the host before the request is published
// (release) and read after the tail is acquired, and never change while the
// request is in flight: L2-coherent loads that skip L1 (.cg) are safe and,
// unlike volatile loads, can be overlapped.
__device__ __forceinline__ float2 ld_pool_f2(const float2* p) { return __ldcg(p); }
__device__ __forceinline__ uint32_t ld_pool_u32(const uint32_t* p) { return __ldcg(p); }

// Claim the next published work item: its index, -1 if stopped, -2 after the idle limit.
__device__ int64_t claim_item(const ServeArgs& a) {
  const uint64_t t0 = gtimer();
  unsigned ns = 32;
  for (;;) {
    const uint32_t tail = ld_acquire_sys(&a.hctl->tail);
    const uint32_t h = atomicAdd(&a.dctl->head, 0u);
    if (h != tail) {
      if (atomicCAS(&a.dctl->head, h, h + 1u) == h) return static_cast<int64_t>(h);
      continue;
    }
    if (ld_sys(&a.hctl->stop)) return -1;
    if (gtimer() - t0 > a.idle_ns) return -2;
    __nanosleep(ns);
    ns = ns < 1024 ? ns * 2 : 1024;
  }
}

__device__ CbDev load_cb(const CbDev* p) {
  CbDev c;
  const volatile int32_t* s = reinterpret_cast<const volatile int32_t*>(p);
  int32_t* d = reinterpret_cast<int32_t*>(&c);
#pragma unroll
  for (int i = 0; i < static_cast<int>(sizeof(CbDev) / 4); ++i) d[i] = s[i];
  return c;
}

// Where the demapper writes: a block's LLRs (LT values), or one half of each
// half2 posterior word of the paired INT8 loop (half 0: block A, 1: block B).
template <typename LT>
struct PlainOut {
  LT* p;
  __device__ PlainOut shift(int n) const { return PlainOut{p + n}; }
  __device__ LT& operator[](int i) const { return p[i]; }
};

struct PairLaneOut {
  __half* p;
  int lane;
  struct Ref {
    __half* q;
    __device__ void operator=(int8_t v) const { *q = __short2half_rn(v); }
  };
  __device__ PairLaneOut shift(int n) const { return PairLaneOut{p + 2 * n, lane}; }
  __device__ Ref operator[](int i) const { return Ref{p + 2 * i + lane}; }
};

// Which resource elements of a code block URLLC punctured: bit r of the
// block's mask words in the host pool, or, for a request that names a
// codebook entry, the entry's bitmap at the element's place on the slot's
// grid.  TB resource element i = re0 + r (re0 = block index * n_re) sits on
// OFDM symbol i / n_sc (mini-slot symbol / 2) and SC grid_sc + i % n_sc,
// i.e. PRB (SC / 12); the entry's bitmaps repeat every book_prb PRBs.
struct PunctSrc {
  const uint32_t* words;  // mask words (book == nullptr)
  const uint32_t* book;   // the entry's 7 bitmaps
  int wpm, prb_period, re0, n_sc, grid_sc;
  __device__ __forceinline__ bool operator()(int r) const {
    if (book == nullptr) return ((ld_pool_u32(words + (r >> 5)) >> (r & 31)) & 1u) != 0u;
    const int i = re0 + r;
    const int sym = i / n_sc;
    const int prb = ((grid_sc + (i - sym * n_sc)) / 12) % prb_period;
    return ((__ldg(book + (sym >> 1) * wpm + (prb >> 5)) >> (prb & 31)) & 1u) != 0u;
  }
};

struct ReqPunct {  // a request's puncturing, read once per item
  int pattern, grid_sc, n_sc, slot;
};

__device__ __forceinline__ PunctSrc punct_src(const ServeArgs& a, const ReqPunct& rp, const CbDev& cb, int cb_index) {
  PunctSrc ps{};
  if (rp.pattern < 0) {
    ps.words = reinterpret_cast<const uint32_t*>(a.host_pool) + cb.mask_off;
    return ps;
  }
  ps.book = a.book + static_cast<int64_t>(rp.pattern) * 7 * a.book_wpm;
  ps.wpm = a.book_wpm;
  ps.prb_period = a.book_prb;
  ps.re0 = (cb_index - rp.slot * kMaxTbCb) * cb.n_re;  // each request slot owns kMaxTbCb block records
  ps.n_sc = rp.n_sc;
  ps.grid_sc = rp.grid_sc;
  return ps;
}

template <typename LT, bool Q = (sizeof(LT) < 4), typename Out>
__device__ __forceinline__ void demap_into_smem(const ServeArgs& a, const CbDev& cb, const PunctSrc& ps, Out L, int k,
                                                int Z) {
  using namespace demapcore;
  const int ncb = cb.n_eff * Z - cb.t0;  // circular buffer: E > ncb repeats it
  for (int p = k; p < cb.t0; p += Z) L[p] = LT(0);
  // buffer offsets k0 + j (mod ncb), j from E to ncb: those the version does not reach
  for (int j = min(cb.E, ncb) + k; j < ncb; j += Z) {
    const int q = cb.k0 + j;
    L[cb.t0 + (q >= ncb ? q - ncb : q)] = LT(0);
  }
  const float2* sym = reinterpret_cast<const float2*>(a.host_pool) + cb.re_off;
  const Out out = L.shift(cb.t0);
#pragma unroll 4
  for (int r = k; r < cb.n_re; r += Z) {
    const float2 y = ld_pool_f2(sym + r);
    const bool punct = ps(r);
    auto ls = [&](int i) { return ld_pool_f2(sym + i); };
    auto lm = [&](int i) { return ps(i); };
    switch (cb.Qm) {
      case 2: demap_re_into<LT, 2, Q>(y, punct, cb.inv_sigma2, out, r, cb.n_re, cb.E, ncb, cb.k0, a.interleave, a.q_scale, a.llr_sat, ls, lm); break;
      case 4: demap_re_into<LT, 4, Q>(y, punct, cb.inv_sigma2, out, r, cb.n_re, cb.E, ncb, cb.k0, a.interleave, a.q_scale, a.llr_sat, ls, lm); break;
      case 6: demap_re_into<LT, 6, Q>(y, punct, cb.inv_sigma2, out, r, cb.n_re, cb.E, ncb, cb.k0, a.interleave, a.q_scale, a.llr_sat, ls, lm); break;
      default: demap_re_into<LT, 8, Q>(y, punct, cb.inv_sigma2, out, r, cb.n_re, cb.E, ncb, cb.k0, a.interleave, a.q_scale, a.llr_sat, ls, lm); break;
    }
  }
}

// Per-item bookkeeping, by every thread of the block: the block that finishes
// a request's last item runs its TB CRC-24 (and the code-block CRCs of a
// segmented TB), copies the bits to the result pool and writes the completion
// record (sequence word last, after a system fence).
__device__ __forceinline__ void finish_item(const ServeArgs& a, int req, int n_items, int tid, int lane, int* s_last,
                                            uint32_t* s_res) {
  // ---- request bookkeeping: the block finishing the last item completes the TB
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    const uint32_t prev = atomicAdd(a.counts + req, 1u);
    *s_last = (prev + 1u == static_cast<uint32_t>(n_items)) ? 1 : 0;
    if (*s_last) {
      a.counts[req] = 0u;
      __threadfence();
    }
  }
  __syncthreads();
  if (*s_last) {
    const ServeReq* rq = a.reqs + req;
    const uint64_t tag = ld_sys(&rq->tag);
    const int n_cb = ld_sys(&rq->n_cb);
    const int W = ld_sys(&rq->words);
    const int seg = ld_sys(&rq->seg);
    const int64_t bits_off = ld_sys(&rq->bits_off);
    const int64_t status_off = ld_sys(&rq->status_off);
    const int64_t result_off = ld_sys(&rq->result_off);
    const volatile uint32_t* bits = a.arena + bits_off;
    const bool rq_ok = check_ok(n_cb >= 1 && n_cb <= kMaxTbCb && W % n_cb == 0, 18, n_cb, W) &&
                       check_ok(bits_off >= 0 && bits_off + W <= a.arena_words, 19, static_cast<int>(bits_off),
                                static_cast<int>(a.arena_words)) &&
                       check_ok(status_off >= 0 && status_off + n_cb <= a.arena_words, 20,
                                static_cast<int>(status_off), static_cast<int>(a.arena_words));
    if (tid < 32 && rq_ok) {
      using namespace crccore;
      // TB CRC over each block's first K/8 - 3*seg bytes (the blocks' K/32
      // words lie back to back), zero-prefixed to whole words as in the
      // batch CRC kernel
      const int kw = W / n_cb;                  // words per block
      const int cbb = 4 * kw - 3 * seg;         // TB bytes per block
      const int tbytes = n_cb * cbb;
      const int pad = (-tbytes) & 3;
      const int VW = (tbytes + pad) >> 2;
      const int per = (VW + 31) >> 5;
      const int w0 = min(VW, lane * per);
      const int w1 = min(VW, w0 + per);
      uint32_t state = 0;
      int b = max(0, 4 * w0 - pad);
      int blk = b / cbb;
      int j = b - blk * cbb;
      int jw = -1;
      uint32_t v = 0;
      for (; b < 4 * w1 - pad; ++b) {
        if ((j >> 2) != jw) {
          jw = j >> 2;
          v = bits[blk * kw + jw];
        }
        state = crc_byte_step(state, msb_first_byte(v, j), a.crc_table);
        if (++j == cbb) {
          ++blk;
          j = 0;
          jw = -1;
        }
      }
      if (w0 < w1) state = gf2_mulmod(state, a.xpow32[VW - w1]);
  #pragma unroll
      for (int o = 16; o > 0; o >>= 1) state ^= __shfl_xor_sync(0xFFFFFFFFu, state, o);
      // and each block's own CRC
      for (int c = 0; seg && c < n_cb; ++c) {
        const int pc = (kw + 31) >> 5;
        const int v0 = min(kw, lane * pc);
        const int v1 = min(kw, v0 + pc);
        uint32_t st = 0;
        for (int w = v0; w < v1; ++w) {
          const uint32_t v = bits[c * kw + w];
  #pragma unroll
          for (int j = 0; j < 4; ++j) st = crc_byte_step(st, msb_first_byte(v, j), a.crc_table_b);
        }
        if (v0 < v1) st = gf2_mulmod(st, a.xpow32_b[kw - v1], kPolyFullB);
  #pragma unroll
        for (int o = 16; o > 0; o >>= 1) st ^= __shfl_xor_sync(0xFFFFFFFFu, st, o);
        state |= st;
      }
      // status words come from other SMs' blocks: read past this SM's L1 like the bits
      uint32_t st = lane < n_cb ? ld_sys(a.arena + status_off + lane) : (1u << 16);
      uint32_t iters = st & 0xFFFFu;
      uint32_t okb = (st >> 16) & 1u;
  #pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        iters = max(iters, __shfl_xor_sync(0xFFFFFFFFu, iters, o));
        okb &= __shfl_xor_sync(0xFFFFFFFFu, okb, o);
      }
      if (lane == 0) {
        s_res[0] = state == 0u ? 1u : 0u;
        s_res[1] = iters;
        s_res[2] = okb;
      }
    }
    if (result_off >= 0) {
      volatile uint32_t* res = reinterpret_cast<volatile uint32_t*>(a.result_pool + result_off);
      for (int i = tid; i < W; i += blockDim.x) res[i] = bits[i];
    }
    __threadfence_system();
    __syncthreads();
    if (tid == 0) {
      const uint32_t slot = atomicAdd(&a.dctl->done, 1u);
      volatile ServeDone* rec = a.done + (slot % a.done_cap);
      rec->tag = tag;
      rec->d = static_cast<int32_t>(s_res[0]);
      rec->max_iters = static_cast<int32_t>(s_res[1]);
      rec->all_ok = static_cast<int32_t>(s_res[2]);
      rec->req = req;
      rec->t_dev = gtimer();
      __threadfence_system();
      rec->seq = slot + 1u;
      __threadfence_system();
    }
  }
}

// Decode of one item's blocks, one block per thread group (single form).
// Loads the shape's table (bulk copy), demaps straight into shared memory,
// runs the layered decoder, writes bits and status to the arena.  Returns
// false if the table copy did not complete within its bounded wait.
// RG: the check messages live in a device-memory slot per (loop block, group),
// as the paired form's do (FP32: a block's 12-byte records do not fit shared
// memory beside its posteriors for the large shapes), else in shared memory.
template <typename LT, typename MT, bool SAT, bool CRC, bool RG>
__device__ __forceinline__ bool single_item(const ServeArgs& a, const ServeShape& ssh, const CbDev& cb_first,
                                            const ReqPunct& rp, int cb0, int count, uint32_t& phase,
                                            uint32_t* s_tab, uint64_t* s_bar, uint8_t* regions) {
  using namespace core;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const ShapeDev& sh = ssh.sh;
  const int Z = sh.Z;
  const int g = tid / Z;
  const int k = tid - g * Z;
  const uint32_t wmask = (Z >= 32) ? 0xFFFFFFFFu : (((1u << Z) - 1u) << (lane & ~(Z - 1)));
  if (tid == 0) {
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(s_bar, static_cast<uint32_t>(sh.tab_words) * 4u);
    bulk_g2s(s_tab, a.tabs + sh.tab_off, static_cast<uint32_t>(sh.tab_words) * 4u, s_bar);
  }
  bool active = g < count && check_ok(count >= 1 && count <= ssh.G, 12, count, ssh.G);
  CbDev cb{};
  LT* L = reinterpret_cast<LT*>(regions + g * ssh.region_bytes);
  uint8_t* rbase = RG ? a.rscratch + (static_cast<int64_t>(blockIdx.x) * a.groups + g) * a.rscratch_group
                      : regions + g * ssh.region_bytes + ssh.L_bytes + ssh.hb_bytes;
  MT* mag1 = reinterpret_cast<MT*>(rbase);
  MT* mag2 = mag1 + ssh.rec_cap;
  uint32_t* meta = reinterpret_cast<uint32_t*>(rbase + 2 * ((ssh.rec_cap * sizeof(MT) + 15) & ~15));
  if (active) {
    cb = load_cb(a.cbs + (static_cast<uint32_t>(cb0 + g) % a.cb_cap));
    if constexpr (kChecked) {  // the block's records against the shape, the arena and the host pool
      active = check_ok(cb.shape == cb_first.shape && cb.Z == Z && cb.n_eff <= sh.nb && cb.m_eff <= sh.mb, 13,
                        cb.shape, cb_first.shape) &&
               check_ok(cb.bits_off >= 0 && cb.bits_off + ((cb.kb * Z) >> 5) <= a.arena_words, 14,
                        static_cast<int>(cb.bits_off), static_cast<int>(a.arena_words)) &&
               check_ok(cb.llr_off >= 0 && cb.llr_off < a.arena_words, 15, static_cast<int>(cb.llr_off),
                        static_cast<int>(a.arena_words)) &&
               check_ok(cb.re_off >= 0 && cb.re_off + cb.n_re <= a.pool_f2, 16, static_cast<int>(cb.re_off),
                        static_cast<int>(a.pool_f2)) &&
               check_ok(rp.pattern >= 0 || (cb.mask_off >= 0 && cb.mask_off + ((cb.n_re + 31) >> 5) <= a.pool_words),
                        17, static_cast<int>(cb.mask_off), static_cast<int>(a.pool_words)) &&
               check_ok(rp.pattern < a.book_n && rp.n_sc > 0, 21, rp.pattern, a.book_n);
    }
  }
  if (active) {
    zero_records(mag1, mag2, meta, cb.m_eff * Z, k, Z);
    if constexpr (SAT)
      st_val(L, ssh.dummy_base + k, a.post_sat);
    else
      L[ssh.dummy_base + k] = LT(kBigF);
    // puncture flushing + max-log, straight into shared memory
    const int ci = static_cast<int>(static_cast<uint32_t>(cb0 + g) % a.cb_cap);
    demap_into_smem<LT, SAT>(a, cb, punct_src(a, rp, cb, ci), PlainOut<LT>{L}, k, Z);
  }
  const bool got = mbar_wait_bounded(s_bar, phase, 1u << 22);
  phase ^= 1u;
  if (!__syncthreads_and(got)) {
    if (tid == 0) atomicOr(&a.dctl->err, LDPC_DEVERR_TMA_TIMEOUT);
    mbar_wait_bounded(s_bar, phase ^ 1u, 1u << 20);
    return false;
  }
  if (active) {
    const uint32_t* rows = s_tab + sh.row_off;
    uint32_t* hb = reinterpret_cast<uint32_t*>(regions + g * ssh.region_bytes + ssh.L_bytes);
    const int m = cb.m_eff;
    const bool wide = (Z & 31) == 0;
    int it = 1;
    bool ok = false, crc_ok = false;
    const bool has_crc = CRC && (cb.flags & LDPC_CB_CRC24B) != 0;
    RowIn<kServeChunk> row = load_row<kServeChunk>(s_tab, rows[0], mag1, mag2, meta, k);
    for (;; ++it) {
      for (int l = 0; l < m; ++l) {
        check_update_exact<LT, MT, SAT, false, kServeChunk>(row, k, Z, L, mag1, mag2, meta, l * Z + k,
                                                            ssh.dummy_base + k, a.beta, a.msg_sat, a.post_sat);
        // the next row's table and record are ready before the barrier
        const int ln = l + 1 < m ? l + 1 : 0;
        row = load_row<kServeChunk>(s_tab, rows[ln], mag1, mag2, meta, ln * Z + k);
        group_sync(Z, g, wmask);
      }
      if (a.early_term || it == a.max_iter) {
        bool bad;
        uint32_t cr = 0;
        const uint32_t* ptab = a.cbcrc + sh.crc_off;
        if (wide) {
          hard_bitmap(L, hb, cb.n_eff, k, Z);
          group_sync(Z, g, wmask);
          bad = syndrome_bitmap<kServeChunk>(s_tab, rows, hb, m, k, Z);
          if (has_crc) cr = cb_crc_part_hb(hb, ptab, cb.kb, k, Z);
        } else {
          bad = syndrome_direct<kServeChunk>(s_tab, rows, m, k, Z, L);
          if (has_crc) cr = cb_crc_part(L, ptab, cb.kb, k, Z);
        }
        ok = !group_any(Z, g, wmask, bad);
        // after that barrier the bitmap's parity words are free: scratch for the CRC's XOR
        if (has_crc) crc_ok = group_xor_zero(Z, g, wmask, cr, hb + cb.kb * (Z >> 5), k);
        if ((ok || crc_ok) && a.early_term) break;
        if (it == a.max_iter) break;
      }
    }
    uint32_t* out = a.arena + cb.bits_off;
    if (wide) {
      const int nw = cb.kb * (Z >> 5);
      for (int i = k; i < nw; i += Z) out[i] = hb[i];
    } else {
      const int sh16 = lane & 16;
      for (int c = 0; c < cb.kb; c += 2) {
        const uint32_t b0 = __ballot_sync(wmask, L[c * Z + k] < LT(0)) >> sh16;
        const uint32_t b1 = __ballot_sync(wmask, L[(c + 1) * Z + k] < LT(0)) >> sh16;
        if (k == 0) out[c >> 1] = (b0 & 0xFFFFu) | (b1 << 16);
      }
    }
    if (k == 0) a.arena[cb.llr_off] = static_cast<uint32_t>(it | (ok ? (1 << 16) : 0) | (crc_ok ? (1 << 17) : 0));
  }
  return true;
}

// The same for INT8 with two blocks per thread group (paired form, the batch
// decoder's half2 arithmetic: block A in the low half, B in the high half;
// every INT8 intermediate is an integer exact in fp16).  The item holds up to
// 2 Gp blocks of one TB (identical geometry), group g decodes blocks 2g and
// 2g+1; the three message words per check sit in a device-memory slot per
// (block, group); the table (the shape's two-edge-chunk copy), posteriors and
// both bitmaps in shared memory.
template <bool CRC>
__device__ __forceinline__ bool pair_item(const ServeArgs& a, const ServeShape& ssh, const CbDev& cb_first,
                                          const ReqPunct& rp, int cb0, int count, uint32_t& phase, uint32_t* s_tab,
                                          uint64_t* s_bar, uint8_t* regions) {
  using namespace core;
  const int tid = threadIdx.x;
  const ShapeDev& sh = ssh.shp;
  const int Z = sh.Z;
  const int g = tid / Z;
  const int k = tid - g * Z;
  const __half2 beta = __float2half2_rn(a.beta);
  const __half2 msg = __float2half2_rn(a.msg_sat);
  const __half2 post = __float2half2_rn(a.post_sat);
  if (tid == 0) {
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(s_bar, static_cast<uint32_t>(sh.tab_words) * 4u);
    bulk_g2s(s_tab, a.tabs + sh.tab_off, static_cast<uint32_t>(sh.tab_words) * 4u, s_bar);
  }
  const int pairs = (count + 1) >> 1;
  bool active = g < pairs && check_ok(count >= 1 && count <= 2 * ssh.Gp, 12, count, 2 * ssh.Gp);
  const bool hasB = 2 * g + 1 < count;
  uint8_t* reg = regions + g * ssh.region_p;
  uint32_t* L = reinterpret_cast<uint32_t*>(reg);
  uint32_t* hbA = reinterpret_cast<uint32_t*>(reg + ssh.Lp_bytes);
  uint32_t* hbB = reinterpret_cast<uint32_t*>(reg + ssh.Lp_bytes + ssh.hb_bytes);
  // per check: (magnitudes, s1) as one 8-byte pair, then s2
  uint2* ms = reinterpret_cast<uint2*>(a.rscratch + (static_cast<int64_t>(blockIdx.x) * a.groups + g) *
                                                        a.rscratch_group);
  uint32_t* sg2 = reinterpret_cast<uint32_t*>(ms) + 2 * ssh.rec_cap;
  CbDev A{}, B{};
  if (active) {
    A = load_cb(a.cbs + (static_cast<uint32_t>(cb0 + 2 * g) % a.cb_cap));
    if (hasB) B = load_cb(a.cbs + (static_cast<uint32_t>(cb0 + 2 * g + 1) % a.cb_cap));
    if constexpr (kChecked) {
      for (int h = 0; h < (hasB ? 2 : 1); ++h) {
        const CbDev& c = h ? B : A;
        active = active &&
                 check_ok(c.shape == cb_first.shape && c.Z == Z && c.n_eff == A.n_eff && c.m_eff == A.m_eff &&
                              c.n_eff <= sh.nb && c.m_eff <= sh.mb, 13, c.shape, cb_first.shape) &&
                 check_ok(c.bits_off >= 0 && c.bits_off + ((c.kb * Z) >> 5) <= a.arena_words, 14,
                          static_cast<int>(c.bits_off), static_cast<int>(a.arena_words)) &&
                 check_ok(c.llr_off >= 0 && c.llr_off < a.arena_words, 15, static_cast<int>(c.llr_off),
                          static_cast<int>(a.arena_words)) &&
                 check_ok(c.re_off >= 0 && c.re_off + c.n_re <= a.pool_f2, 16, static_cast<int>(c.re_off),
                          static_cast<int>(a.pool_f2)) &&
                 check_ok(rp.pattern >= 0 ||
                              (c.mask_off >= 0 && c.mask_off + ((c.n_re + 31) >> 5) <= a.pool_words),
                          17, static_cast<int>(c.mask_off), static_cast<int>(a.pool_words)) &&
                 check_ok(rp.pattern < a.book_n && rp.n_sc > 0, 21, rp.pattern, a.book_n);
      }
    }
  }
  if (active) {
    for (int r = k; r < A.m_eff * Z; r += Z) {
      ms[r] = make_uint2(0u, 0u);
      sg2[r] = 0u;
    }
    // both blocks' LLRs into the two halves of the posterior words (B's half 0 without a second block)
    __half* Lh = reinterpret_cast<__half*>(L);
    const int ciA = static_cast<int>(static_cast<uint32_t>(cb0 + 2 * g) % a.cb_cap);
    demap_into_smem<int8_t>(a, A, punct_src(a, rp, A, ciA), PairLaneOut{Lh, 0}, k, Z);
    if (hasB) {
      demap_into_smem<int8_t>(a, B, punct_src(a, rp, B, ciA + 1), PairLaneOut{Lh, 1}, k, Z);
    } else {
      for (int p = k; p < A.n_eff * Z; p += Z) Lh[2 * p + 1] = __float2half(0.0f);
    }
  }
  const bool got = mbar_wait_bounded(s_bar, phase, 1u << 22);
  phase ^= 1u;
  if (!__syncthreads_and(got)) {
    if (tid == 0) atomicOr(&a.dctl->err, LDPC_DEVERR_TMA_TIMEOUT);
    mbar_wait_bounded(s_bar, phase ^ 1u, 1u << 20);
    return false;
  }
  if (active) {
    const uint32_t* rows = s_tab + sh.row_off;
    const int m = A.m_eff;
    const int dummy = ssh.dummy_base + k;
    bool doneA = false, doneB = !hasB;
    PairIn prow = load_pair_row(s_tab, rows[0], ms, sg2, k);
    for (int it = 1;; ++it) {
      for (int l = 0; l < m; ++l) {
        check_update_x2_by_degree(prow, k, Z, L, ms, sg2, l * Z + k, dummy, beta, msg, post);
        const int ln = l + 1 < m ? l + 1 : 0;
        prow = load_pair_row(s_tab, rows[ln], ms, sg2, ln * Z + k);
        group_sync(Z, g, 0xFFFFFFFFu);
      }
      if (a.early_term || it == a.max_iter) {
        hard_bitmap_x2(L, hbA, hbB, A.n_eff, k, Z);
        group_sync(Z, g, 0xFFFFFFFFu);
        const bool badA = !doneA && syndrome_bitmap<kChunk>(s_tab, rows, hbA, m, k, Z);
        const bool badB = !doneB && syndrome_bitmap<kChunk>(s_tab, rows, hbB, m, k, Z);
        const bool crcA = CRC && !doneA && (A.flags & LDPC_CB_CRC24B) != 0;
        const bool crcB = CRC && !doneB && (B.flags & LDPC_CB_CRC24B) != 0;
        uint32_t rA = 0, rB = 0;
        if (crcA || crcB) {
          const uint32_t* ptab = a.cbcrc + sh.crc_off;
          if (crcA) rA = cb_crc_part_hb(hbA, ptab, A.kb, k, Z);
          if (crcB) rB = cb_crc_part_hb(hbB, ptab, A.kb, k, Z);
        }
        const bool okA = !group_any(Z, g, 0xFFFFFFFFu, badA);
        const bool okB = !group_any(Z, g, 0xFFFFFFFFu, badB);
        bool cA = false, cB = false;
        if (crcA || crcB) {  // both blocks' XORs meet in their bitmaps' (now free) parity words
          const bool zA = group_xor_zero2(Z, g, rA, rB, hbA + A.kb * (Z >> 5), hbB + A.kb * (Z >> 5), k, &cB);
          cA = crcA && zA;
          cB = crcB && cB;
        }
        const bool last = it == a.max_iter;
        const int nw = A.kb * (Z >> 5);
        if (!doneA && (((okA || cA) && a.early_term) || last)) {
          uint32_t* out = a.arena + A.bits_off;
          for (int i = k; i < nw; i += Z) out[i] = hbA[i];
          if (k == 0) a.arena[A.llr_off] = static_cast<uint32_t>(it | (okA ? (1 << 16) : 0) | (cA ? (1 << 17) : 0));
          doneA = true;
        }
        if (!doneB && (((okB || cB) && a.early_term) || last)) {
          uint32_t* out = a.arena + B.bits_off;
          for (int i = k; i < nw; i += Z) out[i] = hbB[i];
          if (k == 0) a.arena[B.llr_off] = static_cast<uint32_t>(it | (okB ? (1 << 16) : 0) | (cB ? (1 << 17) : 0));
          doneB = true;
        }
        if (doneA && doneB) break;
      }
    }
  }
  return true;
}

// The persistent loop, one thread block per SM.  PAIRS (INT8): an item the
// host flagged as paired runs pair_item, the others single_item -- the host
// pairs while the service is loaded (more blocks in flight per SM) and not
// while it is light (lower latency per block).
template <typename LT, typename MT, bool SAT, bool CRC, bool PAIRS>
__global__ void __launch_bounds__(kServeBlock, 1) serve_kernel(const ServeArgs a) {
  extern __shared__ __align__(128) uint8_t smem[];
  uint32_t* s_tab = reinterpret_cast<uint32_t*>(smem);
  uint64_t* s_bar = reinterpret_cast<uint64_t*>(smem + a.hdr_bytes - 16);
  uint8_t* regions = smem + a.hdr_bytes;
  __shared__ long long s_claim;
  __shared__ int s_last;
  __shared__ uint32_t s_res[3];  // d, most iterations, all syndromes zero

  const int tid = threadIdx.x;
  const int lane = tid & 31;
  if (tid == 0) {
    mbar_init(s_bar, 1);
    fence_proxy_async_smem();
  }
  __syncthreads();
  uint32_t phase = 0;

  for (;;) {
    if (tid == 0) s_claim = claim_item(a);  // -2 (idle): exit quietly, the host relaunches on demand
    __syncthreads();
    const long long idx = s_claim;
    if (idx < 0) break;
    const ServeItem* ip = a.items + (static_cast<uint32_t>(idx) % a.item_cap);
    const int req = ld_sys(&ip->req), cb0 = ld_sys(&ip->cb0), count = ld_sys(&ip->count);
    const int n_items = ld_sys(&ip->n_items);
    const bool paired = PAIRS && ld_sys(&ip->pair) != 0;
    const int first_cb = static_cast<int>(static_cast<uint32_t>(cb0) % a.cb_cap);
    const CbDev cb_first = load_cb(a.cbs + first_cb);
    // checked builds: an item whose request or shape index is out of range is dropped
    const bool item_ok = check_ok(static_cast<uint32_t>(req) < static_cast<uint32_t>(a.n_req), 10, req, a.n_req) &&
                         check_ok(static_cast<uint32_t>(cb_first.shape) < static_cast<uint32_t>(a.n_shapes), 11,
                                  cb_first.shape, a.n_shapes);
    if (kChecked && !item_ok) {
      __syncthreads();
      continue;
    }
    const ServeShape ssh = a.shapes[cb_first.shape];
    const ServeReq* rq = a.reqs + req;
    const ReqPunct rp{ld_sys(&rq->pattern), ld_sys(&rq->grid_sc), ld_sys(&rq->n_sc), req};
    bool fine;
    if constexpr (PAIRS) {
      fine = paired ? pair_item<CRC>(a, ssh, cb_first, rp, cb0, count, phase, s_tab, s_bar, regions)
                    : single_item<LT, MT, SAT, CRC, (sizeof(MT) == 4)>(a, ssh, cb_first, rp, cb0, count, phase, s_tab, s_bar, regions);
    } else {
      fine = single_item<LT, MT, SAT, CRC, (sizeof(MT) == 4)>(a, ssh, cb_first, rp, cb0, count, phase, s_tab, s_bar, regions);
    }
    if (!fine) break;
    finish_item(a, req, n_items, tid, lane, &s_last, s_res);
    __syncthreads();
  }
  // the last block to leave tells the host (in mapped memory) that this launch is over
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    if (atomicAdd(&a.dctl->exits, 1u) + 1u == gridDim.x) {
      __threadfence_system();
      *reinterpret_cast<volatile uint32_t*>(&a.lctl->exited_epoch) = a.epoch;
    }
  }
}

template <bool CRC>
const void* serve_kernel_for(int mode, bool pairs) {
  switch (mode) {
    case LDPC_F32: return reinterpret_cast<const void*>(&serve_kernel<float, float, false, CRC, false>);
    // INT8: the single form keeps its posteriors as floats holding the
    // quantised integers (no int8 conversion per edge access; the same
    // values and arithmetic), its messages as bytes
    case LDPC_I8:
      return pairs ? reinterpret_cast<const void*>(&serve_kernel<float, uint8_t, true, CRC, true>)
                   : reinterpret_cast<const void*>(&serve_kernel<float, uint8_t, true, CRC, false>);
    default: return reinterpret_cast<const void*>(&serve_kernel<int16_t, uint16_t, true, CRC, false>);
  }
}

const void* serve_kernel_ptr(int mode, bool crc, bool pairs) {
  return crc ? serve_kernel_for<true>(mode, pairs) : serve_kernel_for<false>(mode, pairs);
}

}  // namespace

cudaError_t read_check_log_serve(uint32_t* out4) { return cudaMemcpyFromSymbol(out4, g_check_log, 16); }

namespace {

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

int align16s(int x) { return (x + 15) & ~15; }

}  // namespace
}  // namespace ldpcgb

using namespace ldpcgb;

struct ldpc_server {
  ldpc_session* s = nullptr;
  int mode = LDPC_I8;
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaEvent_t done_ev = nullptr;
  bool running = false;
  uint32_t epoch = 0;  // loop launches so far
  // host-mapped rings
  HostCtl* hctl = nullptr;
  LoopCtl* lctl = nullptr;
  ServeItem* items = nullptr;
  CbDev* cbs = nullptr;
  ServeReq* reqs = nullptr;
  ServeDone* done = nullptr;
  uint32_t item_cap = 0, cb_cap = 0, done_cap = 0;
  int32_t max_inflight = 0;
  // device
  DevCtl* dctl = nullptr;
  uint32_t* counts = nullptr;
  uint32_t* arena = nullptr;
  ServeShape* shapes = nullptr;
  uint32_t* tabs = nullptr;
  uint32_t* xpow32 = nullptr;
  uint32_t* crc_table = nullptr;
  uint8_t* rscratch = nullptr;
  uint32_t* book = nullptr;  // URLLC codebook bitmaps
  int32_t book_n = 0, book_prb = 0;
  bool pairs = false;  // INT8: items may run in the paired form (two code blocks per thread group)
  PairPolicy policy;   // which requests take it
  // requests, items single, items paired, loop launches; for the last replay: the longest pass of
  // its host loop (ns), its passes longer than 1 ms, when the longest pass began (ns after the
  // replay started), and the replaying thread's involuntary and voluntary context switches and
  // minor and major page faults during it
  int64_t stats[kServeStats] = {};
  bool cb_crc = false;  // LDPC_SERVE_CB_CRC: TBs with code-block CRCs accepted
  std::vector<ServeShape> hshapes;
  ServeArgs args{};
  int smem = 0, grid = 0;
  const uint8_t* host_pool = nullptr;
  uint64_t host_pool_bytes = 0;
  uint8_t* result_pool = nullptr;
  uint64_t result_pool_bytes = 0;
  // host bookkeeping
  Arena* alloc = nullptr;
  std::vector<int32_t> free_slots;
  struct Slot {
    int64_t arena_off = 0, arena_words = 0;
    int32_t n_items = 0, n_cb = 0;
    int64_t t_submit = 0;
    bool busy = false;  // admitted and not yet completed
  };
  std::vector<Slot> slot_info;
  uint32_t tail = 0;
  uint64_t items_inflight = 0, cbs_inflight = 0;
  uint32_t rd = 0;
};

namespace {

int srv_fail(int code, const std::string& m) {
  set_error(m);
  return code;
}

void free_server(ldpc_server* v) {
  if (!v) return;
  cudaFreeHost(v->hctl);
  cudaFreeHost(v->lctl);
  cudaFreeHost(v->items);
  cudaFreeHost(v->cbs);
  cudaFreeHost(v->reqs);
  cudaFreeHost(v->done);
  cudaFree(v->dctl);
  cudaFree(v->counts);
  cudaFree(v->arena);
  cudaFree(v->shapes);
  cudaFree(v->tabs);
  cudaFree(v->xpow32);
  cudaFree(v->crc_table);
  cudaFree(v->rscratch);
  cudaFree(v->book);
  if (v->done_ev) cudaEventDestroy(v->done_ev);
  if (v->stream) cudaStreamDestroy(v->stream);
  delete v->alloc;
  delete v;
}

int launch_loop(ldpc_server* v) {
  v->args.epoch = ++v->epoch;
  ++v->stats[3];
  cudaError_t z = cudaMemsetAsync(&v->args.dctl->exits, 0, sizeof(uint32_t), v->stream);
  if (z != cudaSuccess) return srv_fail(LDPC_ECUDA, std::string("serve loop reset: ") + cudaGetErrorString(z));
  void* kargs[] = {&v->args};
  cudaError_t e = cudaLaunchKernel(serve_kernel_ptr(v->mode, v->cb_crc, v->pairs), dim3(v->grid), dim3(kServeBlock), kargs,
                                   static_cast<size_t>(v->smem), v->stream);
  if (e != cudaSuccess) return srv_fail(LDPC_ECUDA, std::string("serve loop launch: ") + cudaGetErrorString(e));
  e = cudaEventRecord(v->done_ev, v->stream);
  if (e != cudaSuccess) return srv_fail(LDPC_ECUDA, std::string("cudaEventRecord: ") + cudaGetErrorString(e));
  v->running = true;
  return LDPC_OK;
}

// Relaunch the device loop if it has exited (idle limit reached).
int ensure_running(ldpc_server* v) {
  if (v->running) {
    // no driver call while the loop runs: its last block writes the launch number when it leaves
    if (reinterpret_cast<volatile uint32_t*>(&v->lctl->exited_epoch)[0] != v->epoch) return LDPC_OK;
    const cudaError_t q = cudaEventSynchronize(v->done_ev);  // it has left: the kernel ends at once
    if (q != cudaSuccess) return srv_fail(LDPC_ECUDA, std::string("serve loop: ") + cudaGetErrorString(q));
    v->running = false;
  }
  return launch_loop(v);
}

template <typename T>
int host_alloc(T** p, size_t n) {
  const size_t bytes = std::max<size_t>(n, 1) * sizeof(T);
  cudaError_t e = cudaHostAlloc(reinterpret_cast<void**>(p), bytes, cudaHostAllocMapped);
  if (e != cudaSuccess) return srv_fail(LDPC_ENOMEM, std::string("cudaHostAlloc: ") + cudaGetErrorString(e));
  std::memset(*p, 0, bytes);
  return LDPC_OK;
}

template <typename T>
T* dev_ptr(T* host) {
  void* d = nullptr;
  if (cudaHostGetDevicePointer(&d, host, 0) != cudaSuccess) return nullptr;
  return static_cast<T*>(d);
}

}  // namespace

// Accessors into the session (defined in session.cu).
namespace ldpcgb {
int session_serve_info(ldpc_session* s, int* mode, int* interleave, int* max_iter, int* early_term, float* q_scale,
                       float* llr_sat, float* beta, float* msg_sat, float* post_sat, int* num_sms);
int session_shape_count(ldpc_session* s);
int session_shape_table(ldpc_session* s, int shape, int dummy, std::vector<uint32_t>& tabs, ShapeDev& sh,
                        int chunk);
int session_shape_lookup(ldpc_session* s, int bg, int Z);
const uint32_t* session_crc_table(ldpc_session* s);
void session_cb_crc_tables(ldpc_session* s, const uint32_t** table_b, const uint32_t** xpow32_b,
                           const uint32_t** positions);
}  // namespace ldpcgb

extern "C" {

int ldpc_serve_start(ldpc_session* s, const ldpc_serve_desc* d, ldpc_server** out) {
  try {
    if (!s || !d || !out || !d->host_pool || d->max_inflight < 1 || d->max_inflight > 65536 ||
        d->arena_bytes < 1024 || d->idle_timeout_us < 1 || d->loops_per_sm < 0 || d->loops_per_sm > 2 ||
        d->pair_threshold < 0 || d->pair_release < 0 || (d->flags & ~(LDPC_SERVE_CB_CRC | LDPC_SERVE_UNPAIRED | LDPC_SERVE_PAIRED)) ||
        ((d->flags & LDPC_SERVE_UNPAIRED) && (d->flags & LDPC_SERVE_PAIRED)))
      return srv_fail(LDPC_EINVAL, "ldpc_serve_start: bad descriptor");
    if (d->codebook_n < 0 || d->codebook_n > 65536 ||
        (d->codebook_n > 0 && (!d->codebook || d->codebook_prb < 1 || d->codebook_prb > 65536)))
      return srv_fail(LDPC_EINVAL, "ldpc_serve_start: bad URLLC codebook (codebook_n, codebook_prb, codebook)");
    *out = nullptr;
    auto* v = new (std::nothrow) ldpc_server();
    if (!v) return srv_fail(LDPC_ENOMEM, "host allocation");
    v->s = s;
    // two loops per SM (messages in device memory) are withdrawn: under load that
    // variant once made an illegal access and once returned corrupted status
    // words, and the cause is not found yet, so no service starts it
    if (d->loops_per_sm == 2) {
      delete v;
      return srv_fail(LDPC_EINVAL, "ldpc_serve_start: loops_per_sm = 2 is withdrawn (use 1)");
    }
    v->cb_crc = (d->flags & LDPC_SERVE_CB_CRC) != 0;
    int interleave = 1, max_iter = 10, et = 1, sms = 0;
    float q_scale = 4, llr_sat = 63, beta = 1, msg_sat = 63, post_sat = 127;
    session_serve_info(s, &v->mode, &interleave, &max_iter, &et, &q_scale, &llr_sat, &beta, &msg_sat, &post_sat,
                       &sms);
    cudaGetDevice(&v->device);
    v->pairs = v->mode == LDPC_I8 && !(d->flags & LDPC_SERVE_UNPAIRED);
    v->policy.pairs = v->pairs;
    v->policy.always = v->pairs && (d->flags & LDPC_SERVE_PAIRED);
    const int esz = v->mode == LDPC_F32 ? 4 : (v->mode == LDPC_I8 ? 1 : 2);
    // ---- per-shape tables and layouts, sized for the largest block of the shape: the single
    // form (four-edge chunks, check messages in shared memory) and, for INT8, the paired form
    // (two-edge chunks, half2 posteriors, two bitmaps, three message words per check in a
    // device-memory slot per group)
    std::vector<uint32_t> tabs;
    int tw = 0;
    int64_t rec_group = 0;
    const int n_sh = session_shape_count(s);
    for (int i = 0; i < n_sh; ++i) {
      ServeShape ss{};
      ShapeDev sd{};
      std::vector<uint32_t> tmp;
      session_shape_table(s, i, 0, tmp, sd, kServeChunk);  // geometry only
      const int Z = sd.Z;
      ss.dummy_base = sd.nb * Z;
      session_shape_table(s, i, ss.dummy_base, tabs, sd, kServeChunk);
      ss.sh = sd;
      tw = std::max(tw, sd.tab_words);
      ss.rec_cap = sd.mb * Z;
      ss.hb_bytes = (Z % 32 == 0) ? align16s(sd.nb * (Z / 32) * 4) : 0;
      ss.L_bytes = align16s((sd.nb + 1) * Z * (v->mode == LDPC_I8 ? 4 : esz));  // INT8: float posteriors
      // FP32: the single form's messages in a device-memory slot per (loop block, group)
      const int64_t rec_single = 2 * align16s(ss.rec_cap * esz) + align16s(ss.rec_cap * 4);
      ss.region_bytes = ss.L_bytes + ss.hb_bytes + (v->mode == LDPC_F32 ? 0 : static_cast<int>(rec_single));
      if (v->mode == LDPC_F32) rec_group = std::max<int64_t>(rec_group, rec_single);
      ss.G = std::max(1, kServeBlock / Z);
      if (Z > 32) ss.G = std::min(ss.G, 15);
      if (v->pairs && Z % 32 == 0) {
        ShapeDev sp{};
        session_shape_table(s, i, ss.dummy_base, tabs, sp, kChunk);
        ss.shp = sp;
        tw = std::max(tw, sp.tab_words);
        ss.Lp_bytes = align16s((sd.nb + 1) * Z * 4);
        ss.region_p = ss.Lp_bytes + 2 * ss.hb_bytes;
        ss.Gp = ss.G;
        rec_group = std::max<int64_t>(rec_group, 3 * align16s(ss.rec_cap * 4));
      }
      v->hshapes.push_back(ss);
    }
    const int hdr = align16s(tw * 4) + 16;
    int smem = hdr;
    for (auto& ss : v->hshapes) {
      while (ss.G > 1 && hdr + ss.G * ss.region_bytes > kMaxSmem) --ss.G;
      if (ss.sh.Z == 16 && ss.G > 1 && (ss.G & 1)) --ss.G;
      ss.feasible = hdr + ss.G * ss.region_bytes <= kMaxSmem;
      if (ss.feasible) smem = std::max(smem, hdr + ss.G * ss.region_bytes);
      if (ss.Gp > 0) {
        while (ss.Gp > 1 && hdr + ss.Gp * ss.region_p > kMaxSmem) --ss.Gp;
        ss.feasible_p = hdr + ss.Gp * ss.region_p <= kMaxSmem;
        if (ss.feasible_p) smem = std::max(smem, hdr + ss.Gp * ss.region_p);
      }
    }
    v->smem = smem;
    const void* fn = serve_kernel_ptr(v->mode, v->cb_crc, v->pairs);
    cudaFuncAttributes fa{};
    cudaError_t e = cudaFuncGetAttributes(&fa, fn);
    if (e == cudaSuccess && smem + static_cast<int>(fa.sharedSizeBytes) > kMaxSmem) e = cudaErrorInvalidValue;
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    int per_sm = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kServeBlock, smem);
    if (e != cudaSuccess || per_sm < 1) {
      free_server(v);
      return srv_fail(LDPC_ECUDA, std::string("serve loop does not fit an SM (") + std::to_string(smem) +
                                      " B shared, " + std::to_string(fa.numRegs) + " registers): " +
                                      cudaGetErrorString(e));
    }
    v->grid = per_sm * sms;
    // by default pairing starts above two items in flight per loop and stops at one
    v->policy.threshold = d->pair_threshold > 0 ? d->pair_threshold : 2 * static_cast<int64_t>(v->grid);
    v->policy.release = std::min<int64_t>(d->pair_release > 0 ? d->pair_release : v->grid, v->policy.threshold);
    int gmax = 0;  // message slots per loop: the paired form's groups, or FP32's single-form groups
    for (auto& ss : v->hshapes) {
      if (ss.feasible_p) gmax = std::max(gmax, ss.Gp);
      if (v->mode == LDPC_F32 && ss.feasible) gmax = std::max(gmax, ss.G);
    }
    if (gmax > 0) {
      e = cudaMalloc(&v->rscratch, static_cast<size_t>(v->grid) * gmax * rec_group);
      if (e != cudaSuccess) {
        free_server(v);
        return srv_fail(LDPC_ENOMEM, std::string("serve message slots: ") + cudaGetErrorString(e));
      }
    }
    // ---- rings and arena
    v->max_inflight = d->max_inflight;
    v->item_cap = static_cast<uint32_t>(d->max_inflight) * kMaxTbCb;
    v->cb_cap = static_cast<uint32_t>(d->max_inflight) * kMaxTbCb;
    v->done_cap = static_cast<uint32_t>(d->max_inflight);
    int rc;
    const int64_t arena_words = static_cast<int64_t>(d->arena_bytes / 4);
    if ((rc = host_alloc(&v->hctl, 1)) || (rc = host_alloc(&v->lctl, 1)) || (rc = host_alloc(&v->items, v->item_cap)) ||
        (rc = host_alloc(&v->cbs, v->cb_cap)) || (rc = host_alloc(&v->reqs, d->max_inflight)) ||
        (rc = host_alloc(&v->done, v->done_cap))) {
      free_server(v);
      return rc;
    }
    std::vector<uint32_t> xp(kServeXpowWords + 1);
    {
      uint32_t cur = 1;
      for (size_t m = 0; m < xp.size(); ++m) {
        xp[m] = cur;
        for (int i = 0; i < 32; ++i) {
          cur <<= 1;
          if (cur & 0x1000000u) cur ^= 0x1864CFBu;
        }
      }
    }
    auto up = [&](auto** p, const auto& vec) -> int {
      using T = std::remove_reference_t<decltype(vec[0])>;
      cudaError_t ee = cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(vec.size(), 1) * sizeof(T));
      if (ee == cudaSuccess && !vec.empty())
        ee = cudaMemcpy(*p, vec.data(), vec.size() * sizeof(T), cudaMemcpyHostToDevice);
      return ee == cudaSuccess ? LDPC_OK : srv_fail(LDPC_ENOMEM, std::string("serve: ") + cudaGetErrorString(ee));
    };
    std::vector<uint32_t> zeros4(4, 0u), zcount(d->max_inflight, 0u);
    const int book_wpm = d->codebook_n > 0 ? (d->codebook_prb + 31) / 32 : 0;
    std::vector<uint32_t> book;
    if (d->codebook_n > 0) book.assign(d->codebook, d->codebook + static_cast<size_t>(d->codebook_n) * 7 * book_wpm);
    v->book_n = d->codebook_n;
    v->book_prb = d->codebook_prb;
    if ((rc = up(&v->shapes, v->hshapes)) || (rc = up(&v->tabs, tabs)) || (rc = up(&v->xpow32, xp)) ||
        (rc = up(&v->dctl, zeros4)) || (rc = up(&v->counts, zcount)) || (rc = up(&v->book, book))) {
      free_server(v);
      return rc;
    }
    e = cudaMalloc(&v->arena, static_cast<size_t>(arena_words) * 4);
    if (e != cudaSuccess) {
      free_server(v);
      return srv_fail(LDPC_ENOMEM, std::string("serve arena: ") + cudaGetErrorString(e));
    }
    v->alloc = new Arena(arena_words, 2 * static_cast<size_t>(d->max_inflight) + 8);
    for (int i = d->max_inflight - 1; i >= 0; --i) v->free_slots.push_back(i);
    v->slot_info.resize(d->max_inflight);
    v->host_pool = static_cast<const uint8_t*>(d->host_pool);
    v->host_pool_bytes = d->host_pool_bytes;
    v->result_pool = static_cast<uint8_t*>(d->result_pool);
    v->result_pool_bytes = d->result_pool_bytes;
    const uint8_t* pool_dev = dev_ptr(const_cast<uint8_t*>(v->host_pool));
    uint8_t* res_dev = v->result_pool ? dev_ptr(v->result_pool) : nullptr;
    if (!pool_dev || (v->result_pool && !res_dev)) {
      free_server(v);
      return srv_fail(LDPC_EINVAL, "host_pool / result_pool must be pinned, mapped host memory");
    }
    e = cudaStreamCreateWithFlags(&v->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&v->done_ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      free_server(v);
      return srv_fail(LDPC_ECUDA, std::string("serve stream: ") + cudaGetErrorString(e));
    }
    ServeArgs& a = v->args;
    a.shapes = v->shapes;
    a.tabs = v->tabs;
    a.items = dev_ptr(v->items);
    a.item_cap = v->item_cap;
    a.cbs = dev_ptr(v->cbs);
    a.cb_cap = v->cb_cap;
    a.reqs = dev_ptr(v->reqs);
    a.done = dev_ptr(v->done);
    a.done_cap = v->done_cap;
    a.hctl = dev_ptr(v->hctl);
    a.dctl = v->dctl;
    a.lctl = dev_ptr(v->lctl);
    a.counts = v->counts;
    a.arena = v->arena;
    a.host_pool = pool_dev;
    a.result_pool = res_dev;
    a.crc_table = session_crc_table(s);
    a.xpow32 = v->xpow32;
    session_cb_crc_tables(s, &a.crc_table_b, &a.xpow32_b, &a.cbcrc);
    a.book = v->book;
    a.book_wpm = book_wpm;
    a.book_prb = std::max(1, d->codebook_prb);
    a.book_n = d->codebook_n;
    a.hdr_bytes = hdr;
    a.interleave = interleave;
    a.max_iter = max_iter;
    a.early_term = et;
    a.q_scale = q_scale;
    a.llr_sat = llr_sat;
    a.beta = beta;
    a.msg_sat = msg_sat;
    a.post_sat = post_sat;
    a.idle_ns = static_cast<uint64_t>(d->idle_timeout_us) * 1000ull;
    a.rscratch = v->rscratch;
    a.rscratch_group = rec_group;
    a.groups = gmax;
    a.n_shapes = static_cast<int32_t>(v->hshapes.size());
    a.n_req = d->max_inflight;
    a.arena_words = arena_words;
    a.pool_f2 = static_cast<int64_t>(d->host_pool_bytes / 8);
    a.pool_words = static_cast<int64_t>(d->host_pool_bytes / 4);
    if (!a.items || !a.cbs || !a.reqs || !a.done || !a.hctl || !a.lctl) {
      free_server(v);
      return srv_fail(LDPC_ECUDA, "mapped host rings unavailable");
    }
    if ((rc = launch_loop(v))) {
      free_server(v);
      return rc;
    }
    *out = v;
    return LDPC_OK;
  } catch (...) {
    return srv_fail(LDPC_EINVAL, "unexpected host exception");
  }
}

int ldpc_serve_submit(ldpc_server* v, const ldpc_serve_tb* tbs, int32_t n, int32_t* n_admitted) {
  if (!v || (n > 0 && !tbs) || !n_admitted || n < 0) return srv_fail(LDPC_EINVAL, "bad submit arguments");
  *n_admitted = 0;
  // ---- validate every request before admitting any
  for (int i = 0; i < n; ++i) {
    const ldpc_serve_tb& tb = tbs[i];
    // (the message is built only on a refusal: the admission loop allocates nothing)
    const auto at = [i](const char* why) { return "serve request " + std::to_string(i) + ": " + why; };
    const int shape = session_shape_lookup(v->s, tb.bg, tb.Z);
    if (shape < 0) return srv_fail(LDPC_EINVAL, at("unknown (bg, Z)"));
    const ServeShape& ss = v->hshapes[shape];
    if (!ss.feasible && !(v->pairs && ss.feasible_p))
      return srv_fail(LDPC_EINVAL, at("shape does not fit the serving loop's shared memory"));
    const ShapeDev& sd = ss.sh;
    const int t0 = sd.npc * tb.Z;
    if (tb.n_cb < 1 || tb.n_cb > kMaxTbCb || (tb.Qm != 2 && tb.Qm != 4 && tb.Qm != 6 && tb.Qm != 8) || tb.E <= 0 ||
        tb.E % tb.Qm || tb.E > 2 * (sd.nb * tb.Z - t0))  // the circular buffer may wrap once
      return srv_fail(LDPC_EINVAL, at("bad n_cb, Qm or E"));
    const int K = sd.kb * tb.Z;
    const bool seg = tb.n_cb > 1 && tb.payload_bits == tb.n_cb * (K - 24) - 24;
    if (K % 32 || (tb.payload_bits != tb.n_cb * K - 24 && !seg)) return srv_fail(LDPC_EINVAL, at("payload_bits"));
    if (seg && !v->cb_crc)
      return srv_fail(LDPC_EINVAL, at("code-block CRCs need a service started with LDPC_SERVE_CB_CRC"));
    if (static_cast<int64_t>(tb.n_cb) * (K / 32) >= static_cast<int64_t>(kServeXpowWords))
      return srv_fail(LDPC_EINVAL, at("transport block too large"));
    if (tb.rv < 0 || tb.rv > 3) return srv_fail(LDPC_EINVAL, at("rv must be 0..3"));
    if (tb.reserved != 0) return srv_fail(LDPC_EINVAL, at("reserved must be 0"));
    if (rv_k0(sd.nb - sd.npc, tb.rv, tb.Z) < 0)
      return srv_fail(LDPC_EINVAL, at("redundancy versions 1-3 need a buffer of 66 Z or 50 Z positions"));
    const int n_re = tb.E / tb.Qm;
    const int mw = (n_re + 31) / 32;
    if (tb.sym_offset < 0 || tb.sym_offset % 8 ||
        static_cast<uint64_t>(tb.sym_offset) + static_cast<uint64_t>(tb.n_cb) * n_re * 8 > v->host_pool_bytes)
      return srv_fail(LDPC_EINVAL, at("symbols outside the host pool or misaligned"));
    if (tb.pattern < 0) {
      if (tb.pattern != -1 || tb.mask_offset < 0 || tb.mask_offset % 4 ||
          static_cast<uint64_t>(tb.mask_offset) + static_cast<uint64_t>(tb.n_cb) * mw * 4 > v->host_pool_bytes)
        return srv_fail(LDPC_EINVAL, at("masks outside the host pool or misaligned"));
    } else {
      // the TB's resource elements fill its band symbol after symbol within the slot's 14 symbols
      if (tb.pattern >= v->book_n || tb.n_sc < 1 || tb.grid_sc < 0 ||
          static_cast<int64_t>(tb.grid_sc) + tb.n_sc > (int64_t{1} << 30) ||
          static_cast<int64_t>(tb.n_cb) * n_re > 14 * static_cast<int64_t>(tb.n_sc))
        return srv_fail(LDPC_EINVAL, at("pattern not in the codebook, or the TB does not fit its band in one slot"));
    }
    if (tb.result_offset >= 0 &&
        (!v->result_pool || tb.result_offset % 4 ||
         static_cast<uint64_t>(tb.result_offset) + static_cast<uint64_t>(tb.n_cb) * K / 8 > v->result_pool_bytes))
      return srv_fail(LDPC_EINVAL, at("result outside the result pool or misaligned"));
    if (!(tb.inv_sigma2 >= 0.f)) return srv_fail(LDPC_EINVAL, at("inv_sigma2"));
  }
  // ---- admit in order while the request slots, rings and arena have room
  const int64_t t = now_ns();
  int taken = 0;
  for (; taken < n; ++taken) {
    const ldpc_serve_tb& tb = tbs[taken];
    const int shape = session_shape_lookup(v->s, tb.bg, tb.Z);
    const ServeShape& ss = v->hshapes[shape];
    const ShapeDev& sd = ss.sh;
    const int t0 = sd.npc * tb.Z;
    const int K = sd.kb * tb.Z;
    const int n_re = tb.E / tb.Qm;
    const int mw = (n_re + 31) / 32;
    // columns up to the last position sent; a version that wraps the buffer reaches them all
    const int k0 = rv_k0(sd.nb - sd.npc, tb.rv, tb.Z);
    const int cols = decoded_cols(sd.nb, tb.Z, t0, k0, tb.E);
    const int m_eff = std::min(sd.mb, std::max(sd.mc, cols - sd.kb));
    const int n_single = ss.feasible ? (tb.n_cb + ss.G - 1) / ss.G : 0;
    const bool pair = v->policy.choose(static_cast<int64_t>(v->items_inflight), n_single, ss.feasible != 0,
                                       ss.feasible_p != 0);
    const int G = std::max(1, std::min(pair ? 2 * ss.Gp : ss.G, tb.n_cb));  // code blocks per item
    const int n_items = (tb.n_cb + G - 1) / G;
    if (v->free_slots.empty() || v->items_inflight + n_items > v->item_cap || v->cbs_inflight + tb.n_cb > v->cb_cap)
      break;
    const int64_t words = static_cast<int64_t>(tb.n_cb) * (K / 32) + tb.n_cb;
    const int64_t off = v->alloc->alloc(words);
    if (off < 0) break;
    const int slot = v->free_slots.back();
    v->free_slots.pop_back();
    auto& si = v->slot_info[slot];
    si.arena_off = off;
    si.arena_words = words;
    si.n_items = n_items;
    si.n_cb = tb.n_cb;
    si.t_submit = t;
    si.busy = true;
    ServeReq& rq = v->reqs[slot];
    rq.tag = tb.tag;
    rq.n_cb = tb.n_cb;
    rq.words = tb.n_cb * (K / 32);
    rq.shape = shape;
    rq.seg = (tb.n_cb > 1 && tb.payload_bits == tb.n_cb * (K - 24) - 24) ? 1 : 0;
    rq.bits_off = off;
    rq.status_off = off + static_cast<int64_t>(tb.n_cb) * (K / 32);
    rq.result_off = tb.result_offset;
    rq.pattern = tb.pattern;
    rq.grid_sc = tb.grid_sc;
    rq.n_sc = tb.n_sc;
    // each request slot owns kMaxTbCb code-block records: requests complete
    // out of order, so a ring in submission order could hand the records of
    // a request still waiting for its items to a newer one
    const uint32_t cb_first = static_cast<uint32_t>(slot) * kMaxTbCb;
    for (int j = 0; j < tb.n_cb; ++j) {
      CbDev c{};
      c.shape = shape;
      c.Z = tb.Z;
      c.Qm = tb.Qm;
      c.E = tb.E;
      c.t0 = t0;
      c.m_eff = m_eff;
      c.n_eff = sd.kb + m_eff;
      c.n_re = n_re;
      c.kb = sd.kb;
      c.flags = (rq.seg ? LDPC_CB_CRC24B : 0) | LDPC_CB_RV(tb.rv);
      c.k0 = k0;
      c.re_off = tb.sym_offset / 8 + static_cast<int64_t>(j) * n_re;
      c.mask_off = tb.pattern < 0 ? tb.mask_offset / 4 + static_cast<int64_t>(j) * mw : 0;
      c.llr_off = rq.status_off + j;  // status word index in the arena
      c.bits_off = off + static_cast<int64_t>(j) * (K / 32);
      c.inv_sigma2 = tb.inv_sigma2;
      v->cbs[cb_first + j] = c;
    }
    for (int it = 0; it < n_items; ++it) {
      ServeItem& item = v->items[v->tail % v->item_cap];
      item.req = slot;
      item.cb0 = static_cast<int32_t>(cb_first + it * G);
      item.count = std::min(G, tb.n_cb - it * G);
      item.n_items = n_items;
      item.pair = pair ? 1 : 0;
      ++v->tail;
    }
    v->items_inflight += n_items;
    v->cbs_inflight += tb.n_cb;
    ++v->stats[0];
    v->stats[pair ? 2 : 1] += n_items;
  }
  if (taken > 0) {
    std::atomic_thread_fence(std::memory_order_release);
    reinterpret_cast<volatile uint32_t*>(&v->hctl->tail)[0] = v->tail;
    std::atomic_thread_fence(std::memory_order_seq_cst);
    const int rc = ensure_running(v);
    if (rc) return rc;
  }
  *n_admitted = taken;
  return LDPC_OK;
}

int ldpc_serve_poll(ldpc_server* v, ldpc_serve_done* out, int32_t cap, int32_t* n_out) {
  if (!v || !n_out || cap < 0 || (cap > 0 && !out)) return srv_fail(LDPC_EINVAL, "bad poll arguments");
  int n = 0;
  bool bad = false;
  // a completion must name a request slot that is in flight (a corrupt or repeated record does not)
  drain_ring(v->done, v->done_cap, v->rd, cap, [&](volatile ServeDone* rec) {
    const int slot = rec->req;
    if (slot < 0 || slot >= v->max_inflight || !v->slot_info[slot].busy) return false;
    auto& si = v->slot_info[slot];
    ldpc_serve_done o{};
    o.tag = rec->tag;
    o.d = rec->d;
    o.max_iters = rec->max_iters;
    o.all_syndrome_ok = rec->all_ok;
    o.status = 0;
    o.t_submit_ns = si.t_submit;
    o.t_complete_ns = now_ns();
    o.t_device_ns = static_cast<int64_t>(rec->t_dev);
    o.t_admit_ns = si.t_submit;
    out[n++] = o;
    v->alloc->release(si.arena_off, si.arena_words);
    v->items_inflight -= si.n_items;
    v->cbs_inflight -= si.n_cb;
    si.busy = false;
    v->free_slots.push_back(slot);
    return true;
  }, &bad);
  *n_out = n;
  // the good completions before a bad record are handed out first; the bad record stays where it is
  // and the next call, which starts on it, refuses it
  if (bad && n == 0) return srv_fail(LDPC_ECUDA, "serve: a completion record names no request in flight");
  if (v->items_inflight > 0) return ensure_running(v);  // a loop that idled out while items were pending
  return LDPC_OK;
}

int ldpc_serve_replay(ldpc_server* v, const ldpc_serve_tb* tbs, const int64_t* arrival_ns, int32_t n,
                      ldpc_serve_done* out, int32_t timeout_ms) {
  if (!v || n < 0 || (n > 0 && (!tbs || !arrival_ns || !out)) || timeout_ms < 1)
    return srv_fail(LDPC_EINVAL, "bad replay arguments");
  // The schedule, the tag index, the requests and the completions are set up
  // in memory of this call's own before the loop, which then allocates nothing
  // and touches none of the caller's arrays (a page fault in the loop stalls
  // every request due meanwhile).
  std::vector<int64_t> sched;
  std::unordered_map<uint64_t, int> by_tag;
  std::vector<ldpc_serve_done> buf, done;
  std::vector<ldpc_serve_tb> req;
  try {
    sched.resize(static_cast<size_t>(n));
    by_tag.reserve(static_cast<size_t>(n));
    for (int i = 0; i < n; ++i) by_tag.emplace(tbs[i].tag, i);
    buf.resize(1024);
    req.assign(tbs, tbs + n);
    done.resize(static_cast<size_t>(n));
  } catch (const std::bad_alloc&) {
    return srv_fail(LDPC_ENOMEM, "replay: host memory for the schedule");
  }
  if (static_cast<int>(by_tag.size()) != n) return srv_fail(LDPC_EINVAL, "replay: tags must be unique");
  const int64_t t0 = now_ns();
  for (int i = 0; i < n; ++i) sched[i] = t0 + arrival_ns[i];
  int next = 0, got = 0;
  int64_t last_progress = t0;
  // (declared before the counters' guard, so the copy comes after they are read)
  struct CopyOut {  // the completions collected (zeros after them) reach the caller on every return
    const std::vector<ldpc_serve_done>& done;
    ldpc_serve_done* out;
    ~CopyOut() {
      if (!done.empty()) std::memcpy(out, done.data(), done.size() * sizeof(ldpc_serve_done));
    }
  } copy_out{done, out};
  for (int i = 4; i < kServeStats; ++i) v->stats[i] = 0;
  rusage ru0{};
  const bool have_ru = getrusage(RUSAGE_THREAD, &ru0) == 0;
  struct RuDelta {  // the thread's scheduling and paging counts since the replay began, on every return
    ldpc_server* v;
    const rusage& r0;
    bool ok;
    ~RuDelta() {
      rusage r1{};
      if (!ok || getrusage(RUSAGE_THREAD, &r1) != 0) return;
      v->stats[7] = r1.ru_nivcsw - r0.ru_nivcsw;
      v->stats[8] = r1.ru_nvcsw - r0.ru_nvcsw;
      v->stats[9] = r1.ru_minflt - r0.ru_minflt;
      v->stats[10] = r1.ru_majflt - r0.ru_majflt;
    }
  } ru_delta{v, ru0, have_ru};
  int64_t prev = t0;
  while (got < n) {
    const int64_t now = now_ns();
    if (now - prev > v->stats[4]) {
      v->stats[4] = now - prev;
      v->stats[6] = prev - t0;
    }
    if (now - prev > 1000000) ++v->stats[5];
    prev = now;
    int due = next;
    while (due < n && sched[due] <= now) ++due;
    // admission stops at the first request that does not fit: offer a bounded chunk at a time, so
    // a backlog (a saturated service) costs no more host time per pass than a short queue
    while (due > next) {
      const int32_t chunk = std::min(due - next, 64);
      int32_t adm = 0;
      const int rc = ldpc_serve_submit(v, req.data() + next, chunk, &adm);
      if (rc) return rc;
      next += adm;
      if (adm < chunk) break;
    }
    int32_t k = 0;
    const int rc = ldpc_serve_poll(v, buf.data(), static_cast<int32_t>(buf.size()), &k);
    for (int i = 0; i < k; ++i) {  // completions taken are kept even when the poll reports an error
      ldpc_serve_done o = buf[i];
      auto f = by_tag.find(o.tag);
      if (f != by_tag.end()) o.t_submit_ns = sched[f->second];
      done[got++] = o;
    }
    if (rc) return rc;
    if (k > 0 || due > next) last_progress = now_ns();
    if (now_ns() - last_progress > static_cast<int64_t>(timeout_ms) * 1000000ll)
      return srv_fail(LDPC_ETIMEOUT, "replay: no completion within the timeout");
  }
  return LDPC_OK;
}

int ldpc_serve_stats(ldpc_server* v, int64_t* out, int32_t n) {
  if (!v || n < 0 || (n > 0 && !out)) return srv_fail(LDPC_EINVAL, "bad stats arguments");
  for (int i = 0; i < n; ++i) out[i] = i < kServeStats ? v->stats[i] : 0;
  return LDPC_OK;
}

int ldpc_serve_stop(ldpc_server* v) {
  if (!v) return LDPC_OK;
  reinterpret_cast<volatile uint32_t*>(&v->hctl->stop)[0] = 1u;
  std::atomic_thread_fence(std::memory_order_seq_cst);
  int rc = LDPC_OK;
  if (v->running) {
    const cudaError_t e = cudaStreamSynchronize(v->stream);  // the loop sees the stop flag within ~1 us
    if (e != cudaSuccess) rc = srv_fail(LDPC_ECUDA, std::string("serve stop: ") + cudaGetErrorString(e));
  }
  free_server(v);
  return rc;
}

}  // extern "C"
