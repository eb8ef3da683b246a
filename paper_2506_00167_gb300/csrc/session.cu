// Host side of the C-ABI: sessions, batch planning and the entry points.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "host_rules.h"
#include "internal.cuh"

struct ldpc_session {
  int device = 0;
  cudaStream_t stream = nullptr;
  int mode = LDPC_F32;
  int max_iter = 10;
  int early_term = 1;
  float beta_f32 = 0.5f;
  int offset_lsb = 1;
  float q_scale = 4.0f;
  int llr_sat = 63, msg_sat = 63, post_sat = 127;
  int interleave = 1;
  uint64_t budget = 0;
  uint64_t allocated = 0;
  int num_sms = 0;
  struct Bg {
    int mb, nb, kb, mc, npc;
    std::vector<int> row, col, V;
    std::vector<int> maxcol_upto;  // largest column used by rows 0..r
  };
  std::vector<Bg> bgs;
  std::vector<int> zset;
  std::vector<ldpcgb::ShapeDev> shapes;
  std::map<std::pair<int, int>, int> shape_index;  // (bg, Z) -> shape
  std::map<std::pair<int, int>, int> tiles;        // (bg, Z) -> code blocks per work item
  int strategy = LDPC_PLAN_MIXED;
  uint32_t* d_crc_table = nullptr;
  uint32_t* d_crc_table_b = nullptr;  // byte table of the code-block generator g_B
  uint32_t* d_xpow32_b = nullptr;     // x^(32 m) mod g_B, m = 0..largest block's words
  uint32_t* d_cbcrc = nullptr;        // per shape: the code-block CRC byte table (K * 32 words)
  uint32_t* d_err = nullptr;
};

namespace {

struct Launch {
  int G = 1, block = 0, smem = 0, grid = 0;  // G: most groups any item of the launch uses
  bool rglobal = false;
  int kind = ldpcgb::kKindShared;
  int item_begin = 0, item_count = 0;
  int hdr_bytes = 0;
  int64_t rscratch_group = 0;
  int64_t rscratch_off = 0;  // into the batch's scratch buffer
};

}  // namespace

struct ldpc_graph {
  cudaGraphExec_t exec = nullptr;
};

struct ldpc_batch {
  ldpc_session* s = nullptr;
  ldpc_batch_info info{};
  std::vector<ldpcgb::CbDev> cbs;
  ldpcgb::CbDev* d_cbs = nullptr;
  std::vector<Launch> launches;
  ldpcgb::DecodeItem* d_items = nullptr;
  ldpcgb::ShapeDev* d_shapes = nullptr;  // per (launch, shape) edge tables
  uint32_t* d_tabs = nullptr;
  int32_t* d_item_cbs = nullptr;
  uint8_t* d_rscratch = nullptr;
  int64_t rscratch_bytes = 0;
  uint32_t* d_queues = nullptr;  // one work-queue counter per decoder launch
  ldpcgb::DemapTile* d_tiles = nullptr;
  int n_tiles = 0;
  ldpcgb::DemapTile* d_rep_tiles = nullptr;  // repeated bits of blocks whose rate matching wraps
  int n_rep_tiles = 0;
  ldpcgb::TbDev* d_tbs = nullptr;
  int32_t* d_slot_start = nullptr;
  int32_t* d_slot_tbs = nullptr;
  int32_t* d_slot_N = nullptr;
  uint32_t* d_xpow32 = nullptr;
  std::vector<void*> owned;
  uint64_t bytes = 0;
  // the cluster decoder's plan per cluster size (2 and 4 CTAs), built at its first call
  struct ClusterLaunch {
    int n = 0, list_off = 0, block = 0, smem = 0;
    int tab_bytes = 0, L_bytes = 0, hb_bytes = 0, rec_cap = 0;
  };
  struct ClusterPlan {
    bool built = false;
    uint32_t* d_tabs = nullptr;
    ldpcgb::ShapeDev* d_shapes = nullptr;
    int32_t* d_list = nullptr;
    std::vector<ClusterLaunch> launches;
  };
  ClusterPlan cplan[2];
};

namespace ldpcgb {

static thread_local std::string g_err;

void set_error(const std::string& msg) { g_err = msg; }

}  // namespace ldpcgb

using namespace ldpcgb;

namespace {

int fail(int code, const std::string& msg) {
  set_error(msg);
  return code;
}

int cuda_fail(cudaError_t e, const char* where) {
  return fail(LDPC_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// Device allocation charged against the session budget.
template <typename T>
int dev_alloc(ldpc_session* s, T** p, size_t count, std::vector<void*>* owned, uint64_t* charged) {
  size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
  bytes = (bytes + 255) & ~size_t(255);
  if (s->budget && s->allocated + bytes > s->budget)
    return fail(LDPC_ENOMEM, "device-memory budget exceeded (" + std::to_string(s->allocated + bytes) + " > " +
                                 std::to_string(s->budget) + " bytes)");
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), bytes);
  if (e != cudaSuccess) return fail(LDPC_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  s->allocated += bytes;
  if (owned) owned->push_back(*p);
  if (charged) *charged += bytes;
  return LDPC_OK;
}

template <typename T>
int upload(ldpc_session* s, T** p, const std::vector<T>& v, std::vector<void*>* owned, uint64_t* charged) {
  int rc = dev_alloc(s, p, v.size(), owned, charged);
  if (rc) return rc;
  if (!v.empty()) {
    cudaError_t e = cudaMemcpy(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy");
  }
  return LDPC_OK;
}

int align16(int x) { return (x + 15) & ~15; }

bool z_supported(int Z) { return Z == 16 || (Z >= 32 && Z <= kMaxZ && Z % 32 == 0); }

constexpr uint32_t kGenA = 0x1864CFBu;  // g(x) of the transport-block CRC, x^24 term included
constexpr uint32_t kGenB = 0x1800063u;  // g_B(x) of the code-block CRC

uint32_t crc_byte_entry(uint32_t v, uint32_t gen) {
  uint32_t r = v << 16;
  for (int i = 0; i < 8; ++i) {
    r <<= 1;
    if (r & 0x1000000u) r ^= gen;
  }
  return r;
}

std::vector<uint32_t> crc_byte_table(uint32_t gen) {
  std::vector<uint32_t> t(256);
  for (uint32_t v = 0; v < 256; ++v) t[v] = crc_byte_entry(v, gen);
  return t;
}

// x^(32 m) mod g for m = 0..n.
std::vector<uint32_t> xpow32_table(int n, uint32_t gen = kGenA) {
  std::vector<uint32_t> t(n + 1);
  uint32_t cur = 1;  // x^0
  for (int m = 0; m <= n; ++m) {
    t[m] = cur;
    for (int i = 0; i < 32; ++i) {  // multiply by x^32, one bit at a time
      cur <<= 1;
      if (cur & 0x1000000u) cur ^= gen;
    }
  }
  return t;
}

// Code-block CRC table of a K-bit block (first bit in time = highest
// degree): bit p stands for x^(K-1-p), and byte j (bits 8j .. 8j+7, bit 8j+i
// as bit i) with value v contributes XOR_{i: v_i = 1} x^(K-1-8j-i) mod g_B.
// Appends those 256 values for every byte j: K * 32 words.
void cb_crc_byte_table(int K, std::vector<uint32_t>& out) {
  std::vector<uint32_t> single(K);
  uint32_t cur = 1;  // x^0, for bit K-1
  for (int p = K - 1; p >= 0; --p) {
    single[p] = cur;
    cur <<= 1;
    if (cur & 0x1000000u) cur ^= kGenB;
  }
  const size_t base = out.size();
  out.resize(base + static_cast<size_t>(K) * 32);
  for (int j = 0; j < K / 8; ++j) {
    uint32_t* t = out.data() + base + static_cast<size_t>(j) * 256;
    t[0] = 0;
    for (int v = 1; v < 256; ++v) {
      const int i = __builtin_ctz(static_cast<unsigned>(v));
      t[v] = t[v & (v - 1)] ^ single[8 * j + i];
    }
  }
}

// Edge table of base graph g at lifting Z for a launch whose dummy slot is at
// element `dummy`: per row, chunks of `chunk` edges (the bases, then the
// shifts), the last chunk padded with (dummy, 0); then one word per row:
// start | deg << 16.
void build_table(const ldpc_session::Bg& g, int Z, int dummy, std::vector<uint32_t>& tabs, ShapeDev& sh,
                 int chunk = kChunk) {
  sh.tab_off = static_cast<int32_t>(tabs.size());
  std::vector<uint32_t> row_info;
  const int ne = static_cast<int>(g.row.size());
  int e = 0;
  for (int r = 0; r < g.mb; ++r) {
    std::vector<int> cols, sh_;
    for (; e < ne && g.row[e] == r; ++e) {
      cols.push_back(g.col[e] * Z);
      sh_.push_back(g.V[e] % Z);
    }
    const int deg = static_cast<int>(cols.size());
    const int start = static_cast<int>(tabs.size()) - sh.tab_off;
    for (int c = 0; c < (deg + chunk - 1) / chunk; ++c) {
      for (int i = 0; i < chunk; ++i) {
        const int j = chunk * c + i;
        tabs.push_back(static_cast<uint32_t>(j < deg ? cols[j] : dummy));
      }
      for (int i = 0; i < chunk; ++i) {
        const int j = chunk * c + i;
        tabs.push_back(static_cast<uint32_t>(j < deg ? sh_[j] : 0));
      }
    }
    row_info.push_back(static_cast<uint32_t>(start) | (static_cast<uint32_t>(deg) << 16));
  }
  sh.row_off = static_cast<int32_t>(tabs.size()) - sh.tab_off;
  for (uint32_t ri : row_info) tabs.push_back(ri);
  while ((tabs.size() - sh.tab_off) % 4) tabs.push_back(0u);
  sh.tab_words = static_cast<int32_t>(tabs.size()) - sh.tab_off;
}

int default_tile(int Z) {
  int G = std::max(1, 256 / Z);
  if (Z > 32) G = std::min(G, 15);  // named barriers 1..15, one per group
  return G;
}

// Plan the decoder launches of a batch: code blocks of one (base graph, Z)
// shape are chunked into work items of G blocks (the shape's tile, default or
// autotuned); each shape gets one shared-memory layout sized for its largest
// block; items go to one launch (LDPC_PLAN_MIXED: every shape whose state fits
// shared memory, plus a second launch whose check messages live in global
// memory) or one launch per lifting size (LDPC_PLAN_PER_Z); within a launch
// items are ordered largest first and handed out by a work queue.
int plan_decode(ldpc_session* s, ldpc_batch* b) {
  const int n_cb = static_cast<int>(b->cbs.size());
  const int esz = s->mode == LDPC_F32 ? 4 : (s->mode == LDPC_I8 ? 1 : 2);
  struct SP {
    int shape = 0, Z = 0, G = 1, max_n = 0, max_m = 0;
    int L_bytes = 0, hb_bytes = 0, rec_bytes = 0, tab_words = 0;
    bool rglobal = false;
    int kind = kKindShared;
    int pair_region = 0, pair_L = 0;  // paired INT8 layout
    std::vector<int> cbs;
  };
  std::map<int, SP> sps;
  for (int i = 0; i < n_cb; ++i) sps[b->cbs[i].shape].cbs.push_back(i);
  for (auto& kv : sps) {
    SP& p = kv.second;
    p.shape = kv.first;
    const ShapeDev& sd = s->shapes[p.shape];
    p.Z = sd.Z;
    // larger blocks first; among equal sizes, by noise level, so the blocks
    // that share a work item (and, paired, a thread group) need similar
    // iteration counts and finish together
    std::stable_sort(p.cbs.begin(), p.cbs.end(), [&](int x, int y) {
      if (b->cbs[x].m_eff != b->cbs[y].m_eff) return b->cbs[x].m_eff > b->cbs[y].m_eff;
      return b->cbs[x].inv_sigma2 < b->cbs[y].inv_sigma2;
    });
    for (int i : p.cbs) {
      p.max_n = std::max(p.max_n, b->cbs[i].n_eff);
      p.max_m = std::max(p.max_m, b->cbs[i].m_eff);
    }
    p.L_bytes = align16((p.max_n + 1) * p.Z * esz);
    p.hb_bytes = (p.Z % 32 == 0) ? align16(p.max_n * (p.Z / 32) * 4) : 0;
    const int rec_cap = p.max_m * p.Z;
    p.rec_bytes = 2 * align16(rec_cap * esz) + align16(rec_cap * 4);
    std::vector<uint32_t> tmp;
    ShapeDev d = sd;
    build_table(s->bgs[sd.bg], p.Z, p.max_n * p.Z, tmp, d);
    p.tab_words = d.tab_words;
    auto t = s->tiles.find({sd.bg, p.Z});
    p.G = t != s->tiles.end() ? t->second : default_tile(p.Z);
    if (p.Z > 32) p.G = std::min(p.G, 15);
    if (p.G * p.Z > kDecodeMaxBlock) p.G = std::max(1, kDecodeMaxBlock / p.Z);
  }
  // launch groups.  Per shape, both record placements are sized: messages in
  // shared memory (G lowered until the region fits) or in a global slot per
  // resident group; the global form is preferred when it lets more code
  // blocks be resident per SM (shared memory limits the first form, registers
  // the second).  Shapes that share a launch share the placement: global if
  // any of them prefers it, so a mixed batch stays one persistent launch.
  const bool pair_ok = s->mode == LDPC_I8 && s->post_sat >= 2 * s->msg_sat;
  struct Opt {
    bool pair = false, pref_global = false;
    int Gs = 0, Gg = 0, reg = 0, recs = 0;
  };
  std::map<int, Opt> opts;
  std::map<std::pair<int, bool>, bool> key_global;  // (launch key, pair family) -> global placement
  for (auto& kv : sps) {
    SP& p = kv.second;
    Opt o;
    const int hdr = align16(p.tab_words * 4) + 16;
    o.pair = pair_ok && p.Z % 32 == 0;
    if (o.pair) {
      // two code blocks per group: posteriors as half2 pairs, two bitmaps, 3 message words per check
      // (in shared memory the message area first holds both blocks' int8 LLRs)
      p.pair_L = align16((p.max_n + 1) * p.Z * 4);
      o.recs = std::max(align16(3 * p.max_m * p.Z * 4), 2 * align16(p.max_n * p.Z));
      o.reg = p.pair_L + 2 * p.hb_bytes;
      p.rec_bytes = 3 * align16(p.max_m * p.Z * 4);
    } else {
      o.recs = p.rec_bytes;
      o.reg = p.L_bytes + p.hb_bytes;
    }
    auto even16 = [&](int G) { return (p.Z == 16 && G > 1 && (G & 1)) ? G - 1 : G; };
    int G = p.G;
    while (G > 1 && G * p.Z > kDecodeMaxBlock) --G;
    G = even16(G);
    int Gs = G;
    while (Gs > 1 && hdr + Gs * (o.reg + o.recs) > kMaxSmem) --Gs;
    Gs = even16(Gs);
    const int kind_s = o.pair ? kKindPairI8 : kKindShared, kind_g = o.pair ? kKindPairI8Global : kKindGlobal;
    int occ_s = 0, occ_g = 0;
    if (hdr + Gs * (o.reg + o.recs) <= kMaxSmem) {
      cudaError_t e = decode_occupancy(s->mode, kind_s, Gs * p.Z, hdr + Gs * (o.reg + o.recs), &occ_s);
      if (e != cudaSuccess) return fail(LDPC_ECUDA, std::string("occupancy: ") + cudaGetErrorString(e));
    }
    if (hdr + G * o.reg <= kMaxSmem) {
      cudaError_t e = decode_occupancy(s->mode, kind_g, G * p.Z, hdr + G * o.reg, &occ_g);
      if (e != cudaSuccess) return fail(LDPC_ECUDA, std::string("occupancy: ") + cudaGetErrorString(e));
    }
    if (occ_g == 0)
      return fail(LDPC_EINVAL, "Z=" + std::to_string(p.Z) + ": code block too large for shared memory");
    o.Gs = occ_s > 0 ? Gs : 0;
    o.Gg = G;
    o.pref_global = occ_g * G > occ_s * Gs;
    const int key = s->strategy == LDPC_PLAN_PER_Z ? p.Z : 0;
    key_global[{key, o.pair}] = key_global[{key, o.pair}] || o.pref_global;
    opts[kv.first] = o;
  }
  std::map<std::pair<int, int>, std::vector<int>> groups;  // (key, kind) -> shapes
  for (auto& kv : sps) {
    SP& p = kv.second;
    const Opt& o = opts[kv.first];
    const int key = s->strategy == LDPC_PLAN_PER_Z ? p.Z : 0;
    const bool glob = key_global[{key, o.pair}];
    p.G = glob ? o.Gg : o.Gs;
    p.rglobal = glob;
    p.kind = o.pair ? (glob ? kKindPairI8Global : kKindPairI8) : (glob ? kKindGlobal : kKindShared);
    if (o.pair) p.pair_region = glob ? o.reg : o.reg + o.recs;
    groups[{key, p.kind}].push_back(kv.first);
  }
  std::vector<DecodeItem> items;
  std::vector<int32_t> item_cbs;
  std::vector<ShapeDev> lshapes;
  std::vector<uint32_t> tabs;
  int64_t scratch_total = 0;
  for (auto& gkv : groups) {
    const int kind = gkv.first.second;
    const bool rglobal = kind_is_global(kind);
    const bool pair = kind_is_pair(kind);
    Launch L;
    L.rglobal = rglobal;
    L.kind = kind;
    int tw = 0;
    for (int sh : gkv.second) tw = std::max(tw, sps[sh].tab_words);
    L.hdr_bytes = align16(tw * 4) + 16;
    struct Cost {
      double cost;
      DecodeItem it;
      std::vector<int32_t> cbs;
    };
    std::vector<Cost> list;
    int smem = 0, block = 0, gmax = 1;
    int64_t rec_max = 0;
    for (int sh : gkv.second) {
      SP& p = sps[sh];
      const int region = pair ? p.pair_region : p.L_bytes + p.hb_bytes + (rglobal ? 0 : p.rec_bytes);
      while (p.G > 1 && L.hdr_bytes + p.G * region > kMaxSmem) --p.G;
      if (L.hdr_bytes + p.G * region > kMaxSmem)
        return fail(LDPC_EINVAL, "Z=" + std::to_string(p.Z) + ": code block too large for shared memory");
      ShapeDev d = s->shapes[sh];
      build_table(s->bgs[d.bg], p.Z, p.max_n * p.Z, tabs, d);
      const int local = static_cast<int>(lshapes.size());
      lshapes.push_back(d);
      smem = std::max(smem, L.hdr_bytes + p.G * region);
      block = std::max(block, p.G * p.Z);
      gmax = std::max(gmax, p.G);
      rec_max = std::max<int64_t>(rec_max, p.rec_bytes);
      const auto& g = s->bgs[d.bg];
      for (size_t q = 0; q < p.cbs.size();) {
        Cost c;
        c.it = DecodeItem{};
        c.it.shape = local;
        c.it.Z = p.Z;
        c.it.region_bytes = region;
        c.it.L_bytes = pair ? p.pair_L : p.L_bytes;
        c.it.hb_bytes = p.hb_bytes;
        c.it.rec_cap = p.max_m * p.Z;
        c.it.dummy_base = p.max_n * p.Z;
        const int m0 = b->cbs[p.cbs[q]].m_eff;
        int cnt = 0;
        const int per_item = pair ? 2 * p.G : p.G;
        while (q < p.cbs.size() && cnt < per_item) {
          c.cbs.push_back(p.cbs[q]);
          ++q;
          ++cnt;
        }
        c.it.count = cnt;
        const int edges = static_cast<int>(std::count_if(g.row.begin(), g.row.end(), [&](int r) { return r < m0; }));
        c.cost = static_cast<double>(edges) * p.Z;  // groups run side by side: the largest block sets the time
        list.push_back(std::move(c));
      }
    }
    std::stable_sort(list.begin(), list.end(), [](const Cost& x, const Cost& y) { return x.cost > y.cost; });
    L.item_begin = static_cast<int>(items.size());
    for (auto& c : list) {
      c.it.first = static_cast<int32_t>(item_cbs.size());
      for (int i : c.cbs) item_cbs.push_back(i);
      items.push_back(c.it);
    }
    L.item_count = static_cast<int>(items.size()) - L.item_begin;
    // the variant with the code-block CRC exit only where a block needs it
    for (const auto& c : list)
      for (int i : c.cbs)
        if (b->cbs[i].flags & LDPC_CB_CRC24B) L.kind |= kKindCrc;
    L.G = gmax;
    L.block = (block + 31) & ~31;
    L.smem = smem;
    int per_sm = 0;
    cudaError_t e = decode_occupancy(s->mode, L.kind, L.block, L.smem, &per_sm);
    if (e != cudaSuccess) return fail(LDPC_ECUDA, std::string("occupancy: ") + cudaGetErrorString(e));
    if (per_sm < 1) return fail(LDPC_EINVAL, "decoder launch does not fit an SM");
    L.grid = std::min(L.item_count, per_sm * s->num_sms);
    if (L.rglobal) {
      L.rscratch_group = rec_max;
      L.rscratch_off = scratch_total;
      scratch_total += static_cast<int64_t>(L.grid) * L.G * rec_max;
    }
    b->launches.push_back(L);
  }
  int rc;
  if ((rc = upload(s, &b->d_items, items, &b->owned, &b->bytes)) ||
      (rc = upload(s, &b->d_item_cbs, item_cbs, &b->owned, &b->bytes)) ||
      (rc = upload(s, &b->d_shapes, lshapes, &b->owned, &b->bytes)) ||
      (rc = upload(s, &b->d_tabs, tabs, &b->owned, &b->bytes)) ||
      (rc = upload(s, &b->d_queues, std::vector<uint32_t>(std::max<size_t>(1, b->launches.size()), 0u), &b->owned,
                   &b->bytes)))
    return rc;
  if (scratch_total > 0) {
    if ((rc = dev_alloc(s, &b->d_rscratch, static_cast<size_t>(scratch_total), &b->owned, &b->bytes))) return rc;
    b->rscratch_bytes = scratch_total;
  }
  b->info.n_items = static_cast<int32_t>(items.size());
  return LDPC_OK;
}

int session_free(ldpc_session* s) {
  if (!s) return LDPC_OK;
  cudaSetDevice(s->device);
  cudaFree(s->d_crc_table);
  cudaFree(s->d_crc_table_b);
  cudaFree(s->d_xpow32_b);
  cudaFree(s->d_cbcrc);
  cudaFree(s->d_err);
  delete s;
  return LDPC_OK;
}

}  // namespace

namespace ldpcgb {

int session_serve_info(ldpc_session* s, int* mode, int* interleave, int* max_iter, int* early_term, float* q_scale,
                       float* llr_sat, float* beta, float* msg_sat, float* post_sat, int* num_sms) {
  *mode = s->mode;
  *interleave = s->interleave;
  *max_iter = s->max_iter;
  *early_term = s->early_term;
  *q_scale = s->q_scale;
  if (s->mode == LDPC_F32) {
    *llr_sat = 3.0e38f;
    *beta = s->beta_f32;
    *msg_sat = 3.0e38f;
    *post_sat = 3.0e38f;
  } else {
    *llr_sat = static_cast<float>(s->llr_sat);
    *beta = static_cast<float>(s->offset_lsb);
    *msg_sat = static_cast<float>(s->msg_sat);
    *post_sat = static_cast<float>(s->post_sat);
  }
  *num_sms = s->num_sms;
  return LDPC_OK;
}

int session_shape_count(ldpc_session* s) { return static_cast<int>(s->shapes.size()); }

int session_shape_table(ldpc_session* s, int shape, int dummy, std::vector<uint32_t>& tabs, ShapeDev& sh,
                        int chunk) {
  sh = s->shapes[shape];
  build_table(s->bgs[sh.bg], sh.Z, dummy, tabs, sh, chunk);
  return LDPC_OK;
}

int session_shape_lookup(ldpc_session* s, int bg, int Z) {
  auto it = s->shape_index.find({bg, Z});
  return it == s->shape_index.end() ? -1 : it->second;
}

const uint32_t* session_crc_table(ldpc_session* s) { return s->d_crc_table; }

void session_cb_crc_tables(ldpc_session* s, const uint32_t** table_b, const uint32_t** xpow32_b,
                           const uint32_t** positions) {
  *table_b = s->d_crc_table_b;
  *xpow32_b = s->d_xpow32_b;
  *positions = s->d_cbcrc;
}

}  // namespace ldpcgb

extern "C" {

const char* ldpc_last_error(void) { return g_err.c_str(); }

const char* ldpc_version(void) { return "ldpcgb 0.1 sm_103a"; }

int ldpc_session_create(const ldpc_session_desc* d, ldpc_session** out) {
  try {
    if (!d || !out) return fail(LDPC_EINVAL, "null argument");
    *out = nullptr;
    if (d->mode < LDPC_F32 || d->mode > LDPC_I16) return fail(LDPC_EINVAL, "unknown mode");
    if (d->max_iter < 1 || d->max_iter > 64) return fail(LDPC_EINVAL, "max_iter must be 1..64");
    if (d->n_bg < 1 || !d->bgs) return fail(LDPC_EINVAL, "no base graphs");
    if (d->n_z < 1 || !d->z_set) return fail(LDPC_EINVAL, "empty Z set");
    if (d->mode != LDPC_F32) {
      const int lim = d->mode == LDPC_I8 ? 127 : 32767;
      if (d->post_sat < 1 || d->post_sat > lim || d->msg_sat < 1 || d->msg_sat > d->post_sat ||
          d->llr_sat < 1 || d->llr_sat > d->post_sat || d->offset_lsb < 0 || !(d->q_scale > 0.f))
        return fail(LDPC_EINVAL, "integer-mode saturation/offset/scale out of range");
    } else if (!(d->offset_f32 >= 0.f)) {
      return fail(LDPC_EINVAL, "offset_f32 must be >= 0");
    }
    auto* s = new (std::nothrow) ldpc_session();
    if (!s) return fail(LDPC_ENOMEM, "host allocation");
    cudaGetDevice(&s->device);
    s->stream = static_cast<cudaStream_t>(d->cuda_stream);
    s->mode = d->mode;
    s->max_iter = d->max_iter;
    s->early_term = d->early_term ? 1 : 0;
    s->beta_f32 = d->offset_f32;
    s->offset_lsb = d->offset_lsb;
    s->q_scale = d->q_scale;
    s->llr_sat = d->llr_sat;
    s->msg_sat = d->msg_sat;
    s->post_sat = d->post_sat;
    s->interleave = d->interleave ? 1 : 0;
    s->budget = d->device_mem_budget;
    cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device);

    for (int i = 0; i < d->n_z; ++i) {
      if (!z_supported(d->z_set[i])) {
        session_free(s);
        return fail(LDPC_EINVAL, "Z=" + std::to_string(d->z_set[i]) + " unsupported (16 or a multiple of 32 <= 384)");
      }
      s->zset.push_back(d->z_set[i]);
    }
    for (int b = 0; b < d->n_bg; ++b) {
      const ldpc_base_graph& g = d->bgs[b];
      ldpc_session::Bg h{g.mb, g.nb, g.kb, g.mc, g.n_punct_cols, {}, {}, {}, {}};
      if (g.mb < 1 || g.nb <= g.mb || g.kb != g.nb - g.mb || g.mc < 1 || g.mc > g.mb || g.n_punct_cols < 0 ||
          g.n_punct_cols > g.kb || g.n_edges < 1 || !g.row || !g.col || !g.V) {
        session_free(s);
        return fail(LDPC_EINVAL, "base graph " + std::to_string(b) + ": bad sizes (need kb = nb - mb)");
      }
      std::vector<int> deg(g.mb, 0);
      int prev_r = -1, prev_c = -1;
      for (int e = 0; e < g.n_edges; ++e) {
        const int r = g.row[e], c = g.col[e], v = g.V[e];
        if (r < 0 || r >= g.mb || c < 0 || c >= g.nb || v < 0 || (r < prev_r) || (r == prev_r && c <= prev_c)) {
          session_free(s);
          return fail(LDPC_EINVAL, "base graph " + std::to_string(b) + ": edges must be row-major, unique, in range");
        }
        prev_r = r;
        prev_c = c;
        deg[r]++;
        h.row.push_back(r);
        h.col.push_back(c);
        h.V.push_back(v);
      }
      h.maxcol_upto.assign(g.mb, 0);
      for (int e = 0; e < g.n_edges; ++e) h.maxcol_upto[g.row[e]] = std::max(h.maxcol_upto[g.row[e]], int(g.col[e]));
      for (int r = 1; r < g.mb; ++r) h.maxcol_upto[r] = std::max(h.maxcol_upto[r], h.maxcol_upto[r - 1]);
      for (int r = 0; r < g.mb; ++r)
        if (deg[r] < 2 || deg[r] > kMaxDeg) {
          session_free(s);
          return fail(LDPC_EINVAL, "base graph " + std::to_string(b) + ": row degree must be 2.." +
                                       std::to_string(kMaxDeg));
        }
      if ((g.kb * 16) % 32 && std::find(s->zset.begin(), s->zset.end(), 16) != s->zset.end()) {
        session_free(s);
        return fail(LDPC_EINVAL, "Z=16 needs an even number of information columns");
      }
      s->bgs.push_back(h);
    }

    // ---- (base graph, Z) pairs; their edge tables are built per batch launch,
    // their code-block CRC position tables here
    std::vector<uint32_t> cbcrc;
    int max_cb_words = 0;
    for (int b = 0; b < static_cast<int>(s->bgs.size()); ++b) {
      const auto& g = s->bgs[b];
      for (int Z : s->zset) {
        ShapeDev sh{};
        sh.crc_off = static_cast<int32_t>(cbcrc.size());
        cb_crc_byte_table(g.kb * Z, cbcrc);
        max_cb_words = std::max(max_cb_words, g.kb * Z / 32);
        sh.bg = b;
        sh.Z = Z;
        sh.mb = g.mb;
        sh.nb = g.nb;
        sh.kb = g.kb;
        sh.mc = g.mc;
        sh.npc = g.npc;
        s->shape_index[{b, Z}] = static_cast<int>(s->shapes.size());
        s->shapes.push_back(sh);
      }
    }
    int rc;
    if ((rc = upload(s, &s->d_crc_table, crc_byte_table(kGenA), nullptr, nullptr)) ||
        (rc = upload(s, &s->d_crc_table_b, crc_byte_table(kGenB), nullptr, nullptr)) ||
        (rc = upload(s, &s->d_xpow32_b, xpow32_table(max_cb_words, kGenB), nullptr, nullptr)) ||
        (rc = upload(s, &s->d_cbcrc, cbcrc, nullptr, nullptr)) ||
        (rc = upload(s, &s->d_err, std::vector<uint32_t>(4, 0u), nullptr, nullptr))) {
      session_free(s);
      return rc;
    }
    cudaError_t e = decode_prepare(s->mode);
    if (e != cudaSuccess) {
      session_free(s);
      return cuda_fail(e, "cudaFuncSetAttribute");
    }
    *out = s;
    return LDPC_OK;
  } catch (...) {
    return fail(LDPC_EINVAL, "unexpected host exception");
  }
}

int ldpc_session_destroy(ldpc_session* s) { return session_free(s); }

int ldpc_session_set_stream(ldpc_session* s, void* stream) {
  if (!s) return fail(LDPC_EINVAL, "null session");
  s->stream = static_cast<cudaStream_t>(stream);
  return LDPC_OK;
}

int ldpc_batch_destroy(ldpc_batch* b) {
  if (!b) return LDPC_OK;
  cudaSetDevice(b->s->device);
  for (void* p : b->owned) cudaFree(p);
  b->s->allocated -= std::min(b->s->allocated, b->bytes);
  delete b;
  return LDPC_OK;
}

int ldpc_batch_create(ldpc_session* s, const ldpc_cb_desc* cbs, int32_t n_cb, const ldpc_tb_desc* tbs,
                      int32_t n_tb, int32_t n_slots, const int32_t* slot_N, ldpc_batch** out) {
  try {
    if (!s || !out || (n_cb > 0 && !cbs) || n_cb < 0 || n_tb < 0 || (n_tb > 0 && !tbs) || n_slots < 0 ||
        (n_slots > 0 && !slot_N))
      return fail(LDPC_EINVAL, "bad batch arguments");
    *out = nullptr;
    auto* b = new (std::nothrow) ldpc_batch();
    if (!b) return fail(LDPC_ENOMEM, "host allocation");
    b->s = s;
    auto bail = [&](int code, const std::string& msg) {
      ldpc_batch_destroy(b);
      return fail(code, msg);
    };
    const int esz = s->mode == LDPC_F32 ? 4 : (s->mode == LDPC_I8 ? 1 : 2);
    int64_t sym_end = 0, mask_end = 0, llr_end = 0, bits_end = 0, info_bits = 0;
    b->cbs.resize(n_cb);
    for (int i = 0; i < n_cb; ++i) {
      const ldpc_cb_desc& c = cbs[i];
      const std::string at = "code block " + std::to_string(i) + ": ";
      if (c.bg < 0 || c.bg >= static_cast<int>(s->bgs.size())) return bail(LDPC_EINVAL, at + "bad base graph");
      auto it = s->shape_index.find({c.bg, c.Z});
      if (it == s->shape_index.end()) return bail(LDPC_EINVAL, at + "Z not in the session's Z set");
      if (c.Qm != 2 && c.Qm != 4 && c.Qm != 6 && c.Qm != 8) return bail(LDPC_EINVAL, at + "Qm must be 2/4/6/8");
      const auto& g = s->bgs[c.bg];
      const int t0 = g.npc * c.Z;
      // rate matching reads a circular buffer of the nb*Z - t0 positions from t0; it may wrap once
      if (c.E <= 0 || c.E % c.Qm || c.E > 2 * (g.nb * c.Z - t0))
        return bail(LDPC_EINVAL, at + "E must be a positive multiple of Qm with E <= 2 (nb*Z - t0)");
      if (c.re_offset < 0 || c.mask_word_offset < 0 || c.llr_offset < 0 || c.bits_word_offset < 0 ||
          (c.flags & ~(LDPC_CB_CRC24B | LDPC_CB_RV_MASK)))
        return bail(LDPC_EINVAL, at + "negative offset or unknown flag");
      // start of the redundancy version: NR's table for buffers of 66 Z and 50 Z positions
      const int rv = (c.flags & LDPC_CB_RV_MASK) >> LDPC_CB_RV_SHIFT;
      const int k0 = rv_k0(g.nb - g.npc, rv, c.Z);
      if (k0 < 0) return bail(LDPC_EINVAL, at + "redundancy versions 1-3 need a buffer of 66 Z or 50 Z positions");
      if ((c.llr_offset * esz) % 16) return bail(LDPC_EINVAL, at + "llr_offset must be 16-byte aligned");
      if ((g.kb * c.Z) % 32) return bail(LDPC_EINVAL, at + "kb*Z must be a multiple of 32");
      if (!(c.inv_sigma2 >= 0.f)) return bail(LDPC_EINVAL, at + "inv_sigma2 must be >= 0");
      // columns up to the last position sent; a version that wraps the buffer reaches them all
      const int cols = decoded_cols(g.nb, c.Z, t0, k0, c.E);
      const int m_eff = std::min(g.mb, std::max(g.mc, cols - g.kb));
      if (g.maxcol_upto[m_eff - 1] >= g.kb + m_eff)
        return bail(LDPC_EINVAL, at + "a decoded row uses a column beyond the decoded ones (base graph order)");
      CbDev d{};
      d.shape = it->second;
      d.Z = c.Z;
      d.Qm = c.Qm;
      d.E = c.E;
      d.t0 = t0;
      d.m_eff = m_eff;
      d.n_eff = g.kb + m_eff;
      d.n_re = c.E / c.Qm;
      d.kb = g.kb;
      d.flags = c.flags;
      d.k0 = k0;
      d.re_off = c.re_offset;
      d.mask_off = c.mask_word_offset;
      d.llr_off = c.llr_offset;
      d.bits_off = c.bits_word_offset;
      d.inv_sigma2 = c.inv_sigma2;
      b->cbs[i] = d;
      sym_end = std::max<int64_t>(sym_end, c.re_offset + d.n_re);
      mask_end = std::max<int64_t>(mask_end, c.mask_word_offset + (d.n_re + 31) / 32);
      llr_end = std::max<int64_t>(llr_end, c.llr_offset + static_cast<int64_t>(d.n_eff) * c.Z);
      bits_end = std::max<int64_t>(bits_end, c.bits_word_offset + g.kb * c.Z / 32);
      info_bits += static_cast<int64_t>(g.kb) * c.Z;
    }
    int rc = upload(s, &b->d_cbs, b->cbs, &b->owned, &b->bytes);
    if (rc) return bail(rc, g_err);

    // ---- decoder plan
    rc = plan_decode(s, b);
    if (rc) return bail(rc, g_err);

    // ---- demap tiles
    std::vector<DemapTile> tiles;
    for (int i = 0; i < n_cb; ++i)
      for (int r = 0; r < std::max(1, b->cbs[i].n_re); r += kDemapTile) tiles.push_back({i, r});
    b->n_tiles = static_cast<int>(tiles.size());
    if ((rc = upload(s, &b->d_tiles, tiles, &b->owned, &b->bytes))) return bail(rc, g_err);
    // blocks whose rate matching wraps the circular buffer: their repeated bits, kDemapBlock per tile
    std::vector<DemapTile> rep;
    for (int i = 0; i < n_cb; ++i) {
      const CbDev& c = b->cbs[i];
      const int ncb = c.n_eff * c.Z - c.t0;
      for (int e = ncb; e < c.E; e += kDemapBlock) rep.push_back({i, e});
    }
    b->n_rep_tiles = static_cast<int>(rep.size());
    if (!rep.empty() && (rc = upload(s, &b->d_rep_tiles, rep, &b->owned, &b->bytes))) return bail(rc, g_err);

    // ---- transport blocks and slots
    if (n_tb > 0) {
      std::vector<TbDev> tv(n_tb);
      std::vector<std::vector<int>> per_slot(n_slots);
      int max_words = 0;
      for (int t = 0; t < n_tb; ++t) {
        const ldpc_tb_desc& x = tbs[t];
        const std::string at = "transport block " + std::to_string(t) + ": ";
        if (x.first_cb < 0 || x.n_cb < 1 || x.first_cb + x.n_cb > n_cb || x.slot < 0 || x.slot >= n_slots ||
            x.n_sc < 0)
          return bail(LDPC_EINVAL, at + "bad code-block range, slot or n_sc");
        int64_t bits = 0;
        int n_flag = 0;
        for (int i = x.first_cb; i < x.first_cb + x.n_cb; ++i) {
          bits += static_cast<int64_t>(b->cbs[i].kb) * b->cbs[i].Z;
          n_flag += (b->cbs[i].flags & LDPC_CB_CRC24B) ? 1 : 0;
        }
        const int seg = n_flag > 0 ? 1 : 0;
        if (n_flag != 0 && n_flag != x.n_cb)
          return bail(LDPC_EINVAL, at + "LDPC_CB_CRC24B must be set on all or none of its code blocks");
        bits -= 24 * n_flag;
        if (x.payload_bits != bits - 24)
          return bail(LDPC_EINVAL, at + "payload_bits must be sum(K) - 24 (sum(K - 24) - 24 with code-block CRCs)");
        if (bits > (int64_t(1) << 30)) return bail(LDPC_EINVAL, at + "too many bits");
        TbDev td{};
        td.first_cb = x.first_cb;
        td.n_cb = x.n_cb;
        td.n_sc = x.n_sc;
        td.slot = x.slot;
        td.payload_bits = x.payload_bits;
        td.bytes = static_cast<int32_t>(bits / 8);
        td.seg = seg;
        tv[t] = td;
        max_words = std::max(max_words, static_cast<int>((bits / 8 + 3) / 4));
        per_slot[x.slot].push_back(t);
      }
      std::vector<int32_t> start(n_slots + 1, 0), list;
      for (int sl = 0; sl < n_slots; ++sl) {
        start[sl] = static_cast<int32_t>(list.size());
        for (int t : per_slot[sl]) list.push_back(t);
        if (slot_N[sl] <= 0) return bail(LDPC_EINVAL, "slot_N must be positive");
      }
      start[n_slots] = static_cast<int32_t>(list.size());
      std::vector<int32_t> sn(slot_N, slot_N + n_slots);
      if ((rc = upload(s, &b->d_tbs, tv, &b->owned, &b->bytes)) ||
          (rc = upload(s, &b->d_slot_start, start, &b->owned, &b->bytes)) ||
          (rc = upload(s, &b->d_slot_tbs, list, &b->owned, &b->bytes)) ||
          (rc = upload(s, &b->d_slot_N, sn, &b->owned, &b->bytes)) ||
          (rc = upload(s, &b->d_xpow32, xpow32_table(max_words), &b->owned, &b->bytes)))
        return bail(rc, g_err);
    }

    b->info.sym_elems = sym_end;
    b->info.mask_words = mask_end;
    b->info.llr_elems = llr_end;
    b->info.bits_words = bits_end;
    b->info.n_cb = n_cb;
    b->info.n_tb = n_tb;
    b->info.n_slots = n_tb > 0 ? n_slots : 0;
    b->info.info_bits = info_bits;
    *out = b;
    return LDPC_OK;
  } catch (const std::bad_alloc&) {
    return fail(LDPC_ENOMEM, "host allocation");
  } catch (...) {
    return fail(LDPC_EINVAL, "unexpected host exception");
  }
}

int ldpc_session_set_tiles(ldpc_session* s, const ldpc_tile* tiles, int32_t n) {
  if (!s || n < 0 || (n > 0 && !tiles)) return fail(LDPC_EINVAL, "bad tile arguments");
  for (int i = 0; i < n; ++i) {
    const ldpc_tile& t = tiles[i];
    if (t.bg < 0 || t.bg >= static_cast<int>(s->bgs.size()) || !s->shape_index.count({t.bg, t.Z}) || t.G < 1 ||
        t.G * t.Z > kTileMaxBlock || (t.Z > 32 && t.G > 15))
      return fail(LDPC_EINVAL, "tile " + std::to_string(i) + ": unknown (bg, Z) or G out of range");
  }
  for (int i = 0; i < n; ++i) s->tiles[{tiles[i].bg, tiles[i].Z}] = tiles[i].G;
  return LDPC_OK;
}

int ldpc_session_set_strategy(ldpc_session* s, int32_t strategy) {
  if (!s || (strategy != LDPC_PLAN_MIXED && strategy != LDPC_PLAN_PER_Z)) return fail(LDPC_EINVAL, "bad strategy");
  s->strategy = strategy;
  return LDPC_OK;
}

int ldpc_batch_plan_get(const ldpc_batch* b, ldpc_launch_info* out, int32_t cap, int32_t* n_launches) {
  if (!b || !n_launches || cap < 0 || (cap > 0 && !out)) return fail(LDPC_EINVAL, "bad arguments");
  *n_launches = static_cast<int32_t>(b->launches.size());
  for (int i = 0; i < std::min<int>(cap, static_cast<int>(b->launches.size())); ++i) {
    const Launch& L = b->launches[i];
    out[i] = ldpc_launch_info{L.block, L.grid, L.smem, L.item_count, L.rglobal ? 1 : 0, L.G};
  }
  return LDPC_OK;
}

int ldpc_graph_create(ldpc_session* s, const ldpc_batch* b, const void* sym_dev, const uint32_t* mask_dev,
                      void* llr_dev, uint32_t* bits_dev, int32_t* status_dev, uint8_t* d_dev,
                      uint64_t* goodput_bits_dev, uint32_t* goodput_sc_dev, float* reward_dev, ldpc_graph** out) {
  if (!s || !b || !out || b->s != s) return fail(LDPC_EINVAL, "bad graph arguments");
  *out = nullptr;
  cudaStream_t cap = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
  cudaStream_t saved = s->stream;
  s->stream = cap;
  int rc = LDPC_OK;
  cudaGraph_t graph = nullptr;
  e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    rc = cuda_fail(e, "cudaStreamBeginCapture");
  } else {
    rc = puncture_demap(s, b, sym_dev, mask_dev, llr_dev);
    if (!rc) rc = decode_batch(s, b, llr_dev, bits_dev, status_dev);
    if (!rc && b->info.n_tb) rc = tb_crc_goodput(s, b, bits_dev, d_dev, goodput_bits_dev, goodput_sc_dev, reward_dev);
    cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
    if (!rc && e2 != cudaSuccess) rc = cuda_fail(e2, "cudaStreamEndCapture");
  }
  s->stream = saved;
  ldpc_graph* g = nullptr;
  if (!rc) {
    g = new (std::nothrow) ldpc_graph();
    if (!g) {
      rc = fail(LDPC_ENOMEM, "host allocation");
    } else {
      e = cudaGraphInstantiate(&g->exec, graph, 0);
      if (e != cudaSuccess) {
        rc = cuda_fail(e, "cudaGraphInstantiate");
        delete g;
        g = nullptr;
      }
    }
  }
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(cap);
  if (rc) return rc;
  *out = g;
  return LDPC_OK;
}

int ldpc_graph_launch(ldpc_graph* g, void* stream) {
  if (!g) return fail(LDPC_EINVAL, "null graph");
  cudaError_t e = cudaGraphLaunch(g->exec, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? LDPC_OK : cuda_fail(e, "cudaGraphLaunch");
}

int ldpc_graph_destroy(ldpc_graph* g) {
  if (!g) return LDPC_OK;
  cudaGraphExecDestroy(g->exec);
  delete g;
  return LDPC_OK;
}

int ldpc_batch_info_get(const ldpc_batch* b, ldpc_batch_info* out) {
  if (!b || !out) return fail(LDPC_EINVAL, "null argument");
  *out = b->info;
  return LDPC_OK;
}

int puncture_demap(ldpc_session* s, const ldpc_batch* b, const void* sym_dev, const uint32_t* mask_dev,
                   void* llr_dev) {
  if (!s || !b || b->s != s) return fail(LDPC_EINVAL, "batch does not belong to this session");
  if (b->info.n_cb == 0) return LDPC_OK;
  if (!sym_dev || !mask_dev || !llr_dev) return fail(LDPC_EINVAL, "null buffer");
  if (reinterpret_cast<uintptr_t>(sym_dev) % 8) return fail(LDPC_EINVAL, "symbol buffer must be 8-byte aligned");
  DemapArgs a{};
  a.cbs = b->d_cbs;
  a.tiles = b->d_tiles;
  a.sym = static_cast<const float2*>(sym_dev);
  a.mask = mask_dev;
  a.llr = llr_dev;
  a.interleave = s->interleave;
  a.q_scale = s->q_scale;
  a.llr_sat = static_cast<float>(s->llr_sat);
  cudaError_t e = launch_demap(s->mode, b->n_tiles, s->stream, a);
  if (e == cudaSuccess && b->n_rep_tiles > 0) {  // LLR combining of repeated bits, after the main pass
    a.tiles = b->d_rep_tiles;
    e = launch_demap_repeat(s->mode, b->n_rep_tiles, s->stream, a);
  }
  return e == cudaSuccess ? LDPC_OK : cuda_fail(e, "puncture_demap launch");
}

int decode_batch(ldpc_session* s, const ldpc_batch* b, const void* llr_dev, uint32_t* bits_dev,
                 int32_t* status_dev) {
  if (!s || !b || b->s != s) return fail(LDPC_EINVAL, "batch does not belong to this session");
  if (b->info.n_cb == 0) return LDPC_OK;
  if (!llr_dev || !bits_dev || !status_dev) return fail(LDPC_EINVAL, "null buffer");
  if (reinterpret_cast<uintptr_t>(llr_dev) % 16) return fail(LDPC_EINVAL, "LLR buffer must be 16-byte aligned");
  if (!b->launches.empty()) {
    cudaError_t e = cudaMemsetAsync(b->d_queues, 0, b->launches.size() * sizeof(uint32_t), s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "decode_batch queue reset");
  }
  for (size_t li = 0; li < b->launches.size(); ++li) {
    const Launch& L = b->launches[li];
    DecodeArgs a{};
    a.shapes = b->d_shapes;
    a.tabs = b->d_tabs;
    a.cbs = b->d_cbs;
    a.item_cbs = b->d_item_cbs;
    a.items = b->d_items + L.item_begin;
    a.n_items = L.item_count;
    a.queue = b->d_queues + li;
    a.llr = llr_dev;
    a.bits = bits_dev;
    a.status = status_dev;
    a.err = s->d_err;
    a.rscratch = b->d_rscratch ? b->d_rscratch + L.rscratch_off : nullptr;
    a.rscratch_group = L.rscratch_group;
    a.G = L.G;
    a.hdr_bytes = L.hdr_bytes;
    a.max_iter = s->max_iter;
    a.early_term = s->early_term;
    a.cbcrc = s->d_cbcrc;
    if (s->mode == LDPC_F32) {
      a.beta = s->beta_f32;
      a.msg_sat = 3.0e38f;
      a.post_sat = 3.0e38f;
    } else {
      a.beta = static_cast<float>(s->offset_lsb);
      a.msg_sat = static_cast<float>(s->msg_sat);
      a.post_sat = static_cast<float>(s->post_sat);
    }
    cudaError_t e = launch_decode(s->mode, L.kind, dim3(L.grid), dim3(L.block), L.smem, s->stream, a);
    if (e != cudaSuccess) return cuda_fail(e, "decode_batch launch");
  }
  return LDPC_OK;
}

int ldpc_decode_cluster(ldpc_session* s, ldpc_batch* b, const void* llr_dev, uint32_t* bits_dev, int32_t* status_dev,
                        int32_t cluster_ctas) {
  try {
    if (!s || !b || b->s != s) return fail(LDPC_EINVAL, "batch does not belong to this session");
    if (cluster_ctas != 2 && cluster_ctas != 4) return fail(LDPC_EINVAL, "ldpc_decode_cluster: cluster_ctas must be 2 or 4");
    if (b->info.n_cb == 0) return LDPC_OK;
    if (!llr_dev || !bits_dev || !status_dev) return fail(LDPC_EINVAL, "null buffer");
    if (reinterpret_cast<uintptr_t>(llr_dev) % 16) return fail(LDPC_EINVAL, "LLR buffer must be 16-byte aligned");
    const int C = cluster_ctas;
    ldpc_batch::ClusterPlan& P = b->cplan[C == 2 ? 0 : 1];
    if (!P.built) {
      const int esz = s->mode == LDPC_F32 ? 4 : (s->mode == LDPC_I8 ? 1 : 2);
      std::map<int, std::vector<int>> by_z;  // one launch per lifting size (the CTA's threads are Z / C)
      std::map<int, std::pair<int, int>> shape_nm;  // session shape -> largest n_eff, m_eff in the batch
      for (int i = 0; i < b->info.n_cb; ++i) {
        const CbDev& c = b->cbs[i];
        if (c.Z % (32 * C) != 0)
          return fail(LDPC_EINVAL, "ldpc_decode_cluster: Z = " + std::to_string(c.Z) + " does not split into " +
                                       std::to_string(C) + " CTAs of whole warps");
        if (c.flags & LDPC_CB_CRC24B) return fail(LDPC_EINVAL, "ldpc_decode_cluster: code-block CRCs are not supported");
        by_z[c.Z].push_back(i);
        auto& nm = shape_nm[c.shape];
        nm.first = std::max(nm.first, c.n_eff);
        nm.second = std::max(nm.second, c.m_eff);
      }
      std::vector<uint32_t> tabs;
      std::vector<ShapeDev> shapes(s->shapes.size());
      for (auto& kv : shape_nm) {
        ShapeDev d = s->shapes[kv.first];
        build_table(s->bgs[d.bg], d.Z, kv.second.first * d.Z, tabs, d, kChunk);
        shapes[kv.first] = d;
      }
      std::vector<int32_t> list;
      for (auto& kv : by_z) {
        ldpc_batch::ClusterLaunch L;
        const int Z = kv.first;
        L.n = static_cast<int>(kv.second.size());
        L.list_off = static_cast<int>(list.size());
        L.block = Z / C;
        int tw = 0, max_n = 0, max_m = 0;
        for (int i : kv.second) {
          const CbDev& c = b->cbs[i];
          tw = std::max(tw, shapes[c.shape].tab_words);
          max_n = std::max(max_n, c.n_eff);
          max_m = std::max(max_m, c.m_eff);
          list.push_back(i);
        }
        const int msz = esz;
        L.tab_bytes = align16(tw * 4);
        L.L_bytes = align16((max_n + 1) * Z * esz);
        L.hb_bytes = align16(max_n * (Z / 32) * 4);
        L.rec_cap = max_m * L.block;
        L.smem = L.tab_bytes + 32 + L.L_bytes + L.hb_bytes + 2 * align16(L.rec_cap * msz) + align16(L.rec_cap * 4);
        if (L.smem > kMaxSmem)
          return fail(LDPC_EINVAL, "ldpc_decode_cluster: a Z = " + std::to_string(Z) + " block needs " +
                                       std::to_string(L.smem) + " B of shared memory per CTA");
        P.launches.push_back(L);
      }
      auto up = [&](auto** p, const auto& vec) -> cudaError_t {
        using T = std::remove_reference_t<decltype(vec[0])>;
        const size_t nbytes = std::max<size_t>(vec.size(), 1) * sizeof(T);
        cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), nbytes);
        if (e == cudaSuccess) {
          b->owned.push_back(*p);
          b->bytes += nbytes;
          if (!vec.empty()) e = cudaMemcpy(*p, vec.data(), vec.size() * sizeof(T), cudaMemcpyHostToDevice);
        }
        return e;
      };
      cudaError_t e = up(&P.d_tabs, tabs);
      if (e == cudaSuccess) e = up(&P.d_shapes, shapes);
      if (e == cudaSuccess) e = up(&P.d_list, list);
      if (e != cudaSuccess) return cuda_fail(e, "ldpc_decode_cluster plan");
      P.built = true;
    }
    for (const auto& L : P.launches) {
      ClusterArgs a{};
      a.shapes = P.d_shapes;
      a.tabs = P.d_tabs;
      a.cbs = b->d_cbs;
      a.cb_list = P.d_list + L.list_off;
      a.llr = llr_dev;
      a.bits = bits_dev;
      a.status = status_dev;
      a.err = s->d_err;
      a.tab_bytes = L.tab_bytes;
      a.L_bytes = L.L_bytes;
      a.hb_bytes = L.hb_bytes;
      a.rec_cap = L.rec_cap;
      a.max_iter = s->max_iter;
      a.early_term = s->early_term;
      if (s->mode == LDPC_F32) {
        a.beta = s->beta_f32;
        a.msg_sat = 3.0e38f;
        a.post_sat = 3.0e38f;
      } else {
        a.beta = static_cast<float>(s->offset_lsb);
        a.msg_sat = static_cast<float>(s->msg_sat);
        a.post_sat = static_cast<float>(s->post_sat);
      }
      const cudaError_t e = launch_cluster_decode(s->mode, C, L.n, L.block, L.smem, s->stream, a);
      if (e != cudaSuccess) return cuda_fail(e, "ldpc_decode_cluster launch");
    }
    return LDPC_OK;
  } catch (...) {
    return fail(LDPC_EINVAL, "unexpected host exception");
  }
}

int tb_crc_goodput(ldpc_session* s, const ldpc_batch* b, const uint32_t* bits_dev, uint8_t* d_dev,
                   uint64_t* goodput_bits_dev, uint32_t* goodput_sc_dev, float* reward_dev) {
  if (!s || !b || b->s != s) return fail(LDPC_EINVAL, "batch does not belong to this session");
  if (b->info.n_tb == 0) return fail(LDPC_EINVAL, "batch has no transport blocks");
  if (!bits_dev || !d_dev || !goodput_bits_dev || !goodput_sc_dev || !reward_dev)
    return fail(LDPC_EINVAL, "null buffer");
  CrcArgs a{};
  a.tbs = b->d_tbs;
  a.cbs = b->d_cbs;
  a.slot_start = b->d_slot_start;
  a.slot_tbs = b->d_slot_tbs;
  a.slot_N = b->d_slot_N;
  a.crc_table = s->d_crc_table;
  a.xpow32 = b->d_xpow32;
  a.crc_table_b = s->d_crc_table_b;
  a.xpow32_b = s->d_xpow32_b;
  a.bits = bits_dev;
  a.d = d_dev;
  a.goodput_bits = goodput_bits_dev;
  a.goodput_sc = goodput_sc_dev;
  a.reward = reward_dev;
  cudaError_t e = launch_crc(b->info.n_slots, s->stream, a);
  return e == cudaSuccess ? LDPC_OK : cuda_fail(e, "tb_crc_goodput launch");
}

int ldpc_check_log(uint32_t* out8) {
  if (!out8) return fail(LDPC_EINVAL, "null argument");
  cudaError_t e = read_check_log_decode(out8);
  if (e == cudaSuccess) e = read_check_log_serve(out8 + 4);
  return e == cudaSuccess ? LDPC_OK : cuda_fail(e, "ldpc_check_log");
}

int ldpc_device_errors(ldpc_session* s, uint32_t* flags_out) {
  if (!s || !flags_out) return fail(LDPC_EINVAL, "null argument");
  cudaError_t e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  uint32_t v = 0;
  e = cudaMemcpy(&v, s->d_err, sizeof(v), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy");
  *flags_out = v;
  if (v) cudaMemset(s->d_err, 0, sizeof(uint32_t));
  return LDPC_OK;
}

}  // extern "C"
