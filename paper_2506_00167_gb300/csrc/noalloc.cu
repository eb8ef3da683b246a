// decode_uniform_noalloc: layered offset-min-sum decoding of code blocks of
// one shape with no device-memory allocation at all.
//
// Who needs it: callers that cannot call cudaMalloc -- for example code that
// runs under a memory pool or budget that forbids new allocations once set
// up, inside a real-time receive loop where an allocation's latency or
// failure is not acceptable, or in a host application that owns all device
// memory and hands the library only its buffers.  Everything the
// decoder needs beyond the caller's input and output buffers lives in one
// file-scope __device__ array of fixed size (kScratchBytes below), which every
// GPU that loads this library holds until the process exits.
//
// Layout of the array: [error word] [shape record] [edge table] [code-block
// descriptors] [work items] [item list] [check-to-variable messages].  A small
// set-up kernel fills the descriptor part on the device (the edge table
// travels in its kernel parameters), then the regular decoder kernel runs in
// its global-message variant with its messages in the array.
//
// Concurrency: every call uses the same array and leaves its contents
// behind.  Calls whose work overlaps on the GPU (different streams, or
// different host threads on one device) race on it; serialise them.
#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "internal.cuh"

namespace ldpcgb {

namespace {

constexpr size_t kScratchBytes = size_t(24) << 20;  // 24 MiB per device
constexpr int kMaxCb = 32768;                       // code blocks per call
constexpr int kMaxTabWords = 4096;                  // 16 KB edge table (any base graph this library accepts)
constexpr size_t kOffErr = 0;
constexpr size_t kOffShape = 256;
constexpr size_t kOffTab = 512;
constexpr size_t kOffCbs = kOffTab + kMaxTabWords * 4;
constexpr size_t kOffItems = kOffCbs + size_t(kMaxCb) * sizeof(CbDev);
constexpr size_t kOffItemCbs = kOffItems + size_t(kMaxCb) * sizeof(DecodeItem);
constexpr size_t kOffRec = (kOffItemCbs + size_t(kMaxCb) * 4 + 255) & ~size_t(255);

static __device__ __align__(256) uint8_t g_scratch[kScratchBytes];

struct SetupArgs {
  uint32_t tab[kMaxTabWords];
  ShapeDev shape;
  CbDev proto;       // geometry shared by every code block; offsets filled per block
  DecodeItem proto_item;  // layout shared by every work item; first/count filled per item
  int32_t n_cb, G;
  uint8_t* scratch;
};

// Writes the shape, table, per-block descriptors and work items into the array.
__global__ void noalloc_setup_kernel(const SetupArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  uint8_t* base = a.scratch;
  if (i == 0) {
    *reinterpret_cast<uint32_t*>(base + kOffErr) = 0u;
    *reinterpret_cast<ShapeDev*>(base + kOffShape) = a.shape;
  }
  if (blockIdx.x == 0)
    for (int w = threadIdx.x; w < a.shape.tab_words; w += blockDim.x)
      reinterpret_cast<uint32_t*>(base + kOffTab)[w] = a.tab[w];
  if (i < a.n_cb) {
    CbDev d = a.proto;
    d.llr_off = static_cast<int64_t>(i) * d.n_eff * d.Z;
    d.bits_off = static_cast<int64_t>(i) * ((d.kb * d.Z) >> 5);
    reinterpret_cast<CbDev*>(base + kOffCbs)[i] = d;
    reinterpret_cast<int32_t*>(base + kOffItemCbs)[i] = i;
    if (i % a.G == 0) {
      DecodeItem it = a.proto_item;
      it.first = i;
      it.count = min(a.G, a.n_cb - i);
      reinterpret_cast<DecodeItem*>(base + kOffItems)[i / a.G] = it;
    }
  }
}

// A bulk-copy-style wait on an mbarrier that nothing completes: the bounded
// wait the decoder uses gives up after `limit` polls and records
// LDPC_DEVERR_TMA_TIMEOUT in the error word, as a decode whose copy never
// landed would.  Lets a caller check that a wait running out is reported
// (decode_uniform_noalloc_errors) and leaves the context usable.
__global__ void noalloc_wait_check_kernel(uint32_t limit, uint8_t* scratch) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_proxy_async_smem();
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait_bounded(&bar, 0u, limit))
    atomicOr(reinterpret_cast<uint32_t*>(scratch + kOffErr), LDPC_DEVERR_TMA_TIMEOUT);
}

// Device address of g_scratch per device, looked up once per device.
std::mutex g_mu;
std::vector<uint8_t*> g_addr;

int scratch_for_current_device(uint8_t** out, std::string* err) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    *err = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
    return LDPC_ECUDA;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (static_cast<int>(g_addr.size()) <= dev) g_addr.resize(dev + 1, nullptr);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) {
      *err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
      return LDPC_ECUDA;
    }
    for (int mode = LDPC_F32; mode <= LDPC_I16; ++mode) {
      e = decode_prepare(mode);
      if (e != cudaSuccess) {
        *err = std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e);
        return LDPC_ECUDA;
      }
    }
    g_addr[dev] = static_cast<uint8_t*>(p);
  }
  *out = g_addr[dev];
  return LDPC_OK;
}

int align16i(int x) { return (x + 15) & ~15; }

}  // namespace

}  // namespace ldpcgb

using namespace ldpcgb;

extern "C" LDPC_API int decode_uniform_noalloc(const ldpc_base_graph* g, int32_t Z, int32_t E, int32_t n_cb,
                                               int32_t mode, int32_t max_iter, int32_t early_term, float offset_f32,
                                               int32_t offset_lsb, int32_t msg_sat, int32_t post_sat,
                                               const void* llr_dev, uint32_t* bits_dev, int32_t* status_dev,
                                               void* cuda_stream) {
  try {
    // ---- validate (same rules as ldpc_session_create / ldpc_batch_create)
    if (!g || !g->row || !g->col || !g->V) {
      set_error("decode_uniform_noalloc: null base graph");
      return LDPC_EINVAL;
    }
    if (n_cb < 0 || n_cb > kMaxCb) {
      set_error("decode_uniform_noalloc: n_cb must be 0.." + std::to_string(kMaxCb) +
                " (fixed scratch of " + std::to_string(kScratchBytes >> 20) + " MiB)");
      return LDPC_EINVAL;
    }
    if (n_cb == 0) return LDPC_OK;
    if (!llr_dev || !bits_dev || !status_dev || reinterpret_cast<uintptr_t>(llr_dev) % 16) {
      set_error("decode_uniform_noalloc: null or misaligned buffer (LLRs need 16-byte alignment)");
      return LDPC_EINVAL;
    }
    if (mode < LDPC_F32 || mode > LDPC_I16 || max_iter < 1 || max_iter > 64) {
      set_error("decode_uniform_noalloc: bad mode or max_iter");
      return LDPC_EINVAL;
    }
    if (mode != LDPC_F32) {
      const int lim = mode == LDPC_I8 ? 127 : 32767;
      if (post_sat < 1 || post_sat > lim || msg_sat < 1 || msg_sat > post_sat || offset_lsb < 0) {
        set_error("decode_uniform_noalloc: integer saturation/offset out of range");
        return LDPC_EINVAL;
      }
    }
    if (!(Z == 16 || (Z >= 32 && Z <= kMaxZ && Z % 32 == 0))) {
      set_error("decode_uniform_noalloc: Z must be 16 or a multiple of 32 <= 384");
      return LDPC_EINVAL;
    }
    const int mb = g->mb, nb = g->nb, kb = g->kb, mc = g->mc, npc = g->n_punct_cols;
    if (mb < 1 || nb <= mb || kb != nb - mb || mc < 1 || mc > mb || npc < 0 || npc > kb || g->n_edges < 1 ||
        (kb * Z) % 32) {
      set_error("decode_uniform_noalloc: bad base-graph sizes");
      return LDPC_EINVAL;
    }
    const int t0 = npc * Z;
    if (E <= 0 || E > 2 * (nb * Z - t0)) {  // the rate-matching circular buffer may wrap once
      set_error("decode_uniform_noalloc: need 0 < E <= 2 (nb * Z - t0)");
      return LDPC_EINVAL;
    }
    const int m_eff = std::min(mb, std::max(mc, (E + t0 + Z - 1) / Z - kb));
    const int n_eff = kb + m_eff;
    std::vector<std::vector<int>> cols(mb), shs(mb);
    int prev_r = -1, prev_c = -1, maxcol = 0;
    for (int e = 0; e < g->n_edges; ++e) {
      const int r = g->row[e], c = g->col[e], v = g->V[e];
      if (r < 0 || r >= mb || c < 0 || c >= nb || v < 0 || r < prev_r || (r == prev_r && c <= prev_c)) {
        set_error("decode_uniform_noalloc: edges must be row-major, unique, in range");
        return LDPC_EINVAL;
      }
      prev_r = r;
      prev_c = c;
      cols[r].push_back(c * Z);
      shs[r].push_back(v % Z);
      if (r < m_eff) maxcol = std::max(maxcol, c);
    }
    for (int r = 0; r < mb; ++r)
      if (cols[r].size() < 2 || cols[r].size() > static_cast<size_t>(kMaxDeg)) {
        set_error("decode_uniform_noalloc: row degree must be 2..27");
        return LDPC_EINVAL;
      }
    if (maxcol >= n_eff) {
      set_error("decode_uniform_noalloc: a decoded row uses a column beyond the decoded ones");
      return LDPC_EINVAL;
    }

    // ---- geometry and shared-memory plan (one launch, G code blocks per block)
    const int esz = mode == LDPC_F32 ? 4 : (mode == LDPC_I8 ? 1 : 2);
    const int msz = esz;
    const int dummy = n_eff * Z;
    static_assert(sizeof(SetupArgs) < 32000, "kernel parameters");
    SetupArgs sa{};
    std::vector<uint32_t> rowinfo;
    int words = 0;
    for (int r = 0; r < mb; ++r) {
      const int deg = static_cast<int>(cols[r].size());
      const int start = words;
      // chunks of kChunk edges: the column bases, then the shifts (the decoder's table layout)
      for (int c = 0; c < (deg + kChunk - 1) / kChunk; ++c) {
        if (words + 2 * kChunk > kMaxTabWords) {
          set_error("decode_uniform_noalloc: edge table too large");
          return LDPC_EINVAL;
        }
        for (int i = 0; i < kChunk; ++i) sa.tab[words++] = kChunk * c + i < deg ? cols[r][kChunk * c + i] : dummy;
        for (int i = 0; i < kChunk; ++i) sa.tab[words++] = kChunk * c + i < deg ? shs[r][kChunk * c + i] : 0;
      }
      rowinfo.push_back(static_cast<uint32_t>(start) | (static_cast<uint32_t>(deg) << 16));
    }
    const int row_off = words;
    if (words + mb + 3 > kMaxTabWords) {
      set_error("decode_uniform_noalloc: edge table too large");
      return LDPC_EINVAL;
    }
    for (uint32_t ri : rowinfo) sa.tab[words++] = ri;
    while (words % 4) sa.tab[words++] = 0;

    ShapeDev sh{};
    sh.bg = 0;
    sh.Z = Z;
    sh.mb = mb;
    sh.nb = nb;
    sh.kb = kb;
    sh.mc = mc;
    sh.npc = npc;
    sh.tab_off = 0;
    sh.row_off = row_off;
    sh.tab_words = words;

    const int rec_cap = m_eff * Z;
    const int rec_bytes = 2 * align16i(rec_cap * msz) + align16i(rec_cap * 4);
    const int L_bytes = align16i((n_eff + 1) * Z * esz);
    const int hb_bytes = (Z % 32 == 0) ? align16i(n_eff * (Z / 32) * 4) : 0;
    const int hdr_bytes = align16i(words * 4) + 16;
    int G = std::max(1, 256 / Z);
    if (Z > 32) G = std::min(G, 15);
    while (G > 1 && G * Z > kDecodeMaxBlock) --G;
    const int region = L_bytes + hb_bytes;
    while (G > 1 && hdr_bytes + G * region > kMaxSmem) --G;
    // Z = 16: two groups share a warp, so an even group count keeps every warp whole (as the batch planner)
    if (Z == 16 && G > 1 && (G & 1)) --G;
    if (hdr_bytes + G * region > kMaxSmem) {
      set_error("decode_uniform_noalloc: code block too large for shared memory");
      return LDPC_EINVAL;
    }
    const size_t rec_room = kScratchBytes - kOffRec;
    const int max_slots = static_cast<int>(rec_room / (static_cast<size_t>(G) * rec_bytes));
    if (max_slots < 1) {
      set_error("decode_uniform_noalloc: one code block's messages (" + std::to_string(rec_bytes) +
                " bytes) exceed the fixed scratch");
      return LDPC_EINVAL;
    }

    uint8_t* scratch = nullptr;
    std::string err;
    int rc = scratch_for_current_device(&scratch, &err);
    if (rc) {
      set_error("decode_uniform_noalloc: " + err);
      return rc;
    }
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int block = (G * Z + 31) & ~31;
    const int smem = hdr_bytes + G * region;
    cudaError_t e = decode_occupancy(mode, kKindGlobal, block, smem, &per_sm);
    if (e != cudaSuccess || per_sm < 1) {
      set_error("decode_uniform_noalloc: occupancy query failed");
      return LDPC_ECUDA;
    }
    const int n_items = (n_cb + G - 1) / G;
    const int grid = std::min({n_items, per_sm * sms, max_slots});

    // ---- set-up kernel: descriptors into the fixed array
    CbDev proto{};
    proto.shape = 0;
    proto.Z = Z;
    proto.Qm = 2;
    proto.E = E;
    proto.t0 = t0;
    proto.m_eff = m_eff;
    proto.n_eff = n_eff;
    proto.n_re = E / 2;
    proto.kb = kb;
    sa.shape = sh;
    sa.proto = proto;
    DecodeItem pit{};
    pit.shape = 0;
    pit.Z = Z;
    pit.region_bytes = region;
    pit.L_bytes = L_bytes;
    pit.hb_bytes = hb_bytes;
    pit.rec_cap = rec_cap;
    pit.dummy_base = dummy;
    sa.proto_item = pit;
    sa.n_cb = n_cb;
    sa.G = G;
    sa.scratch = scratch;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    void* sargs[] = {&sa};
    e = cudaLaunchKernel(reinterpret_cast<const void*>(&noalloc_setup_kernel), dim3((n_cb + 255) / 256),
                         dim3(256), sargs, 0, st);
    if (e != cudaSuccess) {
      set_error(std::string("decode_uniform_noalloc: setup launch: ") + cudaGetErrorString(e));
      return LDPC_ECUDA;
    }

    // ---- the decoder, messages in the fixed array
    DecodeArgs a{};
    a.shapes = reinterpret_cast<const ShapeDev*>(scratch + kOffShape);
    a.tabs = reinterpret_cast<const uint32_t*>(scratch + kOffTab);
    a.cbs = reinterpret_cast<const CbDev*>(scratch + kOffCbs);
    a.item_cbs = reinterpret_cast<const int32_t*>(scratch + kOffItemCbs);
    a.items = reinterpret_cast<const DecodeItem*>(scratch + kOffItems);
    a.n_items = n_items;
    a.queue = nullptr;
    a.llr = llr_dev;
    a.bits = bits_dev;
    a.status = status_dev;
    a.err = reinterpret_cast<uint32_t*>(scratch + kOffErr);
    a.rscratch = scratch + kOffRec;
    a.rscratch_group = rec_bytes;
    a.G = G;
    a.hdr_bytes = hdr_bytes;
    a.max_iter = max_iter;
    a.early_term = early_term ? 1 : 0;
    if (mode == LDPC_F32) {
      a.beta = offset_f32;
      a.msg_sat = 3.0e38f;
      a.post_sat = 3.0e38f;
    } else {
      a.beta = static_cast<float>(offset_lsb);
      a.msg_sat = static_cast<float>(msg_sat);
      a.post_sat = static_cast<float>(post_sat);
    }
    e = launch_decode(mode, kKindGlobal, dim3(grid), dim3(block), smem, st, a);
    if (e != cudaSuccess) {
      set_error(std::string("decode_uniform_noalloc: decode launch: ") + cudaGetErrorString(e));
      return LDPC_ECUDA;
    }
    return LDPC_OK;
  } catch (...) {
    set_error("decode_uniform_noalloc: unexpected host exception");
    return LDPC_EINVAL;
  }
}

/* The device error word of the no-allocation decoder on the current device: each decode_uniform_noalloc
 * call clears it before it decodes, and a decoder work item whose bounded bulk-copy wait gave up sets
 * LDPC_DEVERR_TMA_TIMEOUT there (that item's bits and status are then not written).  Waits for
 * `cuda_stream`, reads the word into *flags_out and clears it; allocates nothing. */
extern "C" LDPC_API int decode_uniform_noalloc_errors(uint32_t* flags_out, void* cuda_stream) {
  if (!flags_out) {
    set_error("decode_uniform_noalloc_errors: null output");
    return LDPC_EINVAL;
  }
  uint8_t* scratch = nullptr;
  std::string err;
  int rc = scratch_for_current_device(&scratch, &err);
  if (rc) {
    set_error("decode_uniform_noalloc_errors: " + err);
    return rc;
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  uint32_t v = 0;
  cudaError_t e = cudaMemcpyAsync(&v, scratch + kOffErr, sizeof(v), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(scratch + kOffErr, 0, sizeof(uint32_t), st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    set_error(std::string("decode_uniform_noalloc_errors: ") + cudaGetErrorString(e));
    return LDPC_ECUDA;
  }
  *flags_out = v;
  return LDPC_OK;
}

/* Run the decoder's bounded bulk-copy wait on an mbarrier that nothing completes, with a limit of
 * `limit` polls (1..65536): the wait gives up and sets LDPC_DEVERR_TMA_TIMEOUT in the word that
 * decode_uniform_noalloc_errors reads.  For tests of the failure report; enqueued on `cuda_stream`. */
extern "C" LDPC_API int decode_uniform_noalloc_wait_check(int32_t limit, void* cuda_stream) {
  if (limit < 1 || limit > 65536) {
    set_error("decode_uniform_noalloc_wait_check: limit must be 1..65536");
    return LDPC_EINVAL;
  }
  uint8_t* scratch = nullptr;
  std::string err;
  int rc = scratch_for_current_device(&scratch, &err);
  if (rc) {
    set_error("decode_uniform_noalloc_wait_check: " + err);
    return rc;
  }
  noalloc_wait_check_kernel<<<1, 32, 0, static_cast<cudaStream_t>(cuda_stream)>>>(static_cast<uint32_t>(limit),
                                                                                   scratch);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("decode_uniform_noalloc_wait_check: ") + cudaGetErrorString(e));
    return LDPC_ECUDA;
  }
  return LDPC_OK;
}
