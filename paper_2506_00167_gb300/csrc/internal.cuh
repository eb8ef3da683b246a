// Internal types and device helpers shared by the ldpcgb translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "ldpcgb.h"

namespace ldpcgb {

constexpr int kMaxDeg = 27;      // sign bits 0..26 + 5-bit argmin index in one word
constexpr int kChunk = 2;        // edges per edge-table chunk of the batch decoders: bases, then shifts
constexpr int kServeChunk = 4;   // the same for the serving loop (its latency-bound loop wants four)
template <int CH>
struct MaxChunks {
  static constexpr int value = (kMaxDeg + CH - 1) / CH;
};
constexpr int kMaxChunks = MaxChunks<kChunk>::value;
constexpr int kMaxZ = 384;
constexpr int kMaxSmem = 232448; // 227 KB dynamic shared memory per block (sm_100 family)
constexpr int kDecodeMaxBlock = 384;  // decoder blocks: two of them share an SM's registers
constexpr int kTileMaxBlock = 512;    // largest G * Z a tile may request
constexpr int kCrcBlock = 256;

// One (base graph, Z) pair as one decoder launch sees it.  Its edge table is,
// per row, chunks of CH edges as 2 * CH words (CH = kChunk for the batch
// decoders, kServeChunk for the serving loop; one 16-byte load per chunk for
// CH = 2): the column bases (col * Z), then the shifts (V mod Z); a row's
// last chunk is padded with edges whose base is the launch's dummy slot and
// whose shift is 0.  Then one word per row, start | (degree << 16) (start in
// words from the table base); then padding to a multiple of 4 words.
struct ShapeDev {
  int32_t bg, Z, mb, nb, kb, mc, npc;
  int32_t tab_off;    // first word of this shape's table
  int32_t row_off;    // row words, relative to tab_off
  int32_t tab_words;  // multiple of 4 (whole table, 16-byte granules)
  int32_t crc_off;    // first word of its code-block CRC byte table (kb * Z * 32 words)
};

// Per code block geometry, computed on the host at batch creation.
struct CbDev {
  int32_t shape, Z, Qm, E;
  int32_t t0, m_eff, n_eff, n_re;
  int32_t kb, flags;  // flags: LDPC_CB_CRC24B
  int64_t re_off, mask_off, llr_off, bits_off;
  float inv_sigma2;
  int32_t k0;  // start of the redundancy version in the circular buffer (0 for version 0)
};

// One decoder work item: `count` code blocks of one shape, listed from
// item_cbs[first]; each is decoded by its own group of Z threads.  The item
// carries its own shared-memory layout, so one launch can mix lifting sizes:
// group g's region starts at g * region_bytes and holds the posteriors
// (L_bytes, with Z dummy slots at element dummy_base), the hard-decision
// bitmap (hb_bytes) and, unless the launch keeps messages in global memory,
// rec_cap compressed check records.
struct DecodeItem {
  int32_t shape, first, count, Z;
  int32_t region_bytes, L_bytes, hb_bytes, rec_cap;
  int32_t dummy_base, pad0, pad1, pad2;
};

struct DemapTile {
  int32_t cb, re_start;
};

struct TbDev {
  int32_t first_cb, n_cb, n_sc, slot, payload_bits;
  int32_t bytes;  // (payload_bits + 24) / 8: the bytes the TB CRC runs over
  int32_t seg;    // 1: every block carries its own CRC (its last 3 bytes are not TB bytes)
  int32_t pad;
};

struct DecodeArgs {
  const ShapeDev* shapes;
  const uint32_t* tabs;
  const CbDev* cbs;
  const int32_t* item_cbs;
  const DecodeItem* items;
  int32_t n_items;
  uint32_t* queue;          // work-queue counter (zeroed before the launch), or null: static stride
  const void* llr;
  uint32_t* bits;
  int32_t* status;
  uint32_t* err;
  uint8_t* rscratch;        // R records in global memory (RGLOBAL variant)
  int64_t rscratch_group;   // bytes per (block, group) slot
  int32_t G;                // group slots per block in rscratch
  int32_t hdr_bytes;        // edge table + mbarrier + item slot, 16-byte multiple
  int32_t max_iter, early_term;
  float beta, msg_sat, post_sat;
  const uint32_t* cbcrc;    // code-block CRC byte tables (ShapeDev::crc_off), for LDPC_CB_CRC24B blocks
};

// The cluster decoder (decode_cluster.cu): one code block per cluster of C
// CTAs; cb_list names the launch's blocks in cluster order.  Per-CTA shared
// layout: table (tab_bytes), mbarrier and flags (32 bytes), the block's
// posterior replica (L_bytes), its hard-decision bitmap (hb_bytes), the
// messages of the CTA's own checks (rec_cap records).
struct ClusterArgs {
  const ShapeDev* shapes;  // indexed by the session's shape index
  const uint32_t* tabs;
  const CbDev* cbs;
  const int32_t* cb_list;
  const void* llr;
  uint32_t* bits;
  int32_t* status;
  uint32_t* err;
  int32_t tab_bytes, L_bytes, hb_bytes, rec_cap;
  int32_t max_iter, early_term;
  float beta, msg_sat, post_sat;
};

struct DemapArgs {
  const CbDev* cbs;
  const DemapTile* tiles;
  const float2* sym;
  const uint32_t* mask;
  void* llr;
  int32_t interleave;
  float q_scale, llr_sat;
};

struct CrcArgs {
  const TbDev* tbs;
  const CbDev* cbs;
  const int32_t* slot_start;  // n_slots + 1
  const int32_t* slot_tbs;
  const int32_t* slot_N;
  const uint32_t* crc_table;  // 256 entries
  const uint32_t* xpow32;     // x^(32 m) mod g, m = 0..max_words
  const uint32_t* crc_table_b;  // the same two tables for the code-block generator g_B
  const uint32_t* xpow32_b;     // m = 0..largest block's words
  const uint32_t* bits;
  uint8_t* d;
  uint64_t* goodput_bits;
  uint32_t* goodput_sc;
  float* reward;
};

// ---------------------------------------------------------------- host side
void set_error(const std::string& msg);

// Kernel launchers (defined next to their kernels).
// Decoder kernel kinds: messages in shared memory, in global memory, or the
// INT8 kernel that decodes two code blocks per thread group (messages in
// shared or in global memory).
// Either can carry kKindCrc: the variant with the code-block CRC exit.
constexpr int kKindShared = 0;
constexpr int kKindGlobal = 1;
constexpr int kKindPairI8 = 2;
constexpr int kKindPairI8Global = 3;
constexpr int kKinds = 4;
constexpr int kKindCrc = 4;
constexpr bool kind_is_pair(int kind) {
  return (kind & ~kKindCrc) == kKindPairI8 || (kind & ~kKindCrc) == kKindPairI8Global;
}
constexpr bool kind_is_global(int kind) {
  return (kind & ~kKindCrc) == kKindGlobal || (kind & ~kKindCrc) == kKindPairI8Global;
}
cudaError_t launch_decode(int mode, int kind, dim3 grid, dim3 block, int smem, cudaStream_t st,
                          const DecodeArgs& a);
cudaError_t decode_occupancy(int mode, int kind, int block, int smem, int* blocks_per_sm);
cudaError_t decode_prepare(int mode);  // raise the dynamic shared-memory limit
cudaError_t launch_demap(int mode, int n_tiles, cudaStream_t st, const DemapArgs& a);
cudaError_t launch_demap_repeat(int mode, int n_tiles, cudaStream_t st, const DemapArgs& a);
cudaError_t launch_crc(int n_slots, cudaStream_t st, const CrcArgs& a);
cudaError_t launch_cluster_decode(int mode, int C, int n_clusters, int block, int smem, cudaStream_t st,
                                  const ClusterArgs& a);
// Checked builds: the first failed device check of the decoder and of the
// serving loop (4 words each; zeros when none failed or checks are off).
cudaError_t read_check_log_decode(uint32_t* out4);
cudaError_t read_check_log_serve(uint32_t* out4);

constexpr int kDemapBlock = 256;
constexpr int kDemapPerThread = 4;                        // resource elements per thread
constexpr int kDemapTile = kDemapBlock * kDemapPerThread;  // resource elements per block

}  // namespace ldpcgb

// ---------------------------------------------------------------- device helpers
#ifdef __CUDACC__
namespace ldpcgb {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Make generic-proxy shared-memory traffic visible to / ordered with the
// async (bulk-copy) proxy.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

// Bulk (TMA engine) copy global -> this CTA's shared memory, completing on `bar`.
// Both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// Bounded wait: gives up after `limit` polls (each poll may itself suspend
// for a short hardware-defined time).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t limit) {
  for (uint32_t i = 0; i < limit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void named_bar_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// ---- checked builds (nvcc -DLDPC_CHECKED): indices that the kernels trust
// are tested; the first failure of a translation unit is logged as
// {check id, value, limit, block * 1024 + thread} and the access is
// redirected to a safe slot, so a bad index never leaves the buffer.
#ifdef LDPC_CHECKED
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif

static __device__ uint32_t g_check_log[4];

__device__ __forceinline__ bool check_ok(bool ok, uint32_t id, int value, int limit) {
  if constexpr (kChecked) {
    if (!ok && atomicCAS(&g_check_log[0], 0u, id) == 0u) {
      g_check_log[1] = static_cast<uint32_t>(value);
      g_check_log[2] = static_cast<uint32_t>(limit);
      g_check_log[3] = blockIdx.x * 1024u + threadIdx.x;
    }
    return ok;
  } else {
    return true;
  }
}

// i if 0 <= i < limit, else (logged) `safe`.
__device__ __forceinline__ int checked(int i, int limit, int safe, uint32_t id) {
  if constexpr (kChecked)
    return check_ok(static_cast<uint32_t>(i) < static_cast<uint32_t>(limit), id, i, limit) ? i : safe;
  else
    return i;
}

// Barrier over `nthreads` threads on barrier `id` that also ORs `pred`.
__device__ __forceinline__ bool named_bar_or(int id, int nthreads, bool pred) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.or.pred q, %2, %3, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)pred), "r"(id), "r"(nthreads)
      : "memory");
  return r != 0;
}

}  // namespace ldpcgb
#endif
