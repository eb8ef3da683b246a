// Layered offset-min-sum decoding of one code block on a cluster of C CTAs
// (C = 2 or 4 SMs per block): the latency form of the batch decoder.
//
// The decode of one large block on one SM is bound by that SM's issue rate
// (a BG1-shaped Z = 384 block runs ~3,200 warp instructions per layer), so a
// lone block -- the tail of a served stream -- decodes no faster however idle
// the GPU is.  Here the Z lifted checks of every layer are split over the C
// CTAs of a thread-block cluster (CTA r owns checks r Z/C .. (r+1) Z/C - 1),
// and every CTA keeps a full replica of the block's posteriors in its shared
// memory: a check reads its variables from the local replica, and pass 2
// writes each new posterior into all C replicas (st.shared::cluster to the
// other CTAs' copies, through their mapa addresses).  Each check's compressed
// messages stay in its own CTA.  A cluster barrier (release / acquire)
// separates the layers, so every replica holds the same values when the next
// layer reads them -- the layered schedule and its arithmetic are exactly the
// batch decoder's (the same check_update), so results are bit-identical.
// After an iteration every CTA computes the hard decisions and the whole
// syndrome from its own replica; the replicas are equal, so all CTAs reach
// the same early-exit decision and the control flow stays uniform across the
// cluster (no CTA leaves while another could still write into it); one more
// cluster barrier keeps the next iteration's writes from reaching a replica
// still being read for the syndrome.
//
// On GB300 this form decodes a lone block more slowly than one CTA does (a
// BG1-shaped Z = 384 block at R = 1/3, FP32, 10 iterations: 285 us on one CTA,
// 374 us on 2, 470 us on 4): the per-layer cluster barrier and the remote
// replica stores cost more than the halved issue work saves.  The decode
// service therefore keeps one CTA per block.
#include <string>

#include "decode_core.cuh"

namespace ldpcgb {

namespace {

using namespace core;

constexpr int kClusterMaxBlock = 192;  // Z / C threads: 384 / 2

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ uint32_t cluster_id_x() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}

__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t map_rank(uint32_t local_smem, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local_smem), "r"(rank));
  return r;
}

__device__ __forceinline__ void st_cluster_u32(uint32_t a, uint32_t v) {
  asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}

// Z % 32 == 0: is any (row, word) syndrome word nonzero among this thread's
// tasks (task = tid, tid + nthr, ...)?  As syndrome_bitmap, with the CTA's
// threads striding over all m_eff * Z / 32 words.
__device__ __forceinline__ bool syndrome_words(const uint32_t* __restrict__ tab, const uint32_t* __restrict__ rows,
                                               const uint32_t* __restrict__ hb, int m_eff, int tid, int nthr, int Z) {
  const int W = Z >> 5;
  uint32_t bad = 0;
  for (int task = tid; task < m_eff * W; task += nthr) {
    const int l = task / W;
    const int ww = task - l * W;
    const uint32_t info = rows[l];
    const uint32_t* rt = tab + (info & 0xFFFFu);
    const int deg = static_cast<int>(info >> 16);
    uint32_t x = 0;
    for (int e = 0; e < deg; ++e) {
      const uint2 bs = edge_at<kChunk>(rt, e);
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

template <typename LT, typename MT, bool SAT, int C>
__global__ void __launch_bounds__(kClusterMaxBlock) oms_cluster_kernel(const ClusterArgs a) {
  extern __shared__ __align__(128) uint8_t smem[];
  uint32_t* s_tab = reinterpret_cast<uint32_t*>(smem);
  uint64_t* s_bar = reinterpret_cast<uint64_t*>(smem + a.tab_bytes);
  uint32_t* s_flag = reinterpret_cast<uint32_t*>(smem + a.tab_bytes + 16);  // C words: each CTA's copy status
  LT* L = reinterpret_cast<LT*>(smem + a.tab_bytes + 32);
  uint32_t* hb = reinterpret_cast<uint32_t*>(smem + a.tab_bytes + 32 + a.L_bytes);
  uint8_t* rb = smem + a.tab_bytes + 32 + a.L_bytes + a.hb_bytes;
  MT* mag1 = reinterpret_cast<MT*>(rb);
  MT* mag2 = mag1 + a.rec_cap;
  uint32_t* meta = reinterpret_cast<uint32_t*>(rb + 2 * ((a.rec_cap * sizeof(MT) + 15) & ~15));

  const int tid = threadIdx.x;
  const int nthr = blockDim.x;
  const uint32_t rank = cluster_rank();
  const CbDev cb = a.cbs[a.cb_list[cluster_id_x()]];
  const ShapeDev sh = a.shapes[cb.shape];
  const int Z = cb.Z;
  const int k = static_cast<int>(rank) * nthr + tid;  // this thread's lifted check

  if (tid == 0) {
    mbar_init(s_bar, 1);
    fence_proxy_async_smem();
  }
  __syncthreads();
  cluster_sync();  // every CTA of the cluster runs before any writes into another's shared memory
  if (tid == 0) {
    const uint32_t tb = static_cast<uint32_t>(sh.tab_words) * 4u;
    const uint32_t lb = static_cast<uint32_t>(cb.n_eff * Z) * sizeof(LT);
    mbar_arrive_expect_tx(s_bar, tb + lb);
    bulk_g2s(s_tab, a.tabs + sh.tab_off, tb, s_bar);
    bulk_g2s(L, static_cast<const LT*>(a.llr) + cb.llr_off, lb, s_bar);
  }
  zero_records(mag1, mag2, meta, cb.m_eff * nthr, tid, nthr);  // this CTA's checks: record l * nthr + tid
  const bool got = mbar_wait_bounded(s_bar, 0u, 1u << 22);
  const bool all_got = __syncthreads_and(got);
  // every CTA learns whether every copy landed before anything depends on them
  if (tid < C) st_cluster_u32(map_rank(smem_addr(s_flag + rank), static_cast<uint32_t>(tid)), all_got ? 1u : 0u);
  cluster_sync();
  bool fine = true;
#pragma unroll
  for (int r = 0; r < C; ++r) fine = fine && s_flag[r] != 0u;
  if (!fine) {
    if (rank == 0 && tid == 0) atomicOr(a.err, LDPC_DEVERR_TMA_TIMEOUT);
    if (!all_got) mbar_wait_bounded(s_bar, 0u, 1u << 20);  // copies still in flight: a bounded chance to land
    cluster_sync();
    return;
  }
  if constexpr (!SAT) {  // -0.0 from a caller would carry a sign bit while not being < 0
    for (int i = tid; i < cb.n_eff * Z; i += nthr) L[i] = L[i] + LT(0);
  }
  __syncthreads();
  uint32_t rep[C - 1];  // the other CTAs' replicas
  const uint32_t lsh = smem_addr(L);
#pragma unroll
  for (int r = 1; r < C; ++r) rep[r - 1] = map_rank(lsh, (rank + static_cast<uint32_t>(r)) % C);

  const uint32_t* rows = s_tab + sh.row_off;
  const int m = cb.m_eff;
  const int dummy = cb.n_eff * Z + k;  // (checked builds: the replica's posterior slots)
  int it = 1;
  bool ok = false;
  RowIn<kChunk> row = load_row<kChunk>(s_tab, rows[0], mag1, mag2, meta, tid);
  for (;; ++it) {
    for (int l = 0; l < m; ++l) {
      check_update_exact<LT, MT, SAT, false, kChunk, 2, C>(row, k, Z, L, mag1, mag2, meta, l * nthr + tid, dummy,
                                                           a.beta, a.msg_sat, a.post_sat, rep);
      const int ln = l + 1 < m ? l + 1 : 0;
      row = load_row<kChunk>(s_tab, rows[ln], mag1, mag2, meta, ln * nthr + tid);
      cluster_sync();  // every replica holds the layer's posteriors before the next layer reads them
    }
    if (a.early_term || it == a.max_iter) {
      for (int i = tid; i < cb.n_eff * Z; i += nthr) {
        const uint32_t b = __ballot_sync(0xFFFFFFFFu, L[i] < LT(0));
        if ((i & 31) == 0) hb[i >> 5] = b;
      }
      __syncthreads();
      ok = !__syncthreads_or(syndrome_words(s_tab, rows, hb, m, tid, nthr, Z));
      cluster_sync();  // no CTA writes the next iteration into a replica still read for the syndrome
      if ((ok && a.early_term) || it == a.max_iter) break;
    }
  }
  if (rank == 0) {
    const int nw = cb.kb * (Z >> 5);
    for (int i = tid; i < nw; i += nthr) a.bits[cb.bits_off + i] = hb[i];
    if (tid == 0) a.status[a.cb_list[cluster_id_x()]] = it | (ok ? (1 << 16) : 0);
  }
}

template <int C>
const void* cluster_kernel_for(int mode) {
  switch (mode) {
    case LDPC_F32: return reinterpret_cast<const void*>(&oms_cluster_kernel<float, float, false, C>);
    case LDPC_I8: return reinterpret_cast<const void*>(&oms_cluster_kernel<int8_t, uint8_t, true, C>);
    default: return reinterpret_cast<const void*>(&oms_cluster_kernel<int16_t, uint16_t, true, C>);
  }
}

}  // namespace

cudaError_t launch_cluster_decode(int mode, int C, int n_clusters, int block, int smem, cudaStream_t st,
                                  const ClusterArgs& a) {
  if (n_clusters == 0) return cudaSuccess;
  const void* fn = C == 2 ? cluster_kernel_for<2>(mode) : cluster_kernel_for<4>(mode);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(static_cast<unsigned>(n_clusters * C));
  cfg.blockDim = dim3(static_cast<unsigned>(block));
  cfg.dynamicSmemBytes = static_cast<size_t>(smem);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = static_cast<unsigned>(C);
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  void* args[] = {const_cast<ClusterArgs*>(&a)};
  return cudaLaunchKernelExC(&cfg, fn, args);
}

}  // namespace ldpcgb
