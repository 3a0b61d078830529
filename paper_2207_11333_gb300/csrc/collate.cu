// Device-side batch collation: the disjoint union of a batch of graphs read
// from the packed store (global arrays, Sec. 4 Table 1), as the destination-
// sorted CSR the aggregation kernels consume.
//
//   collate_scan_kernel   one block: per-graph node/edge counts, exclusive
//                         scans -> node_off, edge_off, totals, targets
//   collate_graph_kernel  one warp per graph: atom types, graph ids, in-degree
//                         count (shared atomics), warp scan -> row_ptr, then a
//                         rank sort of the graph's edges by (destination,
//                         source, store order) -> col, and the reverse-edge
//                         slot -> rev; degree scalers from a table; the
//                         edges' bond features follow them to their slots
//   collate_small_kernel  both in one launch for batches of at most
//                         kFusedGraphs graphs: every block scans the counts
//                         of all the batch's graphs itself (reading only the
//                         store and the id list, before its dependency wait),
//                         then collates its own graphs as above
//
// Results are bit-identical to a sequential stable sort by (dst, src): every
// position is computed from counts, never from the order of atomics.
#include "kernels.cuh"

namespace gcnn {
namespace {

constexpr int kScanThreads = 1024;
constexpr int kGraphWarps = 8;

__global__ void __launch_bounds__(kScanThreads)
collate_scan_kernel(int G, const int64_t *__restrict__ ids, StoreView st, BatchBuf b, int cap_nodes,
                    int cap_edges, unsigned *err) {
  __shared__ int warp_n[32], warp_e[32];
  __shared__ int carry_n, carry_e;
  pdl_entry(GCNN_K_COLLATE_SCAN);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x == 0) { carry_n = 0; carry_e = 0; }
  __syncthreads();
  for (int base = 0; base < G; base += kScanThreads) {
    const int g = base + threadIdx.x;
    int n = 0, e = 0;
    if (g < G) {
      const int64_t id = ids ? ids[g] : (int64_t)g;
      n = (int)(st.node_ptr[id + 1] - st.node_ptr[id]);
      e = (int)(st.edge_ptr[id + 1] - st.edge_ptr[id]);
      b.y[g] = st.y[id];
    }
    int sn = n, se = e;  // inclusive warp scans
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int tn = __shfl_up_sync(0xffffffffu, sn, o);
      const int te = __shfl_up_sync(0xffffffffu, se, o);
      if (lane >= o) { sn += tn; se += te; }
    }
    if (lane == 31) { warp_n[w] = sn; warp_e[w] = se; }
    __syncthreads();
    if (w == 0) {
      const int vn = warp_n[lane], ve = warp_e[lane];
      int in = vn, ie = ve;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int tn = __shfl_up_sync(0xffffffffu, in, o);
        const int te = __shfl_up_sync(0xffffffffu, ie, o);
        if (lane >= o) { in += tn; ie += te; }
      }
      warp_n[lane] = in - vn;
      warp_e[lane] = ie - ve;
    }
    __syncthreads();
    const int ex_n = carry_n + warp_n[w] + sn - n;
    const int ex_e = carry_e + warp_e[w] + se - e;
    if (g < G) { b.node_off[g] = ex_n; b.edge_off[g] = ex_e; }
    __syncthreads();
    if (threadIdx.x == kScanThreads - 1) { carry_n = ex_n + n; carry_e = ex_e + e; }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    b.node_off[G] = carry_n;
    b.edge_off[G] = carry_e;
    b.dims[0] = G;
    b.dims[1] = carry_n;
    b.dims[2] = carry_e;
    b.dims[3] = 0;
    if (carry_n > cap_nodes || carry_e > cap_edges) {
      atomicOr(err, kErrCapacity);
    } else {
      b.row_ptr[carry_n] = carry_e;
    }
  }
}

// Collation of graph g (store id `id`) by one warp w of the block: its
// atoms start at batch node noff and its edges at batch edge slot eoff.
__device__ __forceinline__ void collate_one(int w, int lane, int g, int64_t id, int noff, int eoff, const StoreView &st,
                                            const BatchBuf &b, const float *__restrict__ scal_tab, int cap_nodes,
                                            int cap_edges, unsigned *err, uint8_t (*s_src)[kMaxGraphEdges],
                                            uint8_t (*s_dst)[kMaxGraphEdges], int (*s_cnt)[256],
                                            int (*s_start)[256]) {
  const int64_t np0 = st.node_ptr[id], ep0 = st.edge_ptr[id];
  const int n = (int)(st.node_ptr[id + 1] - np0);
  const int e = (int)(st.edge_ptr[id + 1] - ep0);
  if (n < 0 || n > kMaxGraphNodes || e < 0 || e > kMaxGraphEdges || noff < 0 || eoff < 0 ||
      noff + n > cap_nodes || eoff + e > cap_edges) {
    if (lane == 0) atomicOr(err, kErrCollateRange);
    return;
  }
  for (int v = lane; v < 256; v += 32) s_cnt[w][v] = 0;
  __syncwarp();
  for (int v = lane; v < n; v += 32) {
    b.types[noff + v] = st.types[np0 + v];
    b.graph_id[noff + v] = g;
    if (b.ynode) b.ynode[noff + v] = st.ynode[np0 + v];
  }
  bool bad = false;
  for (int k = lane; k < e; k += 32) {
    int s = st.edges[2 * (ep0 + k)], d = st.edges[2 * (ep0 + k) + 1];
    if (s >= n || d >= n) { bad = true; s = 0; d = 0; }
    s_src[w][k] = (uint8_t)s;
    s_dst[w][k] = (uint8_t)d;
    atomicAdd(&s_cnt[w][d], 1);
  }
  if (__any_sync(0xffffffffu, bad)) {
    if (lane == 0) atomicOr(err, kErrCollateRange);
    return;
  }
  __syncwarp();
  // exclusive scan of the in-degree counts, 8 entries per lane
  int loc[8], tot = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) { loc[q] = s_cnt[w][lane * 8 + q]; tot += loc[q]; }
  int incl = tot;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  int run = incl - tot;
#pragma unroll
  for (int q = 0; q < 8; ++q) { s_start[w][lane * 8 + q] = run; run += loc[q]; }
  __syncwarp();
  for (int v = lane; v < n; v += 32) {
    const int d = s_cnt[w][v];
    b.row_ptr[noff + v] = eoff + s_start[w][v];
    b.deg[noff + v] = d;
    b.amp[noff + v] = scal_tab[2 * d];
    b.att[noff + v] = scal_tab[2 * d + 1];
  }
  // rank of each edge inside its destination row: by source, then store order
  for (int k = lane; k < e; k += 32) {
    const int s = s_src[w][k], d = s_dst[w][k];
    int rank = 0, rrank = 0, has_rev = 0;
    for (int q = 0; q < e; ++q) {
      const int sq = s_src[w][q], dq = s_dst[w][q];
      rank += (dq == d) & ((sq < s) | ((sq == s) & (q < k)));
      rrank += (dq == s) & (sq < d);
      has_rev |= (dq == s) & (sq == d);
    }
    const int pos = eoff + s_start[w][d] + rank;
    b.col[pos] = noff + s;
    b.rev[pos] = has_rev ? eoff + s_start[w][s] + rrank : -1;
    for (int f = 0; f < st.F; ++f) b.eattr[(size_t)pos * b.eattr_ld + f] = st.eattr[(ep0 + k) * st.F + f];
  }
}

__global__ void __launch_bounds__(kGraphWarps * 32)
collate_graph_kernel(int G, const int64_t *__restrict__ ids, StoreView st, BatchBuf b,
                     const float *__restrict__ scal_tab, int cap_nodes, int cap_edges,
                     unsigned *err) {
  __shared__ uint8_t s_src[kGraphWarps][kMaxGraphEdges];
  __shared__ uint8_t s_dst[kGraphWarps][kMaxGraphEdges];
  __shared__ int s_cnt[kGraphWarps][256];
  __shared__ int s_start[kGraphWarps][256];
  pdl_entry(GCNN_K_COLLATE_GRAPH);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = blockIdx.x * kGraphWarps + w;
  if (g >= G) return;  // warp-uniform; only warp-level synchronisation below
  const int64_t id = ids ? ids[g] : (int64_t)g;
  collate_one(w, lane, g, id, b.node_off[g], b.edge_off[g], st, b, scal_tab, cap_nodes, cap_edges, err, s_src, s_dst,
              s_cnt, s_start);
}

// Batches of at most kFusedGraphs graphs in one launch.  Every block scans
// the node and edge counts of the whole batch (chunks of its 256 threads: the
// same exclusive prefix sums as collate_scan_kernel, integer adds, so the
// same offsets) before its dependency wait, since it reads only the store and
// the id list; then it writes the scan's outputs for its own graphs (block 0
// also the totals and the device-side sizes) and collates them.
constexpr int kFusedGraphs = kCollateOneLaunchGraphs;

__global__ void __launch_bounds__(kGraphWarps * 32)
collate_small_kernel(int G, const int64_t *__restrict__ ids, StoreView st, BatchBuf b,
                     const float *__restrict__ scal_tab, int cap_nodes, int cap_edges, unsigned *err) {
  __shared__ uint8_t s_src[kGraphWarps][kMaxGraphEdges];
  __shared__ uint8_t s_dst[kGraphWarps][kMaxGraphEdges];
  __shared__ int s_cnt[kGraphWarps][256];
  __shared__ int s_start[kGraphWarps][256];
  __shared__ int warp_n[kGraphWarps], warp_e[kGraphWarps], off_n[kGraphWarps], off_e[kGraphWarps];
  __shared__ int carry_n, carry_e;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int base = blockIdx.x * kGraphWarps;
  if (threadIdx.x == 0) { carry_n = 0; carry_e = 0; }
  __syncthreads();
  for (int c0 = 0; c0 < G; c0 += kGraphWarps * 32) {
    const int q = c0 + (int)threadIdx.x;
    int n = 0, e = 0;
    if (q < G) {
      const int64_t id = ids ? ids[q] : (int64_t)q;
      n = (int)(st.node_ptr[id + 1] - st.node_ptr[id]);
      e = (int)(st.edge_ptr[id + 1] - st.edge_ptr[id]);
    }
    int sn = n, se = e;  // inclusive warp scans
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int tn = __shfl_up_sync(0xffffffffu, sn, o);
      const int te = __shfl_up_sync(0xffffffffu, se, o);
      if (lane >= o) { sn += tn; se += te; }
    }
    if (lane == 31) { warp_n[w] = sn; warp_e[w] = se; }
    __syncthreads();
    if (w == 0) {
      const int vn = lane < kGraphWarps ? warp_n[lane] : 0, ve = lane < kGraphWarps ? warp_e[lane] : 0;
      int in = vn, ie = ve;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int tn = __shfl_up_sync(0xffffffffu, in, o);
        const int te = __shfl_up_sync(0xffffffffu, ie, o);
        if (lane >= o) { in += tn; ie += te; }
      }
      if (lane < kGraphWarps) { warp_n[lane] = in - vn; warp_e[lane] = ie - ve; }
    }
    __syncthreads();
    const int ex_n = carry_n + warp_n[w] + sn - n;
    const int ex_e = carry_e + warp_e[w] + se - e;
    if (q >= base && q < base + kGraphWarps) { off_n[q - base] = ex_n; off_e[q - base] = ex_e; }
    __syncthreads();
    if (threadIdx.x == kGraphWarps * 32 - 1) { carry_n = ex_n + n; carry_e = ex_e + e; }
    __syncthreads();
  }
  pdl_entry(GCNN_K_COLLATE);
  const int g = base + w;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    b.node_off[G] = carry_n;
    b.edge_off[G] = carry_e;
    b.dims[0] = G;
    b.dims[1] = carry_n;
    b.dims[2] = carry_e;
    b.dims[3] = 0;
    if (carry_n > cap_nodes || carry_e > cap_edges) atomicOr(err, kErrCapacity);
    else b.row_ptr[carry_n] = carry_e;
  }
  if (g >= G) return;  // warp-uniform; only warp-level synchronisation below
  const int64_t id = ids ? ids[g] : (int64_t)g;
  if (lane == 0) {
    b.node_off[g] = off_n[w];
    b.edge_off[g] = off_e[w];
    b.y[g] = st.y[id];
  }
  if (carry_n > cap_nodes || carry_e > cap_edges) return;
  collate_one(w, lane, g, id, off_n[w], off_e[w], st, b, scal_tab, cap_nodes, cap_edges, err, s_src, s_dst, s_cnt,
              s_start);
}

}  // namespace

int launch_collate(int G, const int64_t *ids, StoreView st, BatchBuf b, const float *scal_tab,
                   int cap_nodes, int cap_edges, unsigned *err, cudaStream_t s) {
  if (G < 0) return set_error(GCNN_EINVAL, "collate: negative graph count");
  if (G > 0 && G <= kFusedGraphs) {
    GCNN_TRY(launch(collate_small_kernel, ceil_div(G, kGraphWarps), kGraphWarps * 32, 0, s, G, ids, st, b, scal_tab,
                    cap_nodes, cap_edges, err));
    return GCNN_OK;
  }
  GCNN_TRY(launch(collate_scan_kernel, 1, kScanThreads, 0, s, G, ids, st, b, cap_nodes, cap_edges, err));
  if (G > 0)
    GCNN_TRY(launch(collate_graph_kernel, ceil_div(G, kGraphWarps), kGraphWarps * 32, 0, s, G, ids, st, b, scal_tab,
                    cap_nodes, cap_edges, err));
  return GCNN_OK;
}

int collate_node_kind(const void *func) {
  if (func == reinterpret_cast<const void *>(collate_scan_kernel)) return 1;
  if (func == reinterpret_cast<const void *>(collate_graph_kernel)) return 2;
  if (func == reinterpret_cast<const void *>(collate_small_kernel)) return 3;
  return 0;
}

int collate_set_nodes(cudaGraphExec_t exec, cudaGraphNode_t scan_node, cudaGraphNode_t graph_node, int G,
                      const int64_t *ids, StoreView st, BatchBuf b, const float *scal_tab, int cap_nodes,
                      int cap_edges, unsigned *err) {
  if (G <= 0) return set_error(GCNN_EINVAL, "collate: a captured collation needs at least one graph");
  cudaKernelNodeParams p{};
  if (G <= kFusedGraphs) {  // one node: the batch's single collation launch
    void *args[] = {&G, &ids, &st, &b, &scal_tab, &cap_nodes, &cap_edges, &err};
    p.func = reinterpret_cast<void *>(collate_small_kernel);
    p.gridDim = dim3(ceil_div(G, kGraphWarps));
    p.blockDim = dim3(kGraphWarps * 32);
    p.kernelParams = args;
    GCNN_CUDA_TRY(cudaGraphExecKernelNodeSetParams(exec, scan_node, &p));
    return GCNN_OK;
  }
  void *scan_args[] = {&G, &ids, &st, &b, &cap_nodes, &cap_edges, &err};
  p.func = reinterpret_cast<void *>(collate_scan_kernel);
  p.gridDim = dim3(1);
  p.blockDim = dim3(kScanThreads);
  p.kernelParams = scan_args;
  GCNN_CUDA_TRY(cudaGraphExecKernelNodeSetParams(exec, scan_node, &p));
  void *graph_args[] = {&G, &ids, &st, &b, &scal_tab, &cap_nodes, &cap_edges, &err};
  p.func = reinterpret_cast<void *>(collate_graph_kernel);
  p.gridDim = dim3(ceil_div(G, kGraphWarps));
  p.blockDim = dim3(kGraphWarps * 32);
  p.kernelParams = graph_args;
  GCNN_CUDA_TRY(cudaGraphExecKernelNodeSetParams(exec, graph_node, &p));
  return GCNN_OK;
}

GCNN_TIMELINE_ATTACH(collate)

}  // namespace gcnn
