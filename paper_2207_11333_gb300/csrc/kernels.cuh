// Launchers of the library's CUDA kernels (one group per source file).
#pragma once

#include "common.cuh"

namespace gcnn {

// ---------------------------------------------------------------- collate.cu
// Read view of a packed store (global arrays), host- or device-resident.
struct StoreView {
  const int64_t *node_ptr;  // [G+1]
  const int64_t *edge_ptr;  // [G+1]
  const uint8_t *types;     // [N]
  const uint8_t *edges;     // [2E] local (src, dst)
  const float *y;           // [G]
  const float *eattr;       // [E][F] bond features (F = 0: nullptr)
  int F;
  const float *ynode;       // [N] node-level targets or nullptr
};

// Writable batch arrays in the context arena.
struct BatchBuf {
  int *node_off, *edge_off, *graph_id, *row_ptr, *col, *rev, *deg;
  float *amp, *att, *y;
  uint8_t *types;
  int *dims;  // {G, N, E, 0}
  float *eattr;  // [E][eattr_ld] bond features in slot order (F = 0: unused)
  int eattr_ld;  // row stride: F rounded up to a multiple of 4 (16-byte rows)
  float *ynode;  // [N] node-level targets (node head only, else nullptr)
};

// Collate graphs ids[0..G) (ids == nullptr: graphs 0..G-1) of `st`.
// scal_tab[2*d], scal_tab[2*d+1] = amplification / attenuation of degree d
// (d = 0..kMaxGraphEdges).
int launch_collate(int G, const int64_t *ids, StoreView st, BatchBuf b, const float *scal_tab,
                   int cap_nodes, int cap_edges, unsigned *err, cudaStream_t s);
// For a collation captured in a CUDA graph: 1 or 2 when `func` is the kernel
// of its scan or its per-graph launch, 3 for the single launch of a batch of
// at most 1024 graphs (0 otherwise); and the update of those nodes of an
// instantiated graph (scan_node: the scan or the single launch; graph_node:
// the per-graph launch, unused for a single launch) to the arguments of
// another batch of the same graph count G.
constexpr int kCollateOneLaunchGraphs = 1024;  // batches up to this size: one collation launch
int collate_node_kind(const void *func);
int collate_set_nodes(cudaGraphExec_t exec, cudaGraphNode_t scan_node, cudaGraphNode_t graph_node, int G,
                      const int64_t *ids, StoreView st, BatchBuf b, const float *scal_tab, int cap_nodes,
                      int cap_edges, unsigned *err);

// ---------------------------------------------------------------- aggregate.cu
// agg[i] = [sum, mean, min, max, std](P_i + Q_j, j in N(i)); PQ is N x 2H.
// agg is nullable; S16 (nullable, row pitch ld16) receives [agg, amp*agg,
// att*agg] (15H BF16), the scaled aggregates as the BF16 operand of the
// update GEMM.
// With F > 0 the message carries the bond term sum_f eattr[e][f] wE[f]
// (eattr: E rows of stride round_up(F, 4) in slot order, wE: F x H).
// idx_early: the sizes in dims, the CSR arrays and the degree scalers were
// written at least two launches before this one on the stream (the model's
// own launch sequences after the collator), so the kernels read them before
// their dependency wait; false for arrays a caller may just have written.
int launch_aggregate_fwd(int n_nodes, int H, DevDims dims, const int *row_ptr, const int *col,
                         const float *PQ, float *agg, float eps, unsigned *err, cudaStream_t s,
                         uint16_t *S16 = nullptr, int ld16 = 0, const float *amp = nullptr,
                         const float *att = nullptr, const float *eattr = nullptr, const float *wE = nullptr,
                         int F = 0, bool idx_early = false);
// dPQ from dagg; scratch is E x H (per-edge message gradients).  With agg
// null the forward's statistics are recomputed from the messages in the
// forward kernel's order (bit-identical).
int launch_aggregate_bwd(int n_nodes, int n_edges, int H, DevDims dims, const int *row_ptr,
                         const int *col, const int *rev, const float *PQ, const float *agg,
                         const float *dagg, float *dPQ, float *scratch, float eps, unsigned *err,
                         cudaStream_t s, uint16_t *dPQ16 = nullptr, int ld16 = 0, const float *eattr = nullptr,
                         const float *wE = nullptr, int F = 0, bool idx_early = false);

// The same gradient for a batch of whole graphs (node_off: G + 1 offsets;
// no edge leaves its graph).  Batches of at least 2 x SMs x 128 edges take the
// fused kernel: chunks of graphs of about 128 edges, each handled by one block
// that keeps its per-edge gradients in shared memory; `chunks` holds
// aggregate_chunk_capacity(n_edges) ints.  Smaller batches, and batches
// with bond features (whose weight gradient reads the per-edge gradients in
// scratch), take the edge + gather pair above.  Same result either way, bitwise.
// make_chunks = false reuses the partition that a previous call on the same
// batch and sizes wrote to `chunks`.
int launch_aggregate_bwd_graphs(int n_graphs, int n_nodes, int n_edges, int H, DevDims dims, const int *node_off,
                                const int *row_ptr, const int *col, const int *rev, const float *PQ,
                                const float *agg, const float *dagg, float *dPQ, float *scratch, int *chunks,
                                float eps, unsigned *err, cudaStream_t s, uint16_t *dPQ16 = nullptr, int ld16 = 0,
                                const float *eattr = nullptr, const float *wE = nullptr, int F = 0,
                                bool make_chunks = true, bool idx_early = false);
int aggregate_chunk_capacity(int n_edges);
// Bond rows' gradient out[f][c] (F x H) = sum over edge slots of eattr[r][f]
// (row stride ld) times dm[r][c] (E x H, the per-edge message gradients at
// reverse slots); fixed-order sums.
int launch_bond_grad(int n_edges, int H, int F, int ld, DevDims dims, const float *eattr, const float *dm, float *out,
                     cudaStream_t s);
bool aggregate_bwd_uses_fused(int n_edges);

// ---------------------------------------------------------------- small.cu
int launch_embed(int n_nodes, int H, DevDims dims, const uint8_t *types, const float *emb,
                 int n_types, float *x0, cudaStream_t s, uint16_t *x0_16 = nullptr, int ld16 = 0);
// dEmb[t] = sum of dx0 over nodes of type t (fixed-order sum, one launch).
int launch_embed_bwd(int n_nodes, int H, DevDims dims, const uint8_t *types, const float *dx0, int n_types,
                     float *demb, cudaStream_t s);
int launch_pool_fwd(int G, int H, DevDims dims, const int *node_off, const float *x, float *pooled,
                    cudaStream_t s);
// D3 (nullable, row pitch ld3) additionally receives [amp*g, att*g, g] (3H
// BF16) with g = dx * [h > 0], the masked, degree-scaled gradient of the last layer.
int launch_pool_bwd(int G, int n_nodes, int H, DevDims dims, const int *node_off,
                    const int *graph_id, const float *dpooled, float *dx, cudaStream_t s,
                    uint16_t *D3 = nullptr, int ld3 = 0, const float *h = nullptr, const float *amp = nullptr,
                    const float *att = nullptr);

// Per-graph part of the head (one block per graph): forward = mean pooling,
// z1 = g W1 + b1, pred = ReLU(z1) . w2 + b2; backward = dpred (dpred_in, or
// the MSE gradient 2 (pred - y) / G), dz1, dg = W1 dz1 and the pooling
// gradient on the graph's nodes (plus D3 as in launch_pool_bwd).
struct HeadArgs {
  int g_cap, H, Hh, rk;  // rk is set by the launcher
  DevDims dims;
  const int *node_off;
  const float *x;
  const float *w1, *b1, *w2, *b2;
  float *pooled, *z1, *pred;
  const float *y, *dpred_in;
  float *dpred, *dz1, *dg, *dx;
  uint16_t *D3;
  int ld3;
  const float *h, *amp, *att;
  const float *dx_add;  // nullable: N x H added to the pooling gradient (node-level head)
  const float *loss_scale;  // nullable: device scalar multiplying dL/dyhat of the MSE (1 when null)
};
int launch_head_graph(HeadArgs a, bool fwd, bool bwd, cudaStream_t s);
// Node-level head on the last layer's atoms (zn = x W1n + b1n from a GEMM):
// pred_n = ReLU(zn) . w2n + b2n per atom; with train, dpred_n = weight * 2
// (pred_n - y_n) / N and dzn = [zn > 0] dpred_n w2n.
struct NodeHeadArgs {
  int n_cap, Hh;
  DevDims dims;
  const float *zn, *w2n, *b2n, *y;
  float *pred, *dpred, *dzn;
  float weight;
  const float *loss_scale;  // nullable: device scalar multiplying the node-level loss gradient
};
int launch_node_pred(const NodeHeadArgs &a, bool train, cudaStream_t s);
// Node head gradients of w2n (Hh) and b2n (1) into grad_w2n[0 .. Hh], summed
// over atoms in a fixed order, and the FP64 loss sums (squared error, count)
// into loss_accum (nullable) as entries 3 and 4.
int launch_node_grad(const NodeHeadArgs &a, float *grad_w2n, double *loss_accum, cudaStream_t s);
// Head parameter gradients (w1, b1, w2, b2, contiguous in layout order) summed
// over the batch's graphs, and the FP64 loss sums into loss_accum (nullable).
struct HeadGradArgs {
  int g_cap, H, Hh;
  DevDims dims;
  const float *pooled, *z1, *dz1, *dpred, *pred, *y;
  float *grad;
  double *loss_accum;
};
int launch_head_grad(const HeadGradArgs &a, cudaStream_t s);

// AdamW over the parameters [b0, b0 + n0) and [b1, b1 + n1) of the flat
// arrays (b0, n0 and b1 multiples of 4; n1 any).  state[0] is the step
// counter: every launch uses the bias corrections of step state[0] + 1, and a
// launch with `advance` set (the last of a step; ticket a zero-initialised
// device word) moves it on once all its blocks are done.  With wb non-null the
// updated parameters are also written as BF16 (flat copy wb, and the packed
// backward operands wpack of every layer when non-null).  max_blocks caps the
// grid (0: up to 8 blocks per SM).
struct AdamPack {
  int H, L;
  long long layers_begin, layer_size;
};
struct AdamSpan {
  long long b0, n0, b1, n1;
};
int launch_adam(AdamSpan span, bool advance, int max_blocks, float *param, const float *grad, float *m, float *v,
                int *state, unsigned *ticket, const float *lr, double beta1, double beta2, float eps, float wd,
                uint16_t *wb, uint16_t *wpack, AdamPack pk, cudaStream_t s);

// ---------------------------------------------------------------- gemm_simt.cu
// C = op(A) . op(B) in FP32 on CUDA cores (FFMA), with operands assembled on
// the fly from up to kMaxSeg segments along the feature dimension (each with
// an optional per-node scale and an optional ReLU mask), optional bias and
// ReLU in the epilogue, and split-K with a deterministic reduction.
constexpr int kMaxSeg = 5;

struct Seg {
  int begin;              // first feature index of the segment
  const float *ptr;       // nullptr: the constant 1
  int ld;                 // leading dimension of ptr (and of mask)
  const float *rowscale;  // per-node factor or nullptr
  const float *mask;      // element kept iff mask > 0, or nullptr
};

struct Operand {
  Seg seg[kMaxSeg];
  int nseg;
};

// Which GEMM dimension runs over the batch's nodes, so that its extent is
// read from the device-side batch sizes (DevDims)
enum NodeDim { kNodeNone = 0, kNodeM = 1, kNodeK = 2 };

struct GemmDesc {
  int M, N, K;          // K: capacity when node_dim == kNodeK
  NodeDim node_dim;
  // A is M x K: a_kcontig -> A(m,k) = seg.ptr[m*ld + k - begin] (segments along K)
  //             else       -> A(m,k) = seg.ptr[k*ld + m - begin] (segments along M)
  bool a_kcontig;
  // B is K x N: b_ncontig -> B(k,n) = seg.ptr[(k - begin)*ld + n] (segments along K)
  //             else       -> B(k,n) = seg.ptr[n*ld + k - begin] (segments along K)
  bool b_ncontig;
  Operand A, B;
  float *C;
  int ldc;
  const float *bias;  // bias[n] for n < bias_n
  int bias_n;
  bool relu;
  int last_row_cols;  // > 0: only the first last_row_cols columns of row M-1 are stored
};

struct GemmWorkspace {
  float *partial;      // split-K partial sums
  size_t floats;       // capacity
  int max_splits = 32; // 1: row-invariant (no split-K)
  int max_ctas = 0;    // tensor-core GEMMs: grid limit (0: one CTA per SM), e.g. to share the GPU with a stream
};

int run_gemm_simt(const GemmDesc &d, DevDims dims, const GemmWorkspace &ws, cudaStream_t s);
size_t gemm_simt_workspace_floats(int M, int N, int K);
// C = epilogue(sum over splits of partial[z]) in split order (deterministic).
int run_splitk_reduce(const GemmDesc &d, DevDims dims, const float *partial, int splits, cudaStream_t s);
int num_sms();

// ---------------------------------------------------------------- gemm_tc.cu
// C = A . B on the tensor cores (TMA + tcgen05): BF16 operands stored as
// uint16_t bit patterns, FP32 accumulation in TMEM.  Each operand is one
// row-major BF16 array of `rows` x `cols` with row pitch `ld`:
//   A (M x K): mn_major false -> A(m,k) = ptr[m*ld + k] (rows = M, cols = K)
//              mn_major true  -> A(m,k) = ptr[k*ld + m] (rows = K, cols = M)
//   B (K x N): mn_major false -> B(k,n) = ptr[n*ld + k] (rows = N, cols = K)
//              mn_major true  -> B(k,n) = ptr[k*ld + n] (rows = K, cols = N)
// Reads past cols / rows return zero, so K may be padded up to 64.
struct TcMat {
  const uint16_t *ptr;
  int ld, rows, cols;
  bool mn_major;
};

struct TcEpilogue {
  float *C;            // FP32 result (nullable)
  int ldc;
  const float *bias;   // bias[n] for n < bias_n
  int bias_n;
  bool relu;
  uint16_t *C16;       // BF16 copy of the result (nullable)
  int ld16;
  // [amp*g | att*g | g] as BF16 into D3 (nullable), g = v*[mask > 0]: the
  // ReLU-masked, degree-scaled output gradient used by the next backward GEMMs
  uint16_t *D3;
  int ld3;
  const float *mask;
  int ldm;
  const float *amp, *att;
};

// Operand not written by the kernel launched just before on the same stream:
// its first pipeline stages are loaded before the dependency wait of
// programmatic dependent launch, overlapping the previous kernel's tail.  A
// kernel starts only once its predecessor has passed its own wait, so every
// earlier kernel is complete by then; only the immediate predecessor's
// outputs must wait.
enum TcStable { kStableNone = 0, kStableA = 1, kStableB = 2 };

struct TcDesc {
  int M, N, K;         // K: multiple of 64 (padded) or, with node_dim == kNodeK, the node capacity
  NodeDim node_dim;
  TcMat A, B;
  TcEpilogue ep;
  TcStable stable;
  // at most 80 registers per thread (the weight-gradient GEMMs beside the
  // aggregation backward); ignored with the masked-gradient epilogue
  bool lean;
};

int run_gemm_tc(const TcDesc &d, DevDims dims, const GemmWorkspace &ws, unsigned *err, cudaStream_t s);
// CTA limit of the weight-gradient GEMMs, which run on the backward's second
// stream beside the data-gradient chain (the same limit in the serial backward,
// so that both pick the same plans)
int side_gemm_ctas();
size_t gemm_tc_workspace_floats(int M, int N, int K);
// Timing study of the training step's BF16 GEMM shapes (gcnn_gemm_study).
int gemm_tc_study(int n_atoms, int H, int mode, double *rows, int max_rows, int *n_rows);
// dst[i] = bf16(src[i]) (round to nearest even)
int launch_cast_bf16(int64_t n, const float *src, uint16_t *dst, cudaStream_t s);
// BF16 weight layouts of one layer for the backward GEMMs (see gemm_tc.cu)
int launch_pack_layer(int H, const float *msg_w, const float *upd_w, uint16_t *Wd, uint16_t *Wx, cudaStream_t s);
// Column sums over the batch's nodes of [a0 * [mask > 0] | a1] (cols0 + cols1
// columns, each a multiple of 4; mask and a1 nullable) into out0[cols0] and
// out1[cols1]; fixed-order sum, one launch.
int launch_colsum2(int n_cap, int cols0, int cols1, DevDims dims, const float *a0, int ld0, const float *mask,
                   int ldm, const float *a1, int ld1, float *out0, float *out1, cudaStream_t s);

// Timeline marker after a train step: records the end of the step's last kernel.
int launch_step_end(cudaStream_t s);

// FP32 FFMA throughput probe over every SM; *flop receives the launch's FLOP.
int launch_ffma_peak(int iters, float *out, cudaStream_t s, double *flop);

// Point the kernels of each translation unit at the timeline buffer (or null).
int timeline_attach_collate(void *tl);
int timeline_attach_aggregate(void *tl);
int timeline_attach_small(void *tl);
int timeline_attach_gemm_simt(void *tl);
int timeline_attach_gemm_tc(void *tl);

}  // namespace gcnn
