// The training step: forward (Sec. 3.2, Fig. 3: GC layers -> global mean
// pooling -> FC layers -> MSE), the hand-written backward and the AdamW step,
// as an ordered sequence of kernel launches on the context's stream.  Every
// launch reads the batch's true sizes from the device ({G, N, E} written by
// the collator), so one sequence captured in a CUDA graph serves every batch
// whose sizes fit its grid.
#include "context.h"

namespace gcnn {
namespace {

struct LayerW {
  float *msg_w, *msg_b, *upd_w, *upd_b;
  float *edge_w;  // bond rows of W_M (F x H), after the head; nullptr when F = 0
};

LayerW layer_ptrs(float *base, const gcnn_ctx *c, int l) {
  float *b = base + (int64_t)c->T * c->H + (int64_t)l * c->layer_size;
  const int64_t H = c->H, F = c->cfg.edge_features;
  // bond rows: after the head, from the next multiple of 4 floats (16-byte aligned)
  const int64_t bonds = ((int64_t)c->T * H + (int64_t)c->L * c->layer_size + H * c->Hh + 2 * c->Hh + 1 + 3) / 4 * 4;
  float *e = F > 0 ? base + bonds + l * F * H : nullptr;
  return LayerW{b, b + 2 * H * H, b + 2 * H * H + H, b + 2 * H * H + H + 16 * H * H, e};
}


float *head_ptr(float *base, const gcnn_ctx *c) {
  return base + (int64_t)c->T * c->H + (int64_t)c->L * c->layer_size;
}

// node-level head w1n[H][Hh], b1n[Hh], w2n[Hh], b2n: after the bond rows (or
// the graph head), from the next multiple of 4 floats
float *node_head_ptr(float *base, const gcnn_ctx *c) {
  const int64_t H = c->H, F = c->cfg.edge_features;
  const int64_t head_end = (int64_t)c->T * H + (int64_t)c->L * c->layer_size + H * c->Hh + 2 * c->Hh + 1;
  const int64_t trunk = F == 0 ? head_end : (head_end + 3) / 4 * 4 + (int64_t)c->L * F * H;
  return base + (trunk + 3) / 4 * 4;
}

Seg seg(int begin, const float *ptr, int ld, const float *rowscale = nullptr,
        const float *mask = nullptr) {
  return Seg{begin, ptr, ld, rowscale, mask};
}

GemmDesc blank() {
  GemmDesc d{};
  d.last_row_cols = 0;
  d.bias = nullptr;
  d.relu = false;
  return d;
}

float *xs_at(const gcnn_ctx *c, int l) { return c->xs + (size_t)l * c->Nc * c->H; }
float *pq_at(const gcnn_ctx *c, int l) { return c->PQ + (size_t)l * c->Nc * 2 * c->H; }
// FP32 aggregates of layer l; the BF16 path keeps none (its backward
// recomputes the statistics from the messages)
float *agg_at(const gcnn_ctx *c, int l) {
  if (!c->agg) return nullptr;
  return c->agg + (c->cfg.recompute ? 0 : (size_t)l * c->Nc * kAgg * c->H);
}

bool bf16(const gcnn_ctx *c);

// Arguments of the per-graph head kernel; its pooling gradient goes to dH
// (and, with BF16 GEMMs, to the masked and scaled operand block G5[0]).
HeadArgs head_args(gcnn_ctx *c, int G, const float *dpred_in) {
  float *hp = head_ptr(c->params, c);
  const int64_t HHh = (int64_t)c->H * c->Hh;
  HeadArgs a{};
  a.g_cap = G; a.H = c->H; a.Hh = c->Hh; a.dims = DevDims{c->bb.dims};
  a.node_off = c->bb.node_off; a.x = xs_at(c, c->L);
  a.w1 = hp; a.b1 = hp + HHh; a.w2 = hp + HHh + c->Hh; a.b2 = hp + HHh + 2 * c->Hh;
  a.pooled = c->pooled; a.z1 = c->z1; a.pred = c->pred;
  a.y = c->bb.y; a.dpred_in = dpred_in;
  a.dpred = c->dpred; a.dz1 = c->dz1; a.dg = c->dg; a.dx = c->dH;
  if (bf16(c)) {
    a.D3 = c->G5[0]; a.ld3 = 5 * c->H;
    a.h = xs_at(c, c->L); a.amp = c->bb.amp; a.att = c->bb.att;
  }
  a.dx_add = c->cfg.node_head ? c->dxn : nullptr;  // formed by the forward (train)
  a.loss_scale = c->loss_scale;
  return a;
}

NodeHeadArgs node_args(gcnn_ctx *c, int Ngrid) {
  const float *w = node_head_ptr(c->params, c);
  const int64_t HHh = (int64_t)c->H * c->Hh;
  NodeHeadArgs a{};
  a.n_cap = Ngrid; a.Hh = c->Hh; a.dims = DevDims{c->bb.dims};
  a.zn = c->zn; a.w2n = w + HHh + c->Hh; a.b2n = w + HHh + 2 * c->Hh; a.y = c->bb.ynode;
  a.pred = c->predn; a.dpred = c->dpredn; a.dzn = c->dzn;
  a.weight = (float)c->cfg.node_loss_weight;
  a.loss_scale = c->loss_scale + 1;
  return a;
}

// Record that the gradients of bucket k (layer k, or every gradient for
// k = L) are final once the work queued so far on stream s has run, for
// callers that start their exchange of a bucket early (gcnn_grad_wait).  In a
// captured forward + backward the record is an external event node of the
// graph; a captured train step runs AdamW itself and records nothing.
int mark_grads_ready(gcnn_ctx *c, int k, cudaStream_t s) {
  if (k < 0 || k >= (int)c->grad_ev.size()) return GCNN_OK;
  if (c->capturing) {
    if (c->cap_grad_events) GCNN_CUDA_TRY(cudaEventRecordWithFlags(c->grad_ev[k], s, cudaEventRecordExternal));
    return GCNN_OK;
  }
  GCNN_CUDA_TRY(cudaEventRecord(c->grad_ev[k], s));
  return GCNN_OK;
}

int gemm(gcnn_ctx *c, const GemmDesc &d) {
  PhaseScope ps(c, GCNN_PHASE_GEMM);
  return run_gemm_simt(d, DevDims{c->bb.dims}, c->ws, c->stream);
}

// Bond rows' gradient: dW_E = eattr^T dm over the batch's edges.  dm holds
// each edge's message gradient at its reverse slot, and both directions of a
// bond carry the same features (checked when the store is opened), so slot r
// pairs dm[r] with eattr[r].
int gemm_bond_rows(gcnn_ctx *c, int Egrid, float *g_edge_w) {
  PhaseScope ps(c, GCNN_PHASE_AGG_BWD);
  return launch_bond_grad(Egrid, c->H, c->cfg.edge_features, c->bb.eattr_ld, DevDims{c->bb.dims}, c->bb.eattr, c->dm,
                          g_edge_w, c->stream);
}

// Node-level head forward on the last layer (zn = x W1n + b1n, then the
// per-atom output); with train also its loss gradient and dxn = dzn W1n^T,
// which the graph head's backward adds to the pooling gradient.
int node_head_forward(gcnn_ctx *c, int Ngrid, bool train) {
  const int H = c->H, Hh = c->Hh;
  const float *w = node_head_ptr(c->params, c);
  {
    GemmDesc d = blank();
    d.M = Ngrid; d.N = Hh; d.K = H; d.node_dim = kNodeM;
    d.a_kcontig = true; d.b_ncontig = true;
    d.A.nseg = 1; d.A.seg[0] = seg(0, xs_at(c, c->L), H);
    d.B.nseg = 1; d.B.seg[0] = seg(0, w, Hh);
    d.C = c->zn; d.ldc = Hh; d.bias = w + (int64_t)H * Hh; d.bias_n = Hh;
    GCNN_TRY(gemm(c, d));
  }
  {
    PhaseScope ps(c, GCNN_PHASE_HEAD);
    GCNN_TRY(launch_node_pred(node_args(c, Ngrid), train, c->stream));
  }
  if (train) {
    GemmDesc d = blank();
    d.M = Ngrid; d.N = H; d.K = Hh; d.node_dim = kNodeM;
    d.a_kcontig = true; d.b_ncontig = false;
    d.A.nseg = 1; d.A.seg[0] = seg(0, c->dzn, Hh);
    d.B.nseg = 1; d.B.seg[0] = seg(0, w, Hh);
    d.C = c->dxn; d.ldc = H;
    GCNN_TRY(gemm(c, d));
  }
  return GCNN_OK;
}

// Node-level head parameter gradients: [x ; 1]^T dzn -> W1n and b1n, then
// w2n, b2n and the node loss sums.
int node_head_backward(gcnn_ctx *c, int Ngrid, double *loss_accum) {
  const int H = c->H, Hh = c->Hh;
  float *gw = node_head_ptr(c->grads, c);
  GemmDesc d = blank();
  d.M = H + 1; d.N = Hh; d.K = Ngrid; d.node_dim = kNodeK;
  d.a_kcontig = false; d.b_ncontig = true;
  d.A.nseg = 2;
  d.A.seg[0] = seg(0, xs_at(c, c->L), H);
  d.A.seg[1] = seg(H, nullptr, 0);
  d.B.nseg = 1; d.B.seg[0] = seg(0, c->dzn, Hh);
  d.C = gw; d.ldc = Hh;
  GCNN_TRY(gemm(c, d));
  PhaseScope ps(c, GCNN_PHASE_HEAD);
  GCNN_TRY(launch_node_grad(node_args(c, Ngrid), gw + (int64_t)H * Hh + Hh, loss_accum, c->stream));
  return GCNN_OK;
}

int tc(gcnn_ctx *c, const TcDesc &d) {
  PhaseScope ps(c, GCNN_PHASE_GEMM);
  return run_gemm_tc(d, DevDims{c->bb.dims}, c->ws, c->err, c->stream);
}

// The stream (and split-K workspace) of a layer's weight- and bias-gradient
// work: a second stream that overlaps the data-gradient chain, or the main
// stream when the step runs serially.
struct Lane {
  cudaStream_t s;
  const GemmWorkspace *ws;
};

int tc_on(gcnn_ctx *c, const TcDesc &d, Lane lane) {
  PhaseScope ps(c, GCNN_PHASE_GEMM);
  return run_gemm_tc(d, DevDims{c->bb.dims}, *lane.ws, c->err, lane.s);
}

// BF16 backward without recompute overlaps unless asked not to (profiling
// times phases on the main stream, so it runs serially too)
bool overlapped(const gcnn_ctx *c) {
  return c->side && !(c->cfg.flags & GCNN_FLAG_SERIAL) && !c->prof_on && !c->cfg.recompute;
}

bool bf16(const gcnn_ctx *c) { return c->cfg.precision == GCNN_PREC_BF16; }

// In a train step whose BF16 backward overlaps, the AdamW update of layer
// l + 1 runs on a third stream while the main stream works on layer l (layer
// l + 1's gradients and its last use of its weights are then complete), and
// layer 0 with the parameters after the layers runs there beside the
// embedding gradient; the step's final update covers the embedding table.
// AdamW is elementwise, so the result is the same bit for bit.
bool layers_updated_early(const gcnn_ctx *c) { return c->fuse_step && bf16(c) && overlapped(c); }

int adam(gcnn_ctx *c, AdamSpan sp, bool advance, int max_blocks, cudaStream_t s) {
  const AdamPack pk{c->H, c->L, (long long)c->T * c->H, (long long)c->layer_size};
  return launch_adam(sp, advance, max_blocks, c->params, c->grads, c->adam_m, c->adam_v, c->opt_state, c->tickets,
                     c->lr_dev, c->cfg.beta1, c->cfg.beta2, (float)c->cfg.adam_eps,
                     (float)c->cfg.weight_decay, c->wb, c->wpack, pk, s);
}

// BF16 views
// [x_l | scaled aggregates] operand of layer l (one shared buffer with recompute)
uint16_t *U_at(const gcnn_ctx *c, int l) {
  return c->U + (c->cfg.recompute ? 0 : (size_t)l * c->Nc * 16 * c->H);
}
// BF16 layer input x_l: columns [0, H) of U_at(l), or its own buffer with recompute
uint16_t *X_at(const gcnn_ctx *c, int l) {
  return c->cfg.recompute ? c->Xb + (size_t)l * c->Nc * c->H : U_at(c, l);
}
int X_ld(const gcnn_ctx *c) { return c->cfg.recompute ? c->H : 16 * c->H; }

// With recompute, place x_l in the first H columns of the shared U buffer.
int stage_x(gcnn_ctx *c, int Ngrid, int l) {
  if (!c->cfg.recompute) return GCNN_OK;
  const size_t w = (size_t)c->H * sizeof(uint16_t);
  GCNN_CUDA_TRY(cudaMemcpy2DAsync(U_at(c, l), 16 * w, X_at(c, l), w, w, (size_t)Ngrid, cudaMemcpyDeviceToDevice,
                                  c->stream));
  return GCNN_OK;
}
const uint16_t *wb_of(const gcnn_ctx *c, const float *p) { return c->wb + (p - c->params); }
const uint16_t *Wd_at(const gcnn_ctx *c, int l) { return c->wpack + (size_t)l * 18 * c->H * c->H; }
const uint16_t *Wx_at(const gcnn_ctx *c, int l) { return Wd_at(c, l) + (size_t)15 * c->H * c->H; }
int pad64(int k) { return (k + 63) / 64 * 64; }

TcMat mat(const uint16_t *ptr, int ld, int rows, int cols, bool mn_major) {
  return TcMat{ptr, ld, rows, cols, mn_major};
}

TcDesc tblank() {
  TcDesc d{};
  return d;
}

// PQ = x [A | B] + [b_M | 0]    (message layer, both halves at once)
int gemm_message(gcnn_ctx *c, int Ngrid, int l) {
  const int H = c->H;
  LayerW w = layer_ptrs(c->params, c, l);
  GemmDesc d = blank();
  d.M = Ngrid; d.N = 2 * H; d.K = H; d.node_dim = kNodeM;
  d.a_kcontig = true; d.b_ncontig = true;
  d.A.nseg = 1; d.A.seg[0] = seg(0, xs_at(c, l), H);
  d.B.nseg = 1; d.B.seg[0] = seg(0, w.msg_w, 2 * H);
  d.C = pq_at(c, l); d.ldc = 2 * H;
  d.bias = w.msg_b; d.bias_n = H;
  return gemm(c, d);
}

// x' = ReLU([x ; agg ; amp*agg ; att*agg] W_U + b_U)
int gemm_update(gcnn_ctx *c, int Ngrid, int l) {
  const int H = c->H;
  LayerW w = layer_ptrs(c->params, c, l);
  const float *agg = agg_at(c, l);
  GemmDesc d = blank();
  d.M = Ngrid; d.N = H; d.K = 16 * H; d.node_dim = kNodeM;
  d.a_kcontig = true; d.b_ncontig = true;
  d.A.nseg = 4;
  d.A.seg[0] = seg(0, xs_at(c, l), H);
  d.A.seg[1] = seg(H, agg, kAgg * H);
  d.A.seg[2] = seg(6 * H, agg, kAgg * H, c->bb.amp);
  d.A.seg[3] = seg(11 * H, agg, kAgg * H, c->bb.att);
  d.B.nseg = 1; d.B.seg[0] = seg(0, w.upd_w, H);
  d.C = xs_at(c, l + 1); d.ldc = H;
  d.bias = w.upd_b; d.bias_n = H; d.relu = true;
  return gemm(c, d);
}

// BF16: PQ = x [A | B] + [b_M | 0]
int tc_message(gcnn_ctx *c, int Ngrid, int l) {
  const int H = c->H;
  LayerW w = layer_ptrs(c->params, c, l);
  TcDesc d = tblank();
  d.M = Ngrid; d.N = 2 * H; d.K = pad64(H); d.node_dim = kNodeM;
  d.A = mat(X_at(c, l), X_ld(c), Ngrid, H, false);
  d.B = mat(wb_of(c, w.msg_w), 2 * H, H, 2 * H, true);
  d.stable = kStableB;  // the weights; x_l comes from the kernel just before
  d.ep.C = pq_at(c, l); d.ep.ldc = 2 * H; d.ep.bias = w.msg_b; d.ep.bias_n = H;
  return tc(c, d);
}

// BF16: x' = ReLU([x | agg | amp*agg | att*agg] W_U + b_U), also written as
// the BF16 input of the next layer
int tc_update(gcnn_ctx *c, int Ngrid, int l) {
  const int H = c->H;
  LayerW w = layer_ptrs(c->params, c, l);
  GCNN_TRY(stage_x(c, Ngrid, l));
  TcDesc d = tblank();
  d.M = Ngrid; d.N = H; d.K = pad64(16 * H); d.node_dim = kNodeM;
  d.A = mat(U_at(c, l), 16 * H, Ngrid, 16 * H, false);
  d.B = mat(wb_of(c, w.upd_w), H, 16 * H, H, true);
  d.stable = kStableB;  // the weights; the aggregates come from the kernel just before
  d.ep.C = xs_at(c, l + 1); d.ep.ldc = H; d.ep.bias = w.upd_b; d.ep.bias_n = H; d.ep.relu = true;
  if (l + 1 < c->L) { d.ep.C16 = X_at(c, l + 1); d.ep.ld16 = X_ld(c); }
  return tc(c, d);
}

// BF16 backward of layer l.  dH holds dL/dx_{l+1} (FP32) and G5[cur] its
// masked, scaled BF16 form in columns [0, 3H).  Writes dX = dL/dx_l and, for
// l > 0, columns [0, 3H) of G5[cur ^ 1]; [dP | dQ] goes to dPQ (FP32) and to
// columns [3H, 5H) of G5[cur].
//
// Critical path on the main stream: dagg -> aggregate backward -> dx.  The
// weight and bias gradients (dW_U, dW_M, their split-K reductions and the
// bias column sums) go to the side lane: dW_U once G5[cur] is final (event
// `fork`), dW_M and the sums once [dP | dQ] is (event `mid`); event `done`
// marks the lane's work of the layer.  dx(l) overwrites G5[cur ^ 1] and the
// FP32 gradient the previous layer's sums read, so it waits for `done` of
// layer l + 1; dPQ alternates between two buffers by layer.
int tc_backward_layer(gcnn_ctx *c, int Gn, int Ngrid, int Egrid, int l, int cur, float *dPQ, bool ov) {
  const int H = c->H;
  DevDims dims{c->bb.dims};
  LayerW gw = layer_ptrs(c->grads, c, l);
  const float *pq = pq_at(c, l), *h = xs_at(c, l + 1);
  float *agg = agg_at(c, l);
  uint16_t *G = c->G5[cur];
  // the weight-gradient GEMMs plan with the side lane's CTA limit in both
  // modes, so the overlapped and the serial backward pick the same split-K
  // plans and give the same results bit for bit
  GemmWorkspace capped = c->ws;
  capped.max_ctas = side_gemm_ctas();
  const Lane lane = ov ? Lane{c->side, &c->ws_side} : Lane{c->stream, &capped};
  cudaEvent_t fork = ov ? c->side_ev[3 * l] : nullptr, mid = ov ? c->side_ev[3 * l + 1] : nullptr;
  cudaEvent_t done = ov ? c->side_ev[3 * l + 2] : nullptr;
  if (c->cfg.recompute) {
    PhaseScope ps(c, GCNN_PHASE_AGG_FWD);
    GCNN_TRY(launch_aggregate_fwd(Ngrid, H, dims, c->bb.row_ptr, c->bb.col, pq, agg, (float)c->cfg.std_eps, c->err,
                                  c->stream, U_at(c, l) + H, 16 * H, c->bb.amp, c->bb.att, c->bb.eattr,
                                  layer_ptrs(c->params, c, l).edge_w, c->cfg.edge_features, true));
    GCNN_TRY(stage_x(c, Ngrid, l));
  }
  if (ov) {
    GCNN_CUDA_TRY(cudaEventRecord(fork, c->stream));
    GCNN_CUDA_TRY(cudaStreamWaitEvent(lane.s, fork, 0));
  }
  {  // dW_U = [x | scaled aggs]^T dpre
    TcDesc d = tblank();
    d.M = 16 * H; d.N = H; d.K = Ngrid; d.node_dim = kNodeK;
    d.A = mat(U_at(c, l), 16 * H, Ngrid, 16 * H, true);
    d.B = mat(G + 2 * H, 5 * H, Ngrid, H, true);
    // the forward's operand, unless recomputed just before
    d.stable = c->cfg.recompute ? kStableNone : kStableA;
    d.ep.C = gw.upd_w; d.ep.ldc = H;
    d.lean = true;
    GCNN_TRY(tc_on(c, d, lane));
  }
  // layer l + 1 on a third stream, joined at the end of the backward: its
  // gradients are complete at `done` of l + 1, its dx before `fork`; one
  // block per SM leaves room for the GEMMs of the other two streams
  if (ov && l + 1 < c->L && layers_updated_early(c)) {
    GCNN_CUDA_TRY(cudaStreamWaitEvent(c->opt, fork, 0));
    GCNN_CUDA_TRY(cudaStreamWaitEvent(c->opt, c->side_ev[3 * (l + 1) + 2], 0));
    const long long b = (long long)c->T * H + (long long)(l + 1) * c->layer_size;
    GCNN_TRY(adam(c, AdamSpan{b, c->layer_size, 0, 0}, false, num_sms(), c->opt));
  }
  {  // dagg = [amp g | att g | g] [W_amp ; W_att ; W_id]^T
    TcDesc d = tblank();
    d.M = Ngrid; d.N = kAgg * H; d.K = pad64(3 * H); d.node_dim = kNodeM;
    d.A = mat(G, 5 * H, Ngrid, 3 * H, false);
    d.B = mat(Wd_at(c, l), 3 * H, kAgg * H, 3 * H, false);
    d.stable = kStableB;
    d.ep.C = c->dagg; d.ep.ldc = kAgg * H;
    GCNN_TRY(tc(c, d));
  }
  {
    PhaseScope ps(c, GCNN_PHASE_AGG_BWD);
    // layers run from L - 1 down: the first one cuts the batch into chunks, the rest reuse them
    GCNN_TRY(launch_aggregate_bwd_graphs(Gn, Ngrid, Egrid, H, dims, c->bb.node_off, c->bb.row_ptr, c->bb.col,
                                         c->bb.rev, pq, agg, c->dagg, dPQ, c->dm, c->chunks,
                                         (float)c->cfg.std_eps, c->err, c->stream, G + 3 * H, 5 * H, c->bb.eattr,
                                         layer_ptrs(c->params, c, l).edge_w, c->cfg.edge_features,
                                         l == c->L - 1, true));
  }
  // before the next layer's aggregation backward reuses dm
  if (c->cfg.edge_features > 0) GCNN_TRY(gemm_bond_rows(c, Egrid, gw.edge_w));
  if (ov) {
    GCNN_CUDA_TRY(cudaEventRecord(mid, c->stream));
    GCNN_CUDA_TRY(cudaStreamWaitEvent(lane.s, mid, 0));
  }
  {  // dW_M = x^T [dP | dQ]
    TcDesc d = tblank();
    d.M = H; d.N = 2 * H; d.K = Ngrid; d.node_dim = kNodeK;
    d.A = mat(X_at(c, l), X_ld(c), Ngrid, H, true);
    d.B = mat(G + 3 * H, 5 * H, Ngrid, 2 * H, true);
    d.stable = kStableA;  // x_l from the forward; [dP | dQ] from the aggregation backward
    d.ep.C = gw.msg_w; d.ep.ldc = 2 * H;
    d.lean = true;
    GCNN_TRY(tc_on(c, d, lane));
    // bias gradients: db_U = sum of dpre, db_M = sum of dP (FP32, fixed order)
    PhaseScope ps(c, GCNN_PHASE_GEMM);
    GCNN_TRY(launch_colsum2(Ngrid, H, H, dims, c->dH, H, h, H, dPQ, 2 * H, gw.upd_b, gw.msg_b, lane.s));
  }
  // layer l's gradients are final: before `done`, which the main stream joins
  GCNN_TRY(mark_grads_ready(c, l, lane.s));
  if (ov) {
    GCNN_CUDA_TRY(cudaEventRecord(done, lane.s));
    if (l + 1 < c->L) GCNN_CUDA_TRY(cudaStreamWaitEvent(c->stream, c->side_ev[3 * (l + 1) + 2], 0));
  }
  {  // dx = [g | dP | dQ] [W_x | A | B]^T ; the next layer's masked, scaled BF16 gradient
    TcDesc d = tblank();
    d.M = Ngrid; d.N = H; d.K = pad64(3 * H); d.node_dim = kNodeM;
    d.A = mat(G + 2 * H, 5 * H, Ngrid, 3 * H, false);
    d.B = mat(Wx_at(c, l), 3 * H, H, 3 * H, false);
    d.stable = kStableB;
    d.ep.C = c->dX; d.ep.ldc = H;
    if (l > 0) {
      d.ep.D3 = c->G5[cur ^ 1]; d.ep.ld3 = 5 * H;
      d.ep.mask = xs_at(c, l); d.ep.ldm = H; d.ep.amp = c->bb.amp; d.ep.att = c->bb.att;
    }
    GCNN_TRY(tc(c, d));
  }
  return GCNN_OK;
}

}  // namespace

PhaseScope::PhaseScope(gcnn_ctx *c, int phase) : c_(c), idx_(-1) {
  if (!c->prof_on) return;
  if (c->capturing) {  // event-record nodes of a profiling graph
    gcnn_ctx::ProfEvent pe{phase, nullptr, nullptr};
    if (cudaEventCreate(&pe.a) != cudaSuccess || cudaEventCreate(&pe.b) != cudaSuccess) {
      if (pe.a) cudaEventDestroy(pe.a);
      cudaGetLastError();
      return;
    }
    c->cap_ev.push_back(pe);
    idx_ = (long)c->cap_ev.size() - 1;
    cudaEventRecordWithFlags(pe.a, c->stream, cudaEventRecordExternal);
    return;
  }
  if (c->prof_used * 2 + 2 > c->prof_ev.size()) {
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
      if (a) cudaEventDestroy(a);
      cudaGetLastError();
      return;
    }
    c->prof_ev.push_back(a);
    c->prof_ev.push_back(b);
    c->prof_cls.push_back(0);
  }
  idx_ = (long)c->prof_used++;
  c->prof_cls[idx_] = phase;
  cudaEventRecord(c->prof_ev[2 * idx_], c->stream);
}

PhaseScope::~PhaseScope() {
  if (idx_ < 0) return;
  if (c_->capturing) cudaEventRecordWithFlags(c_->cap_ev[idx_].b, c_->stream, cudaEventRecordExternal);
  else cudaEventRecord(c_->prof_ev[2 * idx_ + 1], c_->stream);
}

int ctx_forward(gcnn_ctx *c, int G, int Ngrid, int Egrid, bool train) {
  (void)Egrid;
  const int H = c->H;
  DevDims dims{c->bb.dims};
  const bool bf = bf16(c);
  {
    PhaseScope ps(c, GCNN_PHASE_EMBED);
    GCNN_TRY(launch_embed(Ngrid, H, dims, c->bb.types, c->params, c->T, xs_at(c, 0), c->stream,
                          bf ? X_at(c, 0) : nullptr, X_ld(c)));
  }
  for (int l = 0; l < c->L; ++l) {
    if (bf) GCNN_TRY(tc_message(c, Ngrid, l));
    else GCNN_TRY(gemm_message(c, Ngrid, l));
    {
      PhaseScope ps(c, GCNN_PHASE_AGG_FWD);
      GCNN_TRY(launch_aggregate_fwd(Ngrid, H, dims, c->bb.row_ptr, c->bb.col, pq_at(c, l), agg_at(c, l),
                                    (float)c->cfg.std_eps, c->err, c->stream, bf ? U_at(c, l) + H : nullptr,
                                    16 * H, c->bb.amp, c->bb.att, c->bb.eattr, layer_ptrs(c->params, c, l).edge_w,
                                    c->cfg.edge_features, true));
    }
    if (bf) GCNN_TRY(tc_update(c, Ngrid, l));
    else GCNN_TRY(gemm_update(c, Ngrid, l));
  }
  if (c->cfg.node_head) GCNN_TRY(node_head_forward(c, Ngrid, train));
  PhaseScope ps(c, GCNN_PHASE_HEAD);
  GCNN_TRY(launch_head_graph(head_args(c, G, nullptr), true, train && c->fuse_head, c->stream));
  return GCNN_OK;
}

int ctx_backward(gcnn_ctx *c, int G, int Ngrid, int Egrid, const float *dpred, double *loss_accum) {
  const int H = c->H;
  DevDims dims{c->bb.dims};
  if (c->cfg.node_head) GCNN_TRY(node_head_backward(c, Ngrid, loss_accum));
  {
    PhaseScope ps(c, GCNN_PHASE_HEAD);
    if (!c->fuse_head) GCNN_TRY(launch_head_graph(head_args(c, G, dpred), false, true, c->stream));
    HeadGradArgs ga{G, H, c->Hh, dims, c->pooled, c->z1, c->dz1, c->dpred, c->pred, c->bb.y,
                    head_ptr(c->grads, c), loss_accum};
    // the head's parameter gradients and loss sums feed only the optimiser:
    // on the side lane when the backward overlaps
    cudaStream_t hs = c->stream;
    if (bf16(c) && overlapped(c)) {
      cudaEvent_t ev = c->side_ev[3 * c->L];
      GCNN_CUDA_TRY(cudaEventRecord(ev, c->stream));
      GCNN_CUDA_TRY(cudaStreamWaitEvent(c->side, ev, 0));
      hs = c->side;
    }
    GCNN_TRY(launch_head_grad(ga, hs));
  }
  if (bf16(c)) {
    const bool ov = overlapped(c);
    int cur = 0;
    for (int l = c->L - 1; l >= 0; --l) {
      float *dPQ = (ov && (l & 1)) ? c->dPQ2 : c->dPQ;
      GCNN_TRY(tc_backward_layer(c, G, Ngrid, Egrid, l, cur, dPQ, ov));
      cur ^= 1;
      std::swap(c->dH, c->dX);
    }
    // the third stream's updates of layers L-1 .. 1 (each launched during the
    // backward of the layer below it) join the main stream below
    if (layers_updated_early(c) && c->L >= 2) GCNN_CUDA_TRY(cudaEventRecord(c->opt_ev, c->opt));
  }
  for (int l = bf16(c) ? -1 : c->L - 1; l >= 0; --l) {
    LayerW w = layer_ptrs(c->params, c, l);
    LayerW gw = layer_ptrs(c->grads, c, l);
    const float *x = xs_at(c, l), *h = xs_at(c, l + 1), *pq = pq_at(c, l);
    float *agg = agg_at(c, l);
    if (c->cfg.recompute) {
      PhaseScope ps(c, GCNN_PHASE_AGG_FWD);
      GCNN_TRY(launch_aggregate_fwd(Ngrid, H, dims, c->bb.row_ptr, c->bb.col, pq, agg,
                                    (float)c->cfg.std_eps, c->err, c->stream, nullptr, 0, nullptr, nullptr,
                                    c->bb.eattr, w.edge_w, c->cfg.edge_features, true));
    }
    // dW_U (16H x H) and db_U: [x ; agg ; amp agg ; att agg ; 1]^T (dh * [h > 0])
    {
      GemmDesc d = blank();
      d.M = 16 * H + 1; d.N = H; d.K = Ngrid; d.node_dim = kNodeK;
      d.a_kcontig = false; d.b_ncontig = true;
      d.A.nseg = 5;
      d.A.seg[0] = seg(0, x, H);
      d.A.seg[1] = seg(H, agg, kAgg * H);
      d.A.seg[2] = seg(6 * H, agg, kAgg * H, c->bb.amp);
      d.A.seg[3] = seg(11 * H, agg, kAgg * H, c->bb.att);
      d.A.seg[4] = seg(16 * H, nullptr, 0);
      d.B.nseg = 1; d.B.seg[0] = seg(0, c->dH, H, nullptr, h);
      d.C = gw.upd_w; d.ldc = H;
      GCNN_TRY(gemm(c, d));
    }
    // dagg = sum_s s_i (dh * [h > 0]) W_s^T, W_s = rows H + 5Hs .. of W_U
    {
      GemmDesc d = blank();
      d.M = Ngrid; d.N = kAgg * H; d.K = 3 * H; d.node_dim = kNodeM;
      d.a_kcontig = true; d.b_ncontig = false;
      d.A.nseg = 3;
      d.A.seg[0] = seg(0, c->dH, H, nullptr, h);
      d.A.seg[1] = seg(H, c->dH, H, c->bb.amp, h);
      d.A.seg[2] = seg(2 * H, c->dH, H, c->bb.att, h);
      d.B.nseg = 3;
      d.B.seg[0] = seg(0, w.upd_w + (size_t)H * H, H);
      d.B.seg[1] = seg(H, w.upd_w + (size_t)6 * H * H, H);
      d.B.seg[2] = seg(2 * H, w.upd_w + (size_t)11 * H * H, H);
      d.C = c->dagg; d.ldc = kAgg * H;
      GCNN_TRY(gemm(c, d));
    }
    {
      PhaseScope ps(c, GCNN_PHASE_AGG_BWD);
      GCNN_TRY(launch_aggregate_bwd_graphs(G, Ngrid, Egrid, H, dims, c->bb.node_off, c->bb.row_ptr, c->bb.col,
                                           c->bb.rev, pq, agg, c->dagg, c->dPQ, c->dm, c->chunks,
                                           (float)c->cfg.std_eps, c->err, c->stream, nullptr, 0, c->bb.eattr,
                                           w.edge_w, c->cfg.edge_features, l == c->L - 1, true));
    }
    if (c->cfg.edge_features > 0) GCNN_TRY(gemm_bond_rows(c, Egrid, gw.edge_w));
    // dW_M (H x 2H) and db_M: [x ; 1]^T dPQ  (bias row keeps the first H columns)
    {
      GemmDesc d = blank();
      d.M = H + 1; d.N = 2 * H; d.K = Ngrid; d.node_dim = kNodeK;
      d.a_kcontig = false; d.b_ncontig = true;
      d.A.nseg = 2;
      d.A.seg[0] = seg(0, x, H);
      d.A.seg[1] = seg(H, nullptr, 0);
      d.B.nseg = 1; d.B.seg[0] = seg(0, c->dPQ, 2 * H);
      d.C = gw.msg_w; d.ldc = 2 * H; d.last_row_cols = H;
      GCNN_TRY(gemm(c, d));
    }
    GCNN_TRY(mark_grads_ready(c, l, c->stream));
    // dx = (dh * [h > 0]) W_x^T + [dP | dQ] [A | B]^T
    {
      GemmDesc d = blank();
      d.M = Ngrid; d.N = H; d.K = 3 * H; d.node_dim = kNodeM;
      d.a_kcontig = true; d.b_ncontig = false;
      d.A.nseg = 2;
      d.A.seg[0] = seg(0, c->dH, H, nullptr, h);
      d.A.seg[1] = seg(H, c->dPQ, 2 * H);
      d.B.nseg = 2;
      d.B.seg[0] = seg(0, w.upd_w, H);
      d.B.seg[1] = seg(H, w.msg_w, 2 * H);
      d.C = c->dX; d.ldc = H;
      GCNN_TRY(gemm(c, d));
    }
    std::swap(c->dH, c->dX);
  }
  // embedding: dEmb[t] = sum of dx0 over nodes of type t; it needs only the
  // main stream's dx, so it runs beside the second stream's last layer
  {
    PhaseScope ps(c, GCNN_PHASE_EMBED_BWD);
    GCNN_TRY(launch_embed_bwd(Ngrid, H, dims, c->bb.types, c->dH, c->T, c->grads, c->stream));
  }
  if (bf16(c) && overlapped(c)) {
    // every gradient is complete before the optimiser: layer 0's weight
    // gradients and the head's on the second stream, and the third stream's
    // updates join here
    GCNN_CUDA_TRY(cudaStreamWaitEvent(c->stream, c->side_ev[2], 0));
    if (layers_updated_early(c) && c->L >= 2) GCNN_CUDA_TRY(cudaStreamWaitEvent(c->stream, c->opt_ev, 0));
  }
  return mark_grads_ready(c, c->L, c->stream);  // every gradient is final here
}

int ctx_step(gcnn_ctx *c) {
  PhaseScope ps(c, GCNN_PHASE_ADAM);
  const long long lb = (long long)c->T * c->H, le = lb + (long long)c->L * c->layer_size;
  // after a train step's overlapped backward the embedding table, layer 0
  // and the parameters after the layers remain (layers L-1 .. 1 were updated
  // on the third stream); otherwise everything
  const AdamSpan sp = layers_updated_early(c) ? AdamSpan{0, lb + c->layer_size, le, (long long)c->P - le}
                                              : AdamSpan{0, 0, 0, (long long)c->P};
  return adam(c, sp, true, 0, c->stream);
}

int ctx_refresh_bf16(gcnn_ctx *c) {
  if (!c->wb) return GCNN_OK;
  GCNN_TRY(launch_cast_bf16(c->P, c->params, c->wb, c->stream));
  for (int l = 0; l < c->L; ++l) {
    LayerW w = layer_ptrs(c->params, c, l);
    uint16_t *wd = c->wpack + (size_t)l * 18 * c->H * c->H;
    GCNN_TRY(launch_pack_layer(c->H, w.msg_w, w.upd_w, wd, wd + (size_t)15 * c->H * c->H, c->stream));
  }
  return GCNN_OK;
}

}  // namespace gcnn
