// C ABI (include/gcnn.h): argument checking, context lifetime, the arena,
// collation staging, CUDA-graph capture of the training step, checkpoints.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <cstdlib>
#include <mutex>
#include <vector>

#include "context.h"

using namespace gcnn;

namespace {

// process-wide kernel timeline (gcnn_timeline_*)
struct TimelineHost {
  char *buf = nullptr;
  unsigned cap = 0;
  size_t off_t = 0, off_id = 0;
};
TimelineHost g_tl;
std::mutex g_tl_mu;

int timeline_attach_all(void *tl) {
  GCNN_TRY(timeline_attach_collate(tl));
  GCNN_TRY(timeline_attach_aggregate(tl));
  GCNN_TRY(timeline_attach_small(tl));
  GCNN_TRY(timeline_attach_gemm_simt(tl));
  GCNN_TRY(timeline_attach_gemm_tc(tl));
  return GCNN_OK;
}

constexpr size_t kAlign = 256;

struct Carve {
  size_t off = 0;
  template <typename T>
  size_t take(size_t n) {
    off = (off + kAlign - 1) / kAlign * kAlign;
    const size_t at = off;
    off += std::max<size_t>(n, 1) * sizeof(T);
    return at;
  }
};

int64_t layer_size_of(int64_t H) { return 2 * H * H + H + 16 * H * H + H; }

int64_t param_count_of(const gcnn_config &c) {
  const int64_t H = c.hidden, Hh = c.head_hidden;
  const int64_t base = (int64_t)c.n_types * H + (int64_t)c.layers * layer_size_of(H) + H * Hh + 2 * Hh + 1;
  // bond rows, then the node head, each from a multiple of 4 floats (16-byte rows)
  const int64_t trunk = c.edge_features == 0 ? base : (base + 3) / 4 * 4 + (int64_t)c.layers * c.edge_features * H;
  return c.node_head ? (trunk + 3) / 4 * 4 + H * Hh + 2 * Hh + 1 : trunk;
}

int check_config(const gcnn_config *c) {
  if (!c) return set_error(GCNN_EINVAL, "null config");
  if (c->hidden < 8 || c->hidden > 1024 || c->hidden % 8)
    return set_error(GCNN_EINVAL, "hidden must be a multiple of 8 in [8, 1024] (got %d)", c->hidden);
  if (c->layers < 1 || c->layers > 64) return set_error(GCNN_EINVAL, "layers must be in [1, 64]");
  if (c->n_types < 1 || c->n_types > 16) return set_error(GCNN_EINVAL, "n_types must be in [1, 16]");
  if (c->head_hidden < 1 || c->head_hidden > 1024) return set_error(GCNN_EINVAL, "head_hidden must be in [1, 1024]");
  if (c->max_graphs < 1 || c->max_nodes < 1 || c->max_edges < 0)
    return set_error(GCNN_EINVAL, "capacities must be positive");
  if ((int64_t)c->max_nodes * c->hidden * 16 > (int64_t)1 << 31 ||
      (int64_t)c->max_edges * c->hidden > (int64_t)1 << 31)
    return set_error(GCNN_EINVAL, "capacity too large for 32-bit indexing");
  if (c->precision != GCNN_PREC_FP32 && c->precision != GCNN_PREC_BF16)
    return set_error(GCNN_EINVAL, "precision must be GCNN_PREC_FP32 or GCNN_PREC_BF16 (got %d)", c->precision);
  if (!(c->delta > 0.0) || !(c->std_eps >= 0.0)) return set_error(GCNN_EINVAL, "delta must be > 0, std_eps >= 0");
  if (c->edge_features < 0 || c->edge_features > 16)
    return set_error(GCNN_EINVAL, "edge_features must be in [0, 16] (got %d)", c->edge_features);
  if (c->node_head != 0 && c->node_head != 1) return set_error(GCNN_EINVAL, "node_head must be 0 or 1");
  if (c->node_head && (c->head_hidden % 4 || !(c->node_loss_weight >= 0.0)))
    return set_error(GCNN_EINVAL, "node head: head_hidden must be a multiple of 4 and node_loss_weight >= 0");
  return GCNN_OK;
}

int make_scaler_table(gcnn_ctx *c) {
  std::vector<float> tab(2 * (kMaxGraphEdges + 1));
  for (int d = 0; d <= kMaxGraphEdges; ++d) {
    const double dd = d > 1 ? (double)d : 1.0;
    tab[2 * d] = (float)(std::log(dd + 1.0) / c->cfg.delta);
    tab[2 * d + 1] = (float)(c->cfg.delta / std::log(dd + 1.0));
  }
  GCNN_CUDA_TRY(cudaMemcpy(c->scal_tab, tab.data(), tab.size() * sizeof(float), cudaMemcpyHostToDevice));
  return GCNN_OK;
}

size_t stage_bytes_of(int Gc, int Nc, int Ec, int F) {
  // mini-store: node_ptr, edge_ptr (i64 [G+1]), y (f32 [G]), types (u8 [N]), edges (u8 [2E]),
  // bond features (f32 [E][F]), ids
  // (+ node targets f32 [N])
  return 3 * 8 * (size_t)(Gc + 1) + 4 * (size_t)Gc + 5 * (size_t)Nc + 2 * (size_t)Ec + 4 * (size_t)Ec * F + 6 * 64;
}

void destroy_ctx(gcnn_ctx *c) {
  if (!c) return;
  for (auto &kv : c->graphs) {
    cudaGraphExecDestroy(kv.second.exec);
    if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
    for (auto &pe : kv.second.ev) {
      cudaEventDestroy(pe.a);
      cudaEventDestroy(pe.b);
    }
  }
  for (auto &pe : c->cap_ev) {
    cudaEventDestroy(pe.a);
    cudaEventDestroy(pe.b);
  }
  for (cudaEvent_t e : c->prof_ev) cudaEventDestroy(e);
  for (int q = 0; q < 2; ++q) {
    if (c->stage_host[q]) cudaFreeHost(c->stage_host[q]);
    if (c->stage_ev[q]) cudaEventDestroy(c->stage_ev[q]);
  }
  if (c->lr_pinned) cudaFreeHost(c->lr_pinned);
  if (c->scale_pinned) cudaFreeHost(c->scale_pinned);
  for (cudaEvent_t e : c->grad_ev) cudaEventDestroy(e);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->side) cudaStreamDestroy(c->side);
  if (c->opt) cudaStreamDestroy(c->opt);
  if (c->opt_ev) cudaEventDestroy(c->opt_ev);
  for (cudaEvent_t e : c->side_ev) cudaEventDestroy(e);
  if (c->order_dev) cudaFree(c->order_dev);
  if (c->dmem) cudaFree(c->dmem);
  delete c;
}

int sync(gcnn_ctx *c) {
  GCNN_CUDA_TRY(cudaStreamSynchronize(c->stream));
  return GCNN_OK;
}

int same_batch(const gcnn_ctx *c, const gcnn_batch *b) {
  if (!b) return set_error(GCNN_EINVAL, "null batch");
  if (b->node_off != c->bb.node_off) return set_error(GCNN_EINVAL, "batch was not collated by this context");
  if (b->n_graphs < 0 || b->n_graphs > c->Gc || b->n_nodes < 0 || b->n_nodes > c->Nc || b->n_edges < 0 ||
      b->n_edges > c->Ec)
    return set_error(GCNN_EINVAL, "batch exceeds the context capacity");
  return GCNN_OK;
}

int set_lr(gcnn_ctx *c, float lr) {
  if (!(lr >= 0.f) || !std::isfinite(lr)) return set_error(GCNN_EINVAL, "learning rate must be finite and >= 0");
  if (lr != c->lr_host) {
    *c->lr_pinned = lr;
    GCNN_CUDA_TRY(cudaMemcpyAsync(c->lr_dev, c->lr_pinned, sizeof(float), cudaMemcpyHostToDevice, c->stream));
    // the pinned source must stay valid until the copy ran
    GCNN_CUDA_TRY(cudaStreamSynchronize(c->stream));
    c->lr_host = lr;
  }
  return GCNN_OK;
}

int round_up(int v, int m, int cap) { return std::min(cap, (v + m - 1) / m * m); }

// Launch grids cover the batch rounded up to a bucket; kernels read the true
// sizes from the device, so one captured graph serves every batch in a bucket.
int grid_nodes(const gcnn_ctx *c, const gcnn_batch *b) { return round_up(std::max(b->n_nodes, 1), 256, c->Nc); }
int grid_edges(const gcnn_ctx *c, const gcnn_batch *b) { return round_up(std::max(b->n_edges, 1), 512, c->Ec); }

}  // namespace

// ======================================================================= C ABI
extern "C" {

const char *gcnn_last_error(void) { return last_error(); }
int gcnn_version(void) { return 100; }

// ---------------------------------------------------------------- store
int gcnn_store_open(const char *path, gcnn_store **out) { return store_open(path, out); }
int gcnn_store_close(gcnn_store *st) { return store_close(st); }

int gcnn_store_info(const gcnn_store *st, int64_t *g, int64_t *n, int64_t *e) {
  if (!st) return set_error(GCNN_EINVAL, "null store");
  if (g) *g = st->G;
  if (n) *n = st->N;
  if (e) *e = st->E;
  return GCNN_OK;
}

int gcnn_store_edge_features(const gcnn_store *st, int32_t *f) {
  if (!st || !f) return set_error(GCNN_EINVAL, "null argument");
  *f = st->F;
  return GCNN_OK;
}

int gcnn_store_has_node_targets(const gcnn_store *st, int32_t *has) {
  if (!st || !has) return set_error(GCNN_EINVAL, "null argument");
  *has = st->ynode != nullptr;
  return GCNN_OK;
}

int gcnn_store_batch_size(const gcnn_store *st, const int64_t *ids, int64_t n, int64_t *nn, int64_t *ne) {
  if (!st || (!ids && n > 0) || n < 0 || !nn || !ne) return set_error(GCNN_EINVAL, "store_batch_size: bad arguments");
  return store_batch_size(st, ids, n, nn, ne);
}

int gcnn_store_delta(const gcnn_store *st, const int64_t *ids, int64_t n, double *delta) {
  if (!st || !delta || n < 0) return set_error(GCNN_EINVAL, "store_delta: bad arguments");
  return store_delta(st, ids, n, delta);
}

int gcnn_store_set_targets(gcnn_store *st, const float *y, int64_t n) { return store_set_targets(st, y, n); }
int gcnn_store_to_device(gcnn_store *st) { return store_to_device(st); }

// ---------------------------------------------------------------- context
int gcnn_config_default(gcnn_config *cfg, int32_t hidden, int32_t layers, int32_t max_graphs,
                        int32_t max_nodes, int32_t max_edges) {
  if (!cfg) return set_error(GCNN_EINVAL, "null config");
  memset(cfg, 0, sizeof(*cfg));
  cfg->hidden = hidden;
  cfg->layers = layers;
  cfg->n_types = 7;
  cfg->head_hidden = hidden;
  cfg->max_graphs = max_graphs;
  cfg->max_nodes = max_nodes;
  cfg->max_edges = max_edges;
  cfg->precision = GCNN_PREC_FP32;
  cfg->recompute = 0;
  cfg->delta = 1.0;
  cfg->std_eps = 1e-5;
  cfg->beta1 = 0.9;
  cfg->beta2 = 0.999;
  cfg->adam_eps = 1e-8;
  cfg->weight_decay = 0.0;
  cfg->node_loss_weight = 1.0;
  return GCNN_OK;
}

int gcnn_create(const gcnn_config *cfg, void *stream, gcnn_ctx **out) {
  if (!out) return set_error(GCNN_EINVAL, "null output");
  *out = nullptr;
  GCNN_TRY(check_config(cfg));
  gcnn_ctx *c = new gcnn_ctx();
  c->cfg = *cfg;
  c->stream = static_cast<cudaStream_t>(stream);
  cudaError_t e0 = cudaGetDevice(&c->device);
  if (e0 != cudaSuccess) {
    delete c;
    return set_error(GCNN_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e0));
  }
  c->H = cfg->hidden; c->L = cfg->layers; c->T = cfg->n_types; c->Hh = cfg->head_hidden;
  c->layer_size = layer_size_of(c->H);
  c->P = param_count_of(*cfg);
  c->Gc = cfg->max_graphs; c->Nc = cfg->max_nodes; c->Ec = cfg->max_edges;
  const size_t H = c->H, Nc = c->Nc, Ec = c->Ec, Gc = c->Gc, L = c->L, Hh = c->Hh;
  // split-K workspace: the largest of the step's GEMMs
  // (over every node-count bucket a batch can launch with)
  size_t wsf = 0;
  for (int ng = 256;; ng += 256) {
    const int n = std::min(ng, (int)Nc), h = (int)H;
    wsf = std::max(wsf, gemm_simt_workspace_floats(n, 2 * h, h));
    wsf = std::max(wsf, gemm_simt_workspace_floats(n, h, 16 * h));
    wsf = std::max(wsf, gemm_simt_workspace_floats(16 * h + 1, h, n));
    wsf = std::max(wsf, gemm_simt_workspace_floats(n, kAgg * h, 3 * h));
    wsf = std::max(wsf, gemm_simt_workspace_floats(h + 1, 2 * h, n));
    wsf = std::max(wsf, gemm_simt_workspace_floats(n, h, 3 * h));
    if (cfg->node_head) {  // node head: x W1n, dz W1n^T, [x ; 1]^T dz
      wsf = std::max(wsf, gemm_simt_workspace_floats(n, (int)Hh, h));
      wsf = std::max(wsf, gemm_simt_workspace_floats(n, h, (int)Hh));
      wsf = std::max(wsf, gemm_simt_workspace_floats(h + 1, (int)Hh, n));
    }
    if (cfg->precision == GCNN_PREC_BF16) {
      const int r64 = (h + 63) / 64 * 64, r3 = (3 * h + 63) / 64 * 64, r16 = (16 * h + 63) / 64 * 64;
      wsf = std::max(wsf, gemm_tc_workspace_floats(n, 2 * h, r64));
      wsf = std::max(wsf, gemm_tc_workspace_floats(n, h, r16));
      wsf = std::max(wsf, gemm_tc_workspace_floats(16 * h, h, n));
      wsf = std::max(wsf, gemm_tc_workspace_floats(n, kAgg * h, r3));
      wsf = std::max(wsf, gemm_tc_workspace_floats(h, 2 * h, n));
      wsf = std::max(wsf, gemm_tc_workspace_floats(n, h, r3));
    }
    if (n == (int)Nc) break;
  }
  // sizes of every buffer, carved from one allocation
  Carve cv;
  const size_t o_params = cv.take<float>(c->P), o_grads = cv.take<float>(c->P);
  const size_t o_m = cv.take<float>(c->P), o_v = cv.take<float>(c->P);
  const size_t o_opt = cv.take<int>(16), o_lr = cv.take<float>(4), o_ls = cv.take<float>(4);
  const size_t o_tab = cv.take<float>(2 * (kMaxGraphEdges + 1)), o_err = cv.take<unsigned>(4);
  const size_t o_node_off = cv.take<int>(Gc + 1), o_edge_off = cv.take<int>(Gc + 1);
  const size_t o_gid = cv.take<int>(Nc), o_rp = cv.take<int>(Nc + 1), o_col = cv.take<int>(Ec);
  const size_t o_rev = cv.take<int>(Ec), o_deg = cv.take<int>(Nc), o_amp = cv.take<float>(Nc);
  const size_t o_att = cv.take<float>(Nc), o_y = cv.take<float>(Gc), o_types = cv.take<uint8_t>(Nc);
  const size_t o_dims = cv.take<int>(4), o_ids = cv.take<int64_t>(Gc);
  const int F4 = (cfg->edge_features + 3) & ~3;  // 16-byte rows of bond features
  const size_t o_eattr = cv.take<float>((size_t)Ec * F4);
  const size_t NHn = cfg->node_head ? Nc : 0;  // node head buffers
  const size_t o_ynode = cv.take<float>(NHn), o_zn = cv.take<float>(NHn * Hh), o_dzn = cv.take<float>(NHn * Hh);
  const size_t o_predn = cv.take<float>(NHn), o_dpredn = cv.take<float>(NHn), o_dxn = cv.take<float>(NHn * H);
  c->stage_bytes = stage_bytes_of((int)Gc, (int)Nc, (int)Ec, cfg->edge_features);
  const size_t o_stage = cv.take<char>(c->stage_bytes);
  const size_t o_xs = cv.take<float>((L + 1) * Nc * H), o_pq = cv.take<float>(L * Nc * 2 * H);
  const bool fp32_agg = cfg->precision != GCNN_PREC_BF16;  // the BF16 path recomputes them
  const size_t o_agg = cv.take<float>(fp32_agg ? (cfg->recompute ? 1 : L) * Nc * kAgg * H : 0);
  const size_t o_pool = cv.take<float>(Gc * H), o_z1 = cv.take<float>(Gc * Hh), o_pred = cv.take<float>(Gc);
  const size_t o_dpred = cv.take<float>(Gc), o_dz1 = cv.take<float>(Gc * Hh), o_dg = cv.take<float>(Gc * H);
  const size_t o_dH = cv.take<float>(Nc * H), o_dX = cv.take<float>(Nc * H);
  const size_t o_dagg = cv.take<float>(Nc * kAgg * H), o_dPQ = cv.take<float>(Nc * 2 * H);
  const size_t o_dm = cv.take<float>(Ec * H);
  const size_t o_chunks = cv.take<int>(aggregate_chunk_capacity((int)Ec));
  const size_t o_tk = cv.take<unsigned>(16);
  const size_t o_ws = cv.take<float>(wsf);
  const bool bf = cfg->precision == GCNN_PREC_BF16;
  // BF16 without recompute: weight gradients overlap on a second stream,
  // with their own split-K workspace and a second [dP | dQ] buffer
  const bool side = bf && !cfg->recompute;
  const size_t o_ws2 = cv.take<float>(side ? wsf : 0), o_dPQ2 = cv.take<float>(side ? Nc * 2 * H : 0);
  const size_t o_wb = cv.take<uint16_t>(bf ? c->P : 0), o_wp = cv.take<uint16_t>(bf ? L * 18 * H * H : 0);
  const size_t o_U = cv.take<uint16_t>(bf ? (cfg->recompute ? 1 : L) * Nc * 16 * H : 0);
  const size_t o_Xb = cv.take<uint16_t>(bf && cfg->recompute ? L * Nc * H : 0);
  const size_t o_g0 = cv.take<uint16_t>(bf ? Nc * 5 * H : 0), o_g1 = cv.take<uint16_t>(bf ? Nc * 5 * H : 0);
  c->dbytes = cv.off;
  cudaError_t e = cudaMalloc(&c->dmem, c->dbytes);
  if (e != cudaSuccess) {
    destroy_ctx(c);
    return set_error(GCNN_ENOMEM, "cudaMalloc(%zu bytes): %s", c->dbytes, cudaGetErrorString(e));
  }
  char *b = c->dmem;
  c->params = (float *)(b + o_params); c->grads = (float *)(b + o_grads);
  c->adam_m = (float *)(b + o_m); c->adam_v = (float *)(b + o_v);
  c->opt_state = (int *)(b + o_opt); c->lr_dev = (float *)(b + o_lr); c->loss_scale = (float *)(b + o_ls);
  c->scal_tab = (float *)(b + o_tab); c->err = (unsigned *)(b + o_err);
  c->bb.node_off = (int *)(b + o_node_off); c->bb.edge_off = (int *)(b + o_edge_off);
  c->bb.graph_id = (int *)(b + o_gid); c->bb.row_ptr = (int *)(b + o_rp); c->bb.col = (int *)(b + o_col);
  c->bb.rev = (int *)(b + o_rev); c->bb.deg = (int *)(b + o_deg); c->bb.amp = (float *)(b + o_amp);
  c->bb.att = (float *)(b + o_att); c->bb.y = (float *)(b + o_y); c->bb.types = (uint8_t *)(b + o_types);
  c->bb.dims = (int *)(b + o_dims); c->ids_dev = (int64_t *)(b + o_ids);
  c->bb.eattr = cfg->edge_features > 0 ? (float *)(b + o_eattr) : nullptr;
  c->bb.eattr_ld = F4;
  if (cfg->node_head) {
    c->bb.ynode = (float *)(b + o_ynode);
    c->zn = (float *)(b + o_zn); c->dzn = (float *)(b + o_dzn); c->predn = (float *)(b + o_predn);
    c->dpredn = (float *)(b + o_dpredn); c->dxn = (float *)(b + o_dxn);
  }
  c->stage_dev = b + o_stage;
  c->xs = (float *)(b + o_xs); c->PQ = (float *)(b + o_pq); c->agg = fp32_agg ? (float *)(b + o_agg) : nullptr;
  c->pooled = (float *)(b + o_pool); c->z1 = (float *)(b + o_z1); c->pred = (float *)(b + o_pred);
  c->dpred = (float *)(b + o_dpred); c->dz1 = (float *)(b + o_dz1); c->dg = (float *)(b + o_dg);
  c->dH = (float *)(b + o_dH); c->dX = (float *)(b + o_dX); c->dagg = (float *)(b + o_dagg);
  c->dPQ = (float *)(b + o_dPQ); c->dm = (float *)(b + o_dm); c->tickets = (unsigned *)(b + o_tk);
  c->chunks = (int *)(b + o_chunks);
  c->ws.partial = (float *)(b + o_ws); c->ws.floats = wsf;
  c->ws.max_splits = (cfg->flags & GCNN_FLAG_ROW_INVARIANT) ? 1 : 32;
  if (side) {
    c->ws_side = c->ws;
    c->ws_side.partial = (float *)(b + o_ws2);
    c->ws_side.max_ctas = side_gemm_ctas();
    c->dPQ2 = (float *)(b + o_dPQ2);
  }
  if (bf) {
    c->wb = (uint16_t *)(b + o_wb); c->wpack = (uint16_t *)(b + o_wp); c->U = (uint16_t *)(b + o_U);
    if (cfg->recompute) c->Xb = (uint16_t *)(b + o_Xb);
    c->G5[0] = (uint16_t *)(b + o_g0); c->G5[1] = (uint16_t *)(b + o_g1);
  }
  int rc = GCNN_OK;
  if (cudaMemset(c->dmem, 0, c->dbytes) != cudaSuccess) rc = set_error(GCNN_ECUDA, "cudaMemset failed");
  for (int q = 0; q < 2 && rc == GCNN_OK; ++q) {
    if (cudaMallocHost(&c->stage_host[q], c->stage_bytes) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->stage_ev[q], cudaEventDisableTiming) != cudaSuccess)
      rc = set_error(GCNN_ENOMEM, "cannot allocate pinned staging memory");
  }
  if (rc == GCNN_OK && cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
    rc = set_error(GCNN_ECUDA, "cannot create the capture stream");
  if (rc == GCNN_OK && side) {
    if (cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->opt, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->opt_ev, cudaEventDisableTiming) != cudaSuccess)
      rc = set_error(GCNN_ECUDA, "cannot create the side streams");
    for (int q = 0; q < 3 * c->L + 1 && rc == GCNN_OK; ++q) {
      cudaEvent_t ev = nullptr;
      if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess)
        rc = set_error(GCNN_ECUDA, "cannot create events");
      else
        c->side_ev.push_back(ev);
    }
  }
  if (rc == GCNN_OK && (cudaMallocHost(&c->lr_pinned, sizeof(float)) != cudaSuccess ||
                        cudaMallocHost(&c->scale_pinned, 2 * sizeof(float)) != cudaSuccess))
    rc = set_error(GCNN_ENOMEM, "cannot allocate pinned memory");
  if (rc == GCNN_OK) {  // loss-gradient scales start at 1 (a single process)
    const float one[2] = {1.f, 1.f};
    if (cudaMemcpy(c->loss_scale, one, sizeof(one), cudaMemcpyHostToDevice) != cudaSuccess)
      rc = set_error(GCNN_ECUDA, "cannot initialise the loss scale");
  }
  for (int q = 0; q <= c->L && rc == GCNN_OK; ++q) {  // gradient buckets' completion events
    cudaEvent_t ev = nullptr;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess)
      rc = set_error(GCNN_ECUDA, "cannot create events");
    else
      c->grad_ev.push_back(ev);
  }
  if (rc == GCNN_OK) rc = make_scaler_table(c);
  if (rc == GCNN_OK) (void)num_sms();  // cache the SM count outside any capture
  if (rc != GCNN_OK) {
    destroy_ctx(c);
    return rc;
  }
  *out = c;
  return GCNN_OK;
}

int gcnn_destroy(gcnn_ctx *c) {
  if (!c) return GCNN_OK;
  cudaStreamSynchronize(c->stream);
  destroy_ctx(c);
  return GCNN_OK;
}

int gcnn_param_count(const gcnn_ctx *c, int64_t *n) {
  if (!c || !n) return set_error(GCNN_EINVAL, "null argument");
  *n = c->P;
  return GCNN_OK;
}

static int copy_flat(gcnn_ctx *c, float *dev, const float *src, float *dst, int64_t n, int on_device) {
  if (!c || n != c->P) return set_error(GCNN_EINVAL, "expected %lld floats", c ? (long long)c->P : 0LL);
  const cudaMemcpyKind k = src ? (on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice)
                               : (on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost);
  if (src) GCNN_CUDA_TRY(cudaMemcpyAsync(dev, src, n * sizeof(float), k, c->stream));
  else GCNN_CUDA_TRY(cudaMemcpyAsync(dst, dev, n * sizeof(float), k, c->stream));
  return sync(c);
}

// Refresh the BF16 copy of the parameters (BF16 precision only).
static int refresh_bf16(gcnn_ctx *c) {
  if (!c->wb) return GCNN_OK;
  GCNN_TRY(ctx_refresh_bf16(c));
  return sync(c);
}

int gcnn_set_params(gcnn_ctx *c, const float *src, int64_t n, int on_device) {
  if (!src) return set_error(GCNN_EINVAL, "null source");
  GCNN_TRY(copy_flat(c, c ? c->params : nullptr, src, nullptr, n, on_device));
  return refresh_bf16(c);
}
int gcnn_get_params(gcnn_ctx *c, float *dst, int64_t n, int on_device) {
  if (!dst) return set_error(GCNN_EINVAL, "null destination");
  return copy_flat(c, c ? c->params : nullptr, nullptr, dst, n, on_device);
}
int gcnn_get_grads(gcnn_ctx *c, float *dst, int64_t n, int on_device) {
  if (!dst) return set_error(GCNN_EINVAL, "null destination");
  return copy_flat(c, c ? c->grads : nullptr, nullptr, dst, n, on_device);
}

int gcnn_reset_optimizer(gcnn_ctx *c) {
  if (!c) return set_error(GCNN_EINVAL, "null context");
  GCNN_CUDA_TRY(cudaMemsetAsync(c->adam_m, 0, c->P * sizeof(float), c->stream));
  GCNN_CUDA_TRY(cudaMemsetAsync(c->adam_v, 0, c->P * sizeof(float), c->stream));
  GCNN_CUDA_TRY(cudaMemsetAsync(c->opt_state, 0, 16 * sizeof(int), c->stream));
  return sync(c);
}

int gcnn_save(gcnn_ctx *c, const char *path) {
  if (!c || !path) return set_error(GCNN_EINVAL, "null argument");
  std::vector<float> buf(3 * (size_t)c->P);
  int step = 0;
  GCNN_CUDA_TRY(cudaMemcpyAsync(buf.data(), c->params, c->P * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
  GCNN_CUDA_TRY(cudaMemcpyAsync(buf.data() + c->P, c->adam_m, c->P * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
  GCNN_CUDA_TRY(cudaMemcpyAsync(buf.data() + 2 * c->P, c->adam_v, c->P * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
  GCNN_CUDA_TRY(cudaMemcpyAsync(&step, c->opt_state, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  GCNN_TRY(sync(c));
  FILE *f = fopen(path, "wb");
  if (!f) return set_error(GCNN_EINVAL, "cannot write %s", path);
  const int64_t P = c->P;
  bool ok = fwrite("GCNNCKP1", 8, 1, f) == 1 && fwrite(&P, sizeof(P), 1, f) == 1 &&
            fwrite(&step, sizeof(step), 1, f) == 1 && fwrite(buf.data(), sizeof(float), buf.size(), f) == buf.size();
  ok = (fclose(f) == 0) && ok;
  return ok ? GCNN_OK : set_error(GCNN_EINVAL, "short write to %s", path);
}

int gcnn_load(gcnn_ctx *c, const char *path) {
  if (!c || !path) return set_error(GCNN_EINVAL, "null argument");
  FILE *f = fopen(path, "rb");
  if (!f) return set_error(GCNN_EINVAL, "cannot read %s", path);
  char magic[8];
  int64_t P = 0;
  int step = 0;
  std::vector<float> buf(3 * (size_t)c->P);
  bool ok = fread(magic, 8, 1, f) == 1 && memcmp(magic, "GCNNCKP1", 8) == 0 && fread(&P, sizeof(P), 1, f) == 1 &&
            P == c->P && fread(&step, sizeof(step), 1, f) == 1 &&
            fread(buf.data(), sizeof(float), buf.size(), f) == buf.size();
  fclose(f);
  if (!ok) return set_error(GCNN_EFORMAT, "%s is not a checkpoint of this model", path);
  GCNN_CUDA_TRY(cudaMemcpyAsync(c->params, buf.data(), c->P * sizeof(float), cudaMemcpyHostToDevice, c->stream));
  GCNN_CUDA_TRY(cudaMemcpyAsync(c->adam_m, buf.data() + c->P, c->P * sizeof(float), cudaMemcpyHostToDevice, c->stream));
  GCNN_CUDA_TRY(cudaMemcpyAsync(c->adam_v, buf.data() + 2 * c->P, c->P * sizeof(float), cudaMemcpyHostToDevice, c->stream));
  GCNN_CUDA_TRY(cudaMemcpyAsync(c->opt_state, &step, sizeof(int), cudaMemcpyHostToDevice, c->stream));
  GCNN_TRY(sync(c));
  return refresh_bf16(c);
}

int gcnn_check(gcnn_ctx *c) {
  if (!c) return set_error(GCNN_EINVAL, "null context");
  unsigned w = 0;
  GCNN_CUDA_TRY(cudaMemcpyAsync(&w, c->err, sizeof(w), cudaMemcpyDeviceToHost, c->stream));
  GCNN_TRY(sync(c));
  if (w) {
    GCNN_CUDA_TRY(cudaMemsetAsync(c->err, 0, sizeof(unsigned), c->stream));
    GCNN_TRY(sync(c));
    return set_error(GCNN_EDEVICE, "device bounds check fired (bits 0x%x)", w);
  }
  return GCNN_OK;
}

// ---------------------------------------------------------------- batches
int gcnn_collate(gcnn_ctx *c, const gcnn_store *st, const int64_t *ids, int32_t n, gcnn_batch *out) {
  if (!c || !st || !out || n < 0 || (n > 0 && !ids)) return set_error(GCNN_EINVAL, "collate: bad arguments");
  return ctx_collate(c, st, ids, n, out);
}

int gcnn_collate_files(gcnn_ctx *c, const char *const *paths, int32_t n, gcnn_batch *out) {
  if (!c || !out || n < 0 || (n > 0 && !paths)) return set_error(GCNN_EINVAL, "collate_files: bad arguments");
  for (int32_t g = 0; g < n; ++g)
    if (!paths[g]) return set_error(GCNN_EINVAL, "collate_files: null path");
  return ctx_collate_files(c, paths, n, out);
}

int gcnn_store_pack(const char *const *paths, int64_t n_files, const char *out_path, int32_t n_threads) {
  if (!out_path || n_files < 0 || (n_files > 0 && !paths) || n_threads < 1 || n_threads > 256)
    return set_error(GCNN_EINVAL, "store_pack: bad arguments");
  for (int64_t q = 0; q < n_files; ++q)
    if (!paths[q]) return set_error(GCNN_EINVAL, "store_pack: null path");
  return store_pack(paths, n_files, out_path, n_threads);
}

int gcnn_set_order(gcnn_ctx *c, const gcnn_store *st, const int64_t *order, int64_t n) {
  if (!c || !st || !order || n < 1) return set_error(GCNN_EINVAL, "set_order: bad arguments");
  if (!st->dev) return set_error(GCNN_ESTATE, "set_order needs a device-resident store");
  for (int64_t q = 0; q < n; ++q)
    if (order[q] < 0 || order[q] >= st->G) return set_error(GCNN_EINVAL, "set_order: id out of range");
  if (c->order_dev) {
    GCNN_TRY(sync(c));
    cudaFree(c->order_dev);
    c->order_dev = nullptr;
  }
  GCNN_CUDA_TRY(cudaMalloc(&c->order_dev, n * sizeof(int64_t)));
  GCNN_CUDA_TRY(cudaMemcpy(c->order_dev, order, n * sizeof(int64_t), cudaMemcpyHostToDevice));
  c->order_host.assign(order, order + n);
  c->order_store = st;
  return GCNN_OK;
}

int gcnn_collate_range(gcnn_ctx *c, const gcnn_store *st, int64_t first, int32_t count, gcnn_batch *out) {
  if (!c || !st || !out || count < 0) return set_error(GCNN_EINVAL, "collate_range: bad arguments");
  return ctx_collate_range(c, st, first, count, out);
}

int gcnn_batch_export(gcnn_ctx *c, const gcnn_batch *b, int32_t *node_off, int32_t *graph_id, int32_t *row_ptr,
                      int32_t *col, int32_t *rev, int32_t *deg, float *amp, float *att, uint8_t *types, float *y) {
  if (!c) return set_error(GCNN_EINVAL, "null context");
  GCNN_TRY(same_batch(c, b));
  GCNN_TRY(sync(c));
  const size_t G = b->n_graphs, N = b->n_nodes, E = b->n_edges;
  struct Item { void *dst; const void *src; size_t bytes; } items[] = {
      {node_off, b->node_off, (G + 1) * 4}, {graph_id, b->graph_id, N * 4}, {row_ptr, b->row_ptr, (N + 1) * 4},
      {col, b->col, E * 4}, {rev, b->rev, E * 4}, {deg, b->deg, N * 4}, {amp, b->amp, N * 4},
      {att, b->att, N * 4}, {types, b->types, N}, {y, b->y, G * 4}};
  for (auto &it : items)
    if (it.dst && it.bytes) GCNN_CUDA_TRY(cudaMemcpy(it.dst, it.src, it.bytes, cudaMemcpyDeviceToHost));
  return GCNN_OK;
}

// ---------------------------------------------------------------- training
int gcnn_forward(gcnn_ctx *c, const gcnn_batch *b, float *pred, int train) {
  if (!c) return set_error(GCNN_EINVAL, "null context");
  GCNN_TRY(same_batch(c, b));
  // same grid buckets as the captured step, so both give bit-identical results
  GCNN_TRY(ctx_forward(c, b->n_graphs, grid_nodes(c, b), grid_edges(c, b), train != 0));
  if (pred && b->n_graphs > 0)
    GCNN_CUDA_TRY(cudaMemcpyAsync(pred, c->pred, b->n_graphs * sizeof(float), cudaMemcpyDeviceToDevice, c->stream));
  c->have_fwd = train != 0;
  c->fwd_G = b->n_graphs; c->fwd_N = b->n_nodes; c->fwd_E = b->n_edges;
  return GCNN_OK;
}

int gcnn_backward(gcnn_ctx *c, const gcnn_batch *b, const float *dpred, double *loss_accum) {
  if (!c) return set_error(GCNN_EINVAL, "null context");
  GCNN_TRY(same_batch(c, b));
  if (!c->have_fwd || c->fwd_G != b->n_graphs || c->fwd_N != b->n_nodes)
    return set_error(GCNN_ESTATE, "backward needs a forward(train=1) on the same batch");
  return ctx_backward(c, b->n_graphs, grid_nodes(c, b), grid_edges(c, b), dpred, loss_accum);
}

int gcnn_set_loss_scale(gcnn_ctx *c, float graph_scale, float node_scale) {
  if (!c) return set_error(GCNN_EINVAL, "null context");
  if (!std::isfinite(graph_scale) || !std::isfinite(node_scale) || graph_scale < 0.f || node_scale < 0.f)
    return set_error(GCNN_EINVAL, "loss scales must be finite and >= 0");
  if (graph_scale != c->scale_host[0] || node_scale != c->scale_host[1]) {
    c->scale_pinned[0] = graph_scale;
    c->scale_pinned[1] = node_scale;
    GCNN_CUDA_TRY(cudaMemcpyAsync(c->loss_scale, c->scale_pinned, 2 * sizeof(float), cudaMemcpyHostToDevice,
                                  c->stream));
    // the pinned source must stay valid until the copy ran
    GCNN_CUDA_TRY(cudaStreamSynchronize(c->stream));
    c->scale_host[0] = graph_scale;
    c->scale_host[1] = node_scale;
  }
  return GCNN_OK;
}

int gcnn_grad_buckets(const gcnn_ctx *c, int32_t *n_buckets) {
  if (!c || !n_buckets) return set_error(GCNN_EINVAL, "null argument");
  *n_buckets = c->L + 2;
  return GCNN_OK;
}

int gcnn_grad_bucket(const gcnn_ctx *c, int32_t k, int64_t *offset, int64_t *count) {
  if (!c || !offset || !count) return set_error(GCNN_EINVAL, "null argument");
  const int64_t lb = (int64_t)c->T * c->H, le = lb + (int64_t)c->L * c->layer_size;
  if (k >= 0 && k < c->L) {
    *offset = lb + (int64_t)k * c->layer_size;
    *count = c->layer_size;
  } else if (k == c->L) {
    *offset = le;
    *count = c->P - le;
  } else if (k == c->L + 1) {
    *offset = 0;
    *count = lb;
  } else {
    return set_error(GCNN_EINVAL, "bucket %d out of range 0..%d", k, c->L + 1);
  }
  return GCNN_OK;
}

int gcnn_grad_wait(gcnn_ctx *c, int32_t k, void *stream) {
  if (!c) return set_error(GCNN_EINVAL, "null context");
  if (k < 0 || k > c->L + 1) return set_error(GCNN_EINVAL, "bucket %d out of range 0..%d", k, c->L + 1);
  GCNN_CUDA_TRY(cudaStreamWaitEvent(static_cast<cudaStream_t>(stream), c->grad_ev[std::min(k, c->L)], 0));
  return GCNN_OK;
}

int gcnn_grads_device(gcnn_ctx *c, float **grads) {
  if (!c || !grads) return set_error(GCNN_EINVAL, "null argument");
  *grads = c->grads;
  return GCNN_OK;
}

int gcnn_step(gcnn_ctx *c, float lr) {
  if (!c) return set_error(GCNN_EINVAL, "null context");
  GCNN_TRY(set_lr(c, lr));
  return ctx_step(c);
}

namespace {
// Replay (capturing it on first use) the graph of one training step on batch
// b: forward + backward, followed by AdamW when with_step.  Without the step,
// the backward's gradient-bucket events are external nodes of the graph.
// With range_st, the graph begins with the collation of graphs
// order[range_first .. + b->n_graphs) of the device-resident order (b then
// describes that batch before it is collated); a replay for another range
// of the same sizes updates the collation's two kernel nodes.
int run_step_graph(gcnn_ctx *c, const gcnn_batch *b, double *loss_accum, bool with_step,
                   const gcnn_store *range_st = nullptr, int64_t range_first = 0) {
  const int G = b->n_graphs;
  const int Ng = grid_nodes(c, b), Eg = grid_edges(c, b);
  // with profiling on, a separate graph carries event-record nodes around
  // every phase; each of its replays is synchronised and accumulated
  auto key = std::make_tuple(G, Ng, Eg, (const double *)loss_accum, c->prof_on, with_step, range_st != nullptr);
  auto it = c->graphs.find(key);
  // the collation's arguments name the store and the uploaded order's address
  // (gcnn_set_order may have replaced the order since the last launch)
  const int64_t *range_ids = range_st ? c->order_dev + range_first : nullptr;
  if (it != c->graphs.end() && range_st &&
      (it->second.range_store != range_st || it->second.range_ids != range_ids)) {
    GCNN_TRY(ctx_range_update(c, range_st, range_first, G, it->second.exec, it->second.scan_node,
                              it->second.graph_node));
    it->second.range_store = range_st;
    it->second.range_ids = range_ids;
  }
  if (it == c->graphs.end()) {
    // capture on the context's private stream (the legacy default stream
    // cannot be captured); the graph is then launched on the caller's stream
    cudaGraph_t graph = nullptr;
    GCNN_CUDA_TRY(cudaStreamSynchronize(c->stream));
    cudaStream_t user = c->stream;
    c->stream = c->cap_stream;
    c->capturing = true;
    c->cap_grad_events = !with_step;
    c->cap_ev.clear();
    cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      c->stream = user;
      c->capturing = false;
      c->cap_grad_events = false;
      return set_error(GCNN_ECUDA, "begin capture: %s", cudaGetErrorString(e));
    }
    c->fuse_head = true;
    c->fuse_step = with_step;
    int rc = range_st ? ctx_range_launch(c, range_st, range_first, G) : GCNN_OK;
    if (rc == GCNN_OK) rc = ctx_forward(c, G, Ng, Eg, true);
    if (rc == GCNN_OK) rc = ctx_backward(c, G, Ng, Eg, nullptr, loss_accum);
    c->fuse_head = false;
    if (rc == GCNN_OK && with_step) rc = ctx_step(c);
    c->fuse_step = false;
    e = cudaStreamEndCapture(c->stream, &graph);
    c->stream = user;
    c->capturing = false;
    c->cap_grad_events = false;
    std::vector<gcnn_ctx::ProfEvent> ev;
    ev.swap(c->cap_ev);
    auto drop_events = [&ev] {
      for (auto &pe : ev) {
        cudaEventDestroy(pe.a);
        cudaEventDestroy(pe.b);
      }
    };
    if (rc != GCNN_OK) {
      if (graph) cudaGraphDestroy(graph);
      drop_events();
      cudaGetLastError();  // a failed capture must not fail later calls
      return rc;
    }
    if (e != cudaSuccess) {
      drop_events();
      cudaGetLastError();
      return set_error(GCNN_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
    }
    size_t n_nodes = 0;
    cudaGraphGetNodes(graph, nullptr, &n_nodes);
    std::vector<cudaGraphNode_t> nodes(n_nodes);
    int kernels = 0;
    cudaGraphNode_t scan_node = nullptr, graph_node = nullptr;
    if (n_nodes && cudaGraphGetNodes(graph, nodes.data(), &n_nodes) == cudaSuccess) {
      for (auto nd : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nd, &t) != cudaSuccess || t != cudaGraphNodeTypeKernel) continue;
        ++kernels;
        cudaKernelNodeParams kp{};
        if (range_st && cudaGraphKernelNodeGetParams(nd, &kp) == cudaSuccess) {
          const int kind = collate_node_kind(kp.func);
          if (kind == 1 || kind == 3) scan_node = nd;
          if (kind == 2) graph_node = nd;
        }
      }
    }
    cudaGetLastError();
    // one launch for a batch of at most 1024 graphs, a scan and a per-graph launch beyond
    if (range_st && (!scan_node || (G > kCollateOneLaunchGraphs && !graph_node))) {
      cudaGraphDestroy(graph);
      drop_events();
      return set_error(GCNN_ECUDA, "train step: the captured collation nodes were not found");
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    // a graph whose collation nodes are updated later stays alive with its exec
    if (!range_st || e != cudaSuccess) {
      cudaGraphDestroy(graph);
      graph = nullptr;
    }
    if (e != cudaSuccess) {
      drop_events();
      return set_error(GCNN_ECUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
    }
    gcnn_ctx::Graph entry{exec, kernels, std::move(ev)};
    entry.graph = graph;
    entry.scan_node = scan_node;
    entry.graph_node = graph_node;
    entry.range_store = range_st;
    entry.range_ids = range_ids;
    it = c->graphs.emplace(key, std::move(entry)).first;
  }
  GCNN_CUDA_TRY(cudaGraphLaunch(it->second.exec, c->stream));
  bool tl_on;
  {
    std::lock_guard<std::mutex> lock(g_tl_mu);
    tl_on = g_tl.buf != nullptr;
  }
  if (tl_on) GCNN_TRY(launch_step_end(c->stream));
  if (!it->second.ev.empty()) {
    GCNN_CUDA_TRY(cudaStreamSynchronize(c->stream));
    for (auto &pe : it->second.ev) {
      float t = 0.f;
      GCNN_CUDA_TRY(cudaEventElapsedTime(&t, pe.a, pe.b));
      c->prof_ms[pe.phase] += t;
      c->prof_n[pe.phase] += 1;
    }
  }
  c->last_step_kernels = it->second.kernels;
  c->have_fwd = true;
  c->fwd_G = b->n_graphs; c->fwd_N = b->n_nodes; c->fwd_E = b->n_edges;
  return GCNN_OK;
}
}  // namespace

int gcnn_train_step(gcnn_ctx *c, const gcnn_batch *b, float lr, double *loss_accum) {
  if (!c) return set_error(GCNN_EINVAL, "null context");
  GCNN_TRY(same_batch(c, b));
  GCNN_TRY(set_lr(c, lr));
  return run_step_graph(c, b, loss_accum, true);
}

int gcnn_train_step_range(gcnn_ctx *c, const gcnn_store *st, int64_t first, int32_t count, float lr,
                          double *loss_accum, gcnn_batch *out) {
  if (!c || !st || count < 1) return set_error(GCNN_EINVAL, "train_step_range: bad arguments");
  gcnn_batch b{};
  GCNN_TRY(ctx_range_prepare(c, st, first, count, &b));
  GCNN_TRY(set_lr(c, lr));
  c->have_fwd = false;
  GCNN_TRY(run_step_graph(c, &b, loss_accum, true, st, first));
  if (out) *out = b;
  return GCNN_OK;
}

int gcnn_forward_backward(gcnn_ctx *c, const gcnn_batch *b, double *loss_accum) {
  if (!c) return set_error(GCNN_EINVAL, "null context");
  GCNN_TRY(same_batch(c, b));
  return run_step_graph(c, b, loss_accum, false);
}

int gcnn_get_activation(gcnn_ctx *c, int32_t layer, float *dst, int64_t n) {
  if (!c || !dst || layer < 0 || layer > c->L) return set_error(GCNN_EINVAL, "get_activation: bad arguments");
  if (n != (int64_t)c->fwd_N * c->H) return set_error(GCNN_EINVAL, "get_activation: expected N*H floats");
  GCNN_CUDA_TRY(cudaMemcpyAsync(dst, c->xs + (size_t)layer * c->Nc * c->H, n * sizeof(float),
                                cudaMemcpyDeviceToHost, c->stream));
  return sync(c);
}

// ---------------------------------------------------------------- timing
int gcnn_get_node_predictions(gcnn_ctx *c, float *dst, int64_t n) {
  if (!c || !dst) return set_error(GCNN_EINVAL, "get_node_predictions: bad arguments");
  if (!c->predn) return set_error(GCNN_ESTATE, "get_node_predictions: the model has no node-level head");
  if (n != (int64_t)c->fwd_N) return set_error(GCNN_EINVAL, "get_node_predictions: expected N floats");
  GCNN_CUDA_TRY(cudaMemcpyAsync(dst, c->predn, n * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
  return sync(c);
}

int gcnn_profile_enable(gcnn_ctx *c, int enable) {
  if (!c) return set_error(GCNN_EINVAL, "null context");
  c->prof_on = enable != 0;
  return GCNN_OK;
}

int gcnn_profile_read(gcnn_ctx *c, double *ms, int64_t *launches) {
  if (!c || !ms || !launches) return set_error(GCNN_EINVAL, "null argument");
  GCNN_TRY(sync(c));
  for (int q = 0; q < GCNN_NPHASE; ++q) {
    ms[q] = c->prof_ms[q];
    launches[q] = c->prof_n[q];
    c->prof_ms[q] = 0.0;
    c->prof_n[q] = 0;
  }
  for (size_t k = 0; k < c->prof_used; ++k) {
    float t = 0.f;
    GCNN_CUDA_TRY(cudaEventElapsedTime(&t, c->prof_ev[2 * k], c->prof_ev[2 * k + 1]));
    ms[c->prof_cls[k]] += t;
    launches[c->prof_cls[k]] += 1;
  }
  c->prof_used = 0;
  return GCNN_OK;
}

int gcnn_memory(const gcnn_ctx *c, int64_t *arena_bytes) {
  if (!c || !arena_bytes) return set_error(GCNN_EINVAL, "null argument");
  *arena_bytes = (int64_t)c->dbytes;
  return GCNN_OK;
}

int gcnn_step_kernel_count(gcnn_ctx *c, int32_t *n) {
  if (!c || !n) return set_error(GCNN_EINVAL, "null argument");
  *n = c->last_step_kernels;
  return GCNN_OK;
}

int gcnn_timeline_enable(gcnn_ctx *c, int32_t capacity) {
  if (!c || capacity < 0) return set_error(GCNN_EINVAL, "timeline: null context or negative capacity");
  std::lock_guard<std::mutex> lock(g_tl_mu);
  GCNN_CUDA_TRY(cudaDeviceSynchronize());
  if (g_tl.buf) {
    GCNN_TRY(timeline_attach_all(nullptr));
    cudaFree(g_tl.buf);
    g_tl = TimelineHost{};
  }
  if (capacity == 0) return GCNN_OK;
  TimelineHost h;
  h.cap = (unsigned)capacity;
  h.off_t = 256;
  h.off_id = h.off_t + sizeof(unsigned long long) * h.cap;
  const size_t bytes = h.off_id + sizeof(unsigned) * h.cap;
  if (cudaMalloc(&h.buf, bytes) != cudaSuccess) {
    cudaGetLastError();
    return set_error(GCNN_ENOMEM, "timeline: cannot allocate %zu bytes", bytes);
  }
  const Timeline head{0u, h.cap, reinterpret_cast<unsigned long long *>(h.buf + h.off_t),
                      reinterpret_cast<unsigned *>(h.buf + h.off_id)};
  int rc = cudaMemcpy(h.buf, &head, sizeof(head), cudaMemcpyHostToDevice) == cudaSuccess
               ? GCNN_OK
               : set_error(GCNN_ECUDA, "timeline: header copy failed");
  if (rc == GCNN_OK) rc = timeline_attach_all(h.buf);
  if (rc != GCNN_OK) {
    timeline_attach_all(nullptr);
    cudaFree(h.buf);
    return rc;
  }
  g_tl = h;
  return GCNN_OK;
}

int gcnn_gemm_study(int32_t n_atoms, int32_t hidden, int32_t mode, double *rows, int32_t max_rows,
                    int32_t *n_rows) {
  if (!n_rows) return set_error(GCNN_EINVAL, "gemm_study: null argument");
  int n = 0;
  const int rc = gemm_tc_study(n_atoms, hidden, mode, rows, max_rows, &n);
  *n_rows = n;
  return rc;
}

int gcnn_ffma_peak(int32_t iters, double *tflops) {
  if (iters < 1 || !tflops) return set_error(GCNN_EINVAL, "ffma_peak: iters must be >= 1");
  float *out = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = GCNN_OK;
  double flop = 0.0;
  if (cudaMalloc(&out, 4096 * sizeof(float)) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess)
    rc = set_error(GCNN_ECUDA, "ffma_peak: setup failed");
  if (rc == GCNN_OK) rc = launch_ffma_peak(iters, out, s, &flop);  // warm-up
  if (rc == GCNN_OK && cudaEventRecord(e0, s) != cudaSuccess) rc = set_error(GCNN_ECUDA, "ffma_peak: event");
  if (rc == GCNN_OK) rc = launch_ffma_peak(iters, out, s, &flop);
  if (rc == GCNN_OK && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess))
    rc = set_error(GCNN_ECUDA, "ffma_peak: timing failed");
  float ms = 0.f;
  if (rc == GCNN_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = set_error(GCNN_ECUDA, "ffma_peak: timing");
  if (rc == GCNN_OK) *tflops = ms > 0.f ? flop / (ms * 1e-3) / 1e12 : 0.0;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  if (out) cudaFree(out);
  return rc;
}

int gcnn_timeline_read(gcnn_ctx *c, int32_t *ids, int64_t *t_ns, int32_t max, int32_t *n) {
  if (!c || !n || max < 0 || (max > 0 && (!ids || !t_ns))) return set_error(GCNN_EINVAL, "timeline: bad arguments");
  std::lock_guard<std::mutex> lock(g_tl_mu);
  if (!g_tl.buf) return set_error(GCNN_ESTATE, "timeline is not enabled");
  GCNN_CUDA_TRY(cudaDeviceSynchronize());
  unsigned count = 0;
  GCNN_CUDA_TRY(cudaMemcpy(&count, g_tl.buf, sizeof(count), cudaMemcpyDeviceToHost));
  const unsigned k = std::min<unsigned>(std::min(count, g_tl.cap), (unsigned)max);
  if (k > 0) {
    std::vector<unsigned long long> t(k);
    std::vector<unsigned> id(k);
    GCNN_CUDA_TRY(cudaMemcpy(t.data(), g_tl.buf + g_tl.off_t, sizeof(unsigned long long) * k, cudaMemcpyDeviceToHost));
    GCNN_CUDA_TRY(cudaMemcpy(id.data(), g_tl.buf + g_tl.off_id, sizeof(unsigned) * k, cudaMemcpyDeviceToHost));
    for (unsigned q = 0; q < k; ++q) {
      ids[q] = (int32_t)id[q];
      t_ns[q] = (int64_t)t[q];
    }
  }
  GCNN_CUDA_TRY(cudaMemset(g_tl.buf, 0, sizeof(unsigned)));
  *n = (int32_t)k;
  return GCNN_OK;
}

// ---------------------------------------------------------------- operators
int gcnn_op_aggregate_fwd(int32_t n_nodes, int32_t hidden, const int32_t *row_ptr, const int32_t *col,
                          const float *PQ, float *agg, float std_eps, void *stream) {
  if (n_nodes < 0 || hidden <= 0 || hidden % 4 || (n_nodes > 0 && (!row_ptr || !col || !PQ || !agg)))
    return set_error(GCNN_EINVAL, "aggregate_fwd: bad arguments (hidden must be a multiple of 4)");
  if ((reinterpret_cast<uintptr_t>(PQ) | reinterpret_cast<uintptr_t>(agg)) % 16)
    return set_error(GCNN_EINVAL, "aggregate_fwd: PQ and agg must be 16-byte aligned");
  return launch_aggregate_fwd(n_nodes, hidden, DevDims{nullptr}, row_ptr, col, PQ, agg, std_eps, nullptr,
                              static_cast<cudaStream_t>(stream));
}

int gcnn_op_aggregate_bwd(int32_t n_nodes, int32_t n_edges, int32_t hidden, const int32_t *row_ptr,
                          const int32_t *col, const int32_t *rev, const float *PQ, const float *agg,
                          const float *dagg, float *dPQ, float *scratch, float std_eps, void *stream) {
  if (n_nodes < 0 || n_edges < 0 || hidden <= 0 || hidden % 4 ||
      (n_nodes > 0 && (!row_ptr || !col || !rev || !PQ || !agg || !dagg || !dPQ || (n_edges > 0 && !scratch))))
    return set_error(GCNN_EINVAL, "aggregate_bwd: bad arguments (hidden must be a multiple of 4)");
  if ((reinterpret_cast<uintptr_t>(PQ) | reinterpret_cast<uintptr_t>(agg) | reinterpret_cast<uintptr_t>(dagg) |
       reinterpret_cast<uintptr_t>(dPQ) | reinterpret_cast<uintptr_t>(scratch)) % 16)
    return set_error(GCNN_EINVAL, "aggregate_bwd: float buffers must be 16-byte aligned");
  return launch_aggregate_bwd(n_nodes, n_edges, hidden, DevDims{nullptr}, row_ptr, col, rev, PQ, agg, dagg, dPQ,
                              scratch, std_eps, nullptr, static_cast<cudaStream_t>(stream));
}

int gcnn_op_aggregate_bwd_graphs(int32_t n_graphs, int32_t n_nodes, int32_t n_edges, int32_t hidden,
                                 const int32_t *node_off, const int32_t *row_ptr, const int32_t *col,
                                 const int32_t *rev, const float *PQ, const float *agg, const float *dagg,
                                 float *dPQ, float *scratch, float std_eps, void *stream) {
  if (n_graphs < 0 || n_nodes < 0 || n_edges < 0 || hidden <= 0 || hidden % 4 ||
      (n_nodes > 0 && (!node_off || !row_ptr || !col || !rev || !PQ || !agg || !dagg || !dPQ || !scratch)))
    return set_error(GCNN_EINVAL, "aggregate_bwd_graphs: bad arguments (hidden must be a multiple of 4)");
  if ((reinterpret_cast<uintptr_t>(PQ) | reinterpret_cast<uintptr_t>(agg) | reinterpret_cast<uintptr_t>(dagg) |
       reinterpret_cast<uintptr_t>(dPQ) | reinterpret_cast<uintptr_t>(scratch)) % 16)
    return set_error(GCNN_EINVAL, "aggregate_bwd_graphs: float buffers must be 16-byte aligned");
  // the chunk partition follows the per-edge part of scratch
  int *chunks = reinterpret_cast<int *>(scratch + (size_t)n_edges * hidden);
  return launch_aggregate_bwd_graphs(n_graphs, n_nodes, n_edges, hidden, DevDims{nullptr}, node_off, row_ptr, col, rev,
                                     PQ, agg, dagg, dPQ, scratch, chunks, std_eps, nullptr,
                                     static_cast<cudaStream_t>(stream));
}

int gcnn_op_pool_fwd(int32_t n_graphs, int32_t hidden, const int32_t *node_off, const float *x, float *pooled,
                     void *stream) {
  if (n_graphs < 0 || hidden <= 0 || hidden % 4 || (n_graphs > 0 && (!node_off || !x || !pooled)))
    return set_error(GCNN_EINVAL, "pool_fwd: bad arguments (hidden must be a multiple of 4)");
  return launch_pool_fwd(n_graphs, hidden, DevDims{nullptr}, node_off, x, pooled, static_cast<cudaStream_t>(stream));
}

int gcnn_op_pool_bwd(int32_t n_graphs, int32_t n_nodes, int32_t hidden, const int32_t *node_off,
                     const int32_t *graph_id, const float *dpooled, float *dx, void *stream) {
  if (n_graphs < 0 || n_nodes < 0 || hidden <= 0 || hidden % 4 ||
      (n_nodes > 0 && (!node_off || !graph_id || !dpooled || !dx)))
    return set_error(GCNN_EINVAL, "pool_bwd: bad arguments (hidden must be a multiple of 4)");
  return launch_pool_bwd(n_graphs, n_nodes, hidden, DevDims{nullptr}, node_off, graph_id, dpooled, dx,
                         static_cast<cudaStream_t>(stream));
}

}  // extern "C"
