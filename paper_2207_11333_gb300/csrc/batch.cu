// Host side of batch collation: the per-batch read of the store (the paper's
// data-loading phase, Sec. 4 and Fig. 5), either straight from a device-
// resident store or through pinned staging memory and one host-to-device copy.
#include <cstring>
#include <vector>

#include "context.h"

namespace gcnn {
namespace {

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

void fill_batch(const gcnn_ctx *c, int G, int64_t N, int64_t E, gcnn_batch *out) {
  out->n_graphs = G;
  out->n_nodes = (int32_t)N;
  out->n_edges = (int32_t)E;
  out->reserved = 0;
  out->node_off = c->bb.node_off;
  out->edge_off = c->bb.edge_off;
  out->graph_id = c->bb.graph_id;
  out->row_ptr = c->bb.row_ptr;
  out->col = c->bb.col;
  out->rev = c->bb.rev;
  out->deg = c->bb.deg;
  out->amp = c->bb.amp;
  out->att = c->bb.att;
  out->types = c->bb.types;
  out->y = c->bb.y;
  out->edge_attr = c->cfg.edge_features > 0 ? c->bb.eattr : nullptr;
  out->node_y = c->bb.ynode;
}

int check_features(const gcnn_ctx *c, const gcnn_store *st) {
  if (st->F != c->cfg.edge_features)
    return set_error(GCNN_EINVAL, "store has %d bond features per edge, the model %d", st->F, c->cfg.edge_features);
  if (c->cfg.node_head && !st->ynode)
    return set_error(GCNN_EINVAL, "the model has a node-level head but the store carries no node targets");
  return GCNN_OK;
}

int check_caps(const gcnn_ctx *c, int64_t G, int64_t N, int64_t E) {
  if (G > c->Gc || N > c->Nc || E > c->Ec)
    return set_error(GCNN_EINVAL, "batch (%lld graphs, %lld nodes, %lld edges) exceeds capacity (%d, %d, %d)",
                     (long long)G, (long long)N, (long long)E, c->Gc, c->Nc, c->Ec);
  return GCNN_OK;
}

// Wait until the pinned staging buffer q is no longer read by a pending copy.
int claim_stage(gcnn_ctx *c, int q) {
  if (c->stage_used[q]) GCNN_CUDA_TRY(cudaEventSynchronize(c->stage_ev[q]));
  c->stage_used[q] = false;
  return GCNN_OK;
}

// Gather n graphs into a mini-store in pinned staging memory (node_ptr,
// edge_ptr, y, types, edges, bond features, node targets), copy it to the
// device in one transfer and collate it.  sizes(g) gives graph g's (nodes,
// edges); fill(g, types, edges, y, attr, ynode) writes its slices at the
// given destinations (ynode is nullptr without the node head).
template <class Sizes, class Fill>
int collate_staged(gcnn_ctx *c, int32_t n, int64_t N, int64_t E, int F, Sizes sizes, Fill fill, gcnn_batch *out) {
  const int q = c->stage_i;
  c->stage_i ^= 1;
  GCNN_TRY(claim_stage(c, q));
  char *h = c->stage_host[q];
  size_t o = 0;
  const size_t o_np = o; o = align_up(o + 8 * (size_t)(n + 1), 16);
  const size_t o_ep = o; o = align_up(o + 8 * (size_t)(n + 1), 16);
  const size_t o_y = o;  o = align_up(o + 4 * (size_t)n, 16);
  const size_t o_t = o;  o = align_up(o + (size_t)N, 16);
  const size_t o_e = o;  o = align_up(o + 2 * (size_t)E, 16);
  const size_t o_a = o;  o = align_up(o + 4 * (size_t)E * F, 16);
  const bool yn_on = c->bb.ynode != nullptr;
  const size_t o_yn = o; o = align_up(o + (yn_on ? 4 * (size_t)N : 0), 16);
  if (o > c->stage_bytes) return set_error(GCNN_EINVAL, "staging buffer too small");
  int64_t *np = reinterpret_cast<int64_t *>(h + o_np), *ep = reinterpret_cast<int64_t *>(h + o_ep);
  float *y = reinterpret_cast<float *>(h + o_y), *at = reinterpret_cast<float *>(h + o_a);
  float *yn = reinterpret_cast<float *>(h + o_yn);
  uint8_t *ty = reinterpret_cast<uint8_t *>(h + o_t), *ed = reinterpret_cast<uint8_t *>(h + o_e);
  np[0] = 0;
  ep[0] = 0;
  for (int32_t g = 0; g < n; ++g) {
    int64_t nn = 0, ne = 0;
    sizes(g, &nn, &ne);
    if (np[g] + nn > N || ep[g] + ne > E) return set_error(GCNN_EINVAL, "collate: graph sizes changed while staging");
    fill(g, ty + np[g], ed + 2 * ep[g], y + g, at + ep[g] * F, yn_on ? yn + np[g] : nullptr);
    np[g + 1] = np[g] + nn;
    ep[g + 1] = ep[g] + ne;
  }
  GCNN_CUDA_TRY(cudaMemcpyAsync(c->stage_dev, h, o, cudaMemcpyHostToDevice, c->stream));
  GCNN_CUDA_TRY(cudaEventRecord(c->stage_ev[q], c->stream));
  c->stage_used[q] = true;
  const char *d = c->stage_dev;
  StoreView v{reinterpret_cast<const int64_t *>(d + o_np), reinterpret_cast<const int64_t *>(d + o_ep),
              reinterpret_cast<const uint8_t *>(d + o_t), reinterpret_cast<const uint8_t *>(d + o_e),
              reinterpret_cast<const float *>(d + o_y), F > 0 ? reinterpret_cast<const float *>(d + o_a) : nullptr, F,
              yn_on ? reinterpret_cast<const float *>(d + o_yn) : nullptr};
  {
    PhaseScope ps(c, GCNN_PHASE_COLLATE);
    GCNN_TRY(launch_collate(n, nullptr, v, c->bb, c->scal_tab, c->Nc, c->Ec, c->err, c->stream));
  }
  fill_batch(c, n, N, E, out);
  c->have_fwd = false;
  return GCNN_OK;
}

}  // namespace

int ctx_collate(gcnn_ctx *c, const gcnn_store *st, const int64_t *ids, int32_t n, gcnn_batch *out) {
  int64_t N = 0, E = 0;
  GCNN_TRY(check_features(c, st));
  GCNN_TRY(check_caps(c, n, 0, 0));
  GCNN_TRY(store_batch_size(st, ids, n, &N, &E));
  GCNN_TRY(check_caps(c, n, N, E));
  if (!st->dev) {
    // gather the graphs' slices into a mini-store in pinned memory, one copy
    const int F = st->F;
    auto sizes = [&](int32_t g, int64_t *nn, int64_t *ne) {
      const int64_t id = ids[g];
      *nn = st->node_ptr[id + 1] - st->node_ptr[id];
      *ne = st->edge_ptr[id + 1] - st->edge_ptr[id];
    };
    auto fill = [&](int32_t g, uint8_t *ty, uint8_t *ed, float *y, float *at, float *yn) {
      const int64_t id = ids[g];
      const int64_t nn = st->node_ptr[id + 1] - st->node_ptr[id], ne = st->edge_ptr[id + 1] - st->edge_ptr[id];
      memcpy(ty, st->types + st->node_ptr[id], (size_t)nn);
      memcpy(ed, st->edges + 2 * st->edge_ptr[id], 2 * (size_t)ne);
      if (F > 0) memcpy(at, st->eattr + st->edge_ptr[id] * F, sizeof(float) * (size_t)ne * F);
      if (yn) memcpy(yn, st->ynode + st->node_ptr[id], sizeof(float) * (size_t)nn);
      *y = st->y[id];
    };
    return collate_staged(c, n, N, E, F, sizes, fill, out);
  }
  // resident store: only the graph ids travel
  const int q = c->stage_i;
  c->stage_i ^= 1;
  GCNN_TRY(claim_stage(c, q));
  char *h = c->stage_host[q];
  memcpy(h, ids, sizeof(int64_t) * (size_t)n);
  if (n > 0)
    GCNN_CUDA_TRY(cudaMemcpyAsync(c->ids_dev, h, sizeof(int64_t) * (size_t)n, cudaMemcpyHostToDevice, c->stream));
  GCNN_CUDA_TRY(cudaEventRecord(c->stage_ev[q], c->stream));
  c->stage_used[q] = true;
  {
    PhaseScope ps(c, GCNN_PHASE_COLLATE);
    GCNN_TRY(launch_collate(n, c->ids_dev, store_device_view(st), c->bb, c->scal_tab, c->Nc, c->Ec, c->err,
                            c->stream));
  }
  fill_batch(c, n, N, E, out);
  c->have_fwd = false;
  return GCNN_OK;
}

int ctx_collate_files(gcnn_ctx *c, const char *const *paths, int32_t n, gcnn_batch *out) {
  // one read per file, in order (the per-graph-file loading path)
  std::vector<GraphFile> files((size_t)n);
  int64_t N = 0, E = 0;
  if (c->cfg.node_head) return set_error(GCNN_EINVAL, "per-graph files carry no node targets (node head)");
  GCNN_TRY(check_caps(c, n, 0, 0));
  for (int32_t g = 0; g < n; ++g) {
    GCNN_TRY(read_graph_file(paths[g], &files[(size_t)g]));
    if (files[(size_t)g].F != c->cfg.edge_features)
      return set_error(GCNN_EINVAL, "%s has %d bond features per edge, the model %d", paths[g], files[(size_t)g].F,
                       c->cfg.edge_features);
    N += files[(size_t)g].n;
    E += files[(size_t)g].e;
  }
  GCNN_TRY(check_caps(c, n, N, E));
  const int F = c->cfg.edge_features;
  auto sizes = [&](int32_t g, int64_t *nn, int64_t *ne) {
    *nn = files[(size_t)g].n;
    *ne = files[(size_t)g].e;
  };
  auto fill = [&](int32_t g, uint8_t *ty, uint8_t *ed, float *y, float *at, float *) {
    const GraphFile &f = files[(size_t)g];
    memcpy(ty, f.types, (size_t)f.n);
    memcpy(ed, f.edges, 2 * (size_t)f.e);
    if (F > 0) memcpy(at, f.attr, sizeof(float) * (size_t)f.e * F);
    *y = f.y;
  };
  return collate_staged(c, n, N, E, F, sizes, fill, out);
}

int ctx_range_prepare(gcnn_ctx *c, const gcnn_store *st, int64_t first, int32_t count, gcnn_batch *out) {
  if (!c->order_dev || c->order_store != st) return set_error(GCNN_ESTATE, "collate_range: call gcnn_set_order first");
  if (!st->dev) return set_error(GCNN_ESTATE, "collate_range needs a device-resident store");
  if (first < 0 || first + count > (int64_t)c->order_host.size())
    return set_error(GCNN_EINVAL, "collate_range: range outside the order");
  int64_t N = 0, E = 0;
  GCNN_TRY(check_features(c, st));
  GCNN_TRY(check_caps(c, count, 0, 0));
  GCNN_TRY(store_batch_size(st, c->order_host.data() + first, count, &N, &E));
  GCNN_TRY(check_caps(c, count, N, E));
  fill_batch(c, count, N, E, out);
  return GCNN_OK;
}

int ctx_range_launch(gcnn_ctx *c, const gcnn_store *st, int64_t first, int32_t count) {
  PhaseScope ps(c, GCNN_PHASE_COLLATE);
  return launch_collate(count, c->order_dev + first, store_device_view(st), c->bb, c->scal_tab, c->Nc, c->Ec, c->err,
                        c->stream);
}

int ctx_range_update(gcnn_ctx *c, const gcnn_store *st, int64_t first, int32_t count, cudaGraphExec_t exec,
                     cudaGraphNode_t scan_node, cudaGraphNode_t graph_node) {
  return collate_set_nodes(exec, scan_node, graph_node, count, c->order_dev + first, store_device_view(st), c->bb,
                           c->scal_tab, c->Nc, c->Ec, c->err);
}

int ctx_collate_range(gcnn_ctx *c, const gcnn_store *st, int64_t first, int32_t count, gcnn_batch *out) {
  GCNN_TRY(ctx_range_prepare(c, st, first, count, out));
  GCNN_TRY(ctx_range_launch(c, st, first, count));
  c->have_fwd = false;
  return GCNN_OK;
}

}  // namespace gcnn
