// Packed graph store: the whole file in pinned host memory, validated once,
// optionally mirrored in device memory ("resident" mode).  One global array
// per graph attribute, like the paper's ADIOS schema (Sec. 4, Table 1), in a
// single file instead of per-graph files.
#include <cmath>
#include <cstdint>
#include <cstdarg>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "store.h"

namespace gcnn {

namespace {
thread_local char g_msg[512] = "no error";
}

int set_error(int code, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
  va_end(ap);
  return code;
}

const char *last_error() { return g_msg; }

namespace {

struct Header {
  char magic[8];
  uint32_t version, n_types;
  int64_t G, N, E, o_node_ptr, o_edge_ptr, o_types, o_edges, o_y, size;
  int64_t F, o_eattr;  // version 2: bond features per edge and their offset
  int64_t o_ynode;     // version 2: node-level targets (0: none)
};
static_assert(sizeof(Header) == 112, "store header layout");
constexpr int kMaxEdgeFeatures = 16;

bool range_ok(int64_t off, int64_t bytes, int64_t size) {
  return off >= 0 && bytes >= 0 && off <= size && bytes <= size - off;
}

int validate(const gcnn_store *st) {
  if (st->node_ptr[0] != 0 || st->edge_ptr[0] != 0 || st->node_ptr[st->G] != st->N ||
      st->edge_ptr[st->G] != st->E)
    return set_error(GCNN_EFORMAT, "store: offset arrays do not span the data");
  std::vector<int> adj(256 * 256, 0);  // 1 + store index of edge (s, d)
  for (int64_t g = 0; g < st->G; ++g) {
    const int64_t n = st->node_ptr[g + 1] - st->node_ptr[g];
    const int64_t e = st->edge_ptr[g + 1] - st->edge_ptr[g];
    if (n < 1 || n > kMaxGraphNodes)
      return set_error(GCNN_EFORMAT, "store: graph %lld has %lld nodes (1..%d allowed)", (long long)g,
                       (long long)n, kMaxGraphNodes);
    if (e < 0 || e > kMaxGraphEdges)
      return set_error(GCNN_EFORMAT, "store: graph %lld has %lld edges (<= %d allowed)", (long long)g,
                       (long long)e, kMaxGraphEdges);
    const uint8_t *ed = st->edges + 2 * st->edge_ptr[g];
    for (int64_t k = 0; k < e; ++k) {
      const int s = ed[2 * k], d = ed[2 * k + 1];
      if (s >= n || d >= n)
        return set_error(GCNN_EFORMAT, "store: graph %lld edge %lld has a node id >= %lld", (long long)g,
                         (long long)k, (long long)n);
      adj[s * 256 + d] = (int)k + 1;
    }
    bool sym = true, same = true;
    for (int64_t k = 0; k < e; ++k) {
      const int s = ed[2 * k], d = ed[2 * k + 1];
      const int r = adj[d * 256 + s];
      if (!r) {
        sym = false;
      } else if (st->F > 0) {  // both directions of a bond carry the same features
        const float *a = st->eattr + (st->edge_ptr[g] + k) * st->F;
        const float *b = st->eattr + (st->edge_ptr[g] + r - 1) * st->F;
        if (memcmp(a, b, sizeof(float) * st->F) != 0) same = false;
      }
    }
    for (int64_t k = 0; k < e; ++k) adj[ed[2 * k] * 256 + ed[2 * k + 1]] = 0;
    if (!sym)
      return set_error(GCNN_EFORMAT, "store: graph %lld is not stored in both directions", (long long)g);
    if (!same)
      return set_error(GCNN_EFORMAT, "store: graph %lld has a bond whose two directions differ in features",
                       (long long)g);
    const uint8_t *ty = st->types + st->node_ptr[g];
    for (int64_t v = 0; v < n; ++v)
      if (ty[v] >= st->n_types)
        return set_error(GCNN_EFORMAT, "store: graph %lld has atom type %d >= %u", (long long)g, ty[v],
                         st->n_types);
  }
  return GCNN_OK;
}

}  // namespace

int store_open(const char *path, gcnn_store **out) {
  if (!path || !out) return set_error(GCNN_EINVAL, "store_open: null argument");
  *out = nullptr;
  FILE *f = fopen(path, "rb");
  if (!f) return set_error(GCNN_EINVAL, "store_open: cannot open %s", path);
  Header h;
  if (fread(&h, sizeof(h), 1, f) != 1 || memcmp(h.magic, "GCNNPKD1", 8) != 0 || (h.version != 1 && h.version != 2)) {
    fclose(f);
    return set_error(GCNN_EFORMAT, "store_open: %s is not a packed graph store (v1 or v2)", path);
  }
  if (h.version == 1) {
    h.F = 0;
    h.o_eattr = 0;
    h.o_ynode = 0;
  }
  fseek(f, 0, SEEK_END);
  const long long fsize = ftell(f);
  if (h.size != fsize || h.G < 0 || h.N < 0 || h.E < 0 || h.n_types < 1 || h.n_types > 16 ||
      !range_ok(h.o_node_ptr, 8 * (h.G + 1), h.size) || !range_ok(h.o_edge_ptr, 8 * (h.G + 1), h.size) ||
      !range_ok(h.o_types, h.N, h.size) || !range_ok(h.o_edges, 2 * h.E, h.size) ||
      !range_ok(h.o_y, 4 * h.G, h.size) || h.o_node_ptr % 8 || h.o_edge_ptr % 8 || h.o_y % 4 || h.F < 0 ||
      h.F > kMaxEdgeFeatures || (h.F > 0 && (h.E > INT64_MAX / (4 * h.F) || !range_ok(h.o_eattr, 4 * h.E * h.F, h.size) ||
                                             h.o_eattr % 16)) ||
      (h.o_ynode != 0 && (!range_ok(h.o_ynode, 4 * h.N, h.size) || h.o_ynode % 4))) {
    fclose(f);
    return set_error(GCNN_EFORMAT, "store_open: inconsistent header in %s", path);
  }
  gcnn_store *st = new gcnn_store();
  st->bytes = (size_t)h.size;
  if (cudaMallocHost(&st->host, st->bytes) == cudaSuccess) {
    st->pinned = true;
  } else {
    cudaGetLastError();
    st->host = malloc(st->bytes);
    st->pinned = false;
  }
  if (!st->host) {
    fclose(f);
    delete st;
    return set_error(GCNN_ENOMEM, "store_open: cannot allocate %zu bytes", (size_t)h.size);
  }
  fseek(f, 0, SEEK_SET);
  const size_t got = fread(st->host, 1, st->bytes, f);
  fclose(f);
  char *b = static_cast<char *>(st->host);
  st->G = h.G; st->N = h.N; st->E = h.E; st->n_types = h.n_types;
  st->off_node_ptr = h.o_node_ptr; st->off_edge_ptr = h.o_edge_ptr; st->off_types = h.o_types;
  st->off_edges = h.o_edges; st->off_y = h.o_y;
  st->F = (int32_t)h.F; st->off_eattr = h.o_eattr; st->off_ynode = h.o_ynode;
  st->node_ptr = reinterpret_cast<const int64_t *>(b + h.o_node_ptr);
  st->edge_ptr = reinterpret_cast<const int64_t *>(b + h.o_edge_ptr);
  st->types = reinterpret_cast<const uint8_t *>(b + h.o_types);
  st->edges = reinterpret_cast<const uint8_t *>(b + h.o_edges);
  st->y = reinterpret_cast<float *>(b + h.o_y);
  st->eattr = h.F > 0 ? reinterpret_cast<const float *>(b + h.o_eattr) : nullptr;
  st->ynode = h.o_ynode ? reinterpret_cast<float *>(b + h.o_ynode) : nullptr;
  int rc = got == st->bytes ? validate(st) : set_error(GCNN_EFORMAT, "store_open: short read");
  if (rc != GCNN_OK) {
    store_close(st);
    return rc;
  }
  *out = st;
  return GCNN_OK;
}

int store_close(gcnn_store *st) {
  if (!st) return GCNN_OK;
  if (st->dev) cudaFree(st->dev);
  if (st->host) {
    if (st->pinned) cudaFreeHost(st->host);
    else free(st->host);
  }
  delete st;
  return GCNN_OK;
}

int store_to_device(gcnn_store *st) {
  if (!st) return set_error(GCNN_EINVAL, "store_to_device: null store");
  int dev = 0;
  GCNN_CUDA_TRY(cudaGetDevice(&dev));
  if (st->dev && st->dev_id == dev) return GCNN_OK;
  if (st->dev) {
    cudaFree(st->dev);
    st->dev = nullptr;
  }
  GCNN_CUDA_TRY(cudaMalloc(&st->dev, st->bytes));
  GCNN_CUDA_TRY(cudaMemcpy(st->dev, st->host, st->bytes, cudaMemcpyHostToDevice));
  st->dev_id = dev;
  return GCNN_OK;
}

StoreView store_device_view(const gcnn_store *st) {
  const char *b = static_cast<const char *>(st->dev);
  return StoreView{reinterpret_cast<const int64_t *>(b + st->off_node_ptr),
                   reinterpret_cast<const int64_t *>(b + st->off_edge_ptr),
                   reinterpret_cast<const uint8_t *>(b + st->off_types),
                   reinterpret_cast<const uint8_t *>(b + st->off_edges),
                   reinterpret_cast<const float *>(b + st->off_y),
                   st->F > 0 ? reinterpret_cast<const float *>(b + st->off_eattr) : nullptr, st->F,
                   st->off_ynode ? reinterpret_cast<const float *>(b + st->off_ynode) : nullptr};
}

int store_batch_size(const gcnn_store *st, const int64_t *ids, int64_t n, int64_t *nn, int64_t *ne) {
  int64_t a = 0, e = 0;
  for (int64_t q = 0; q < n; ++q) {
    const int64_t g = ids[q];
    if (g < 0 || g >= st->G)
      return set_error(GCNN_EINVAL, "graph id %lld out of range [0, %lld)", (long long)g, (long long)st->G);
    a += st->node_ptr[g + 1] - st->node_ptr[g];
    e += st->edge_ptr[g + 1] - st->edge_ptr[g];
  }
  *nn = a;
  *ne = e;
  return GCNN_OK;
}

int store_delta(const gcnn_store *st, const int64_t *ids, int64_t n, double *delta) {
  if (!ids) n = st->G;
  double s = 0.0;
  int64_t nodes = 0;
  int cnt[256];
  for (int64_t q = 0; q < n; ++q) {
    const int64_t g = ids ? ids[q] : q;
    if (g < 0 || g >= st->G) return set_error(GCNN_EINVAL, "graph id out of range");
    const int64_t nv = st->node_ptr[g + 1] - st->node_ptr[g];
    const int64_t ne = st->edge_ptr[g + 1] - st->edge_ptr[g];
    for (int v = 0; v < nv; ++v) cnt[v] = 0;
    const uint8_t *ed = st->edges + 2 * st->edge_ptr[g];
    for (int64_t k = 0; k < ne; ++k) cnt[ed[2 * k + 1]] += 1;
    for (int v = 0; v < nv; ++v) s += std::log((double)cnt[v] + 1.0);
    nodes += nv;
  }
  *delta = nodes > 0 ? s / (double)nodes : 1.0;
  return GCNN_OK;
}

int store_set_targets(gcnn_store *st, const float *y, int64_t n) {
  if (!st || !y || n != st->G) return set_error(GCNN_EINVAL, "set_targets: need one target per graph");
  memcpy(st->y, y, sizeof(float) * (size_t)n);
  if (st->dev) {
    int cur = 0;
    GCNN_CUDA_TRY(cudaGetDevice(&cur));
    if (cur != st->dev_id) GCNN_CUDA_TRY(cudaSetDevice(st->dev_id));
    cudaError_t e = cudaMemcpy(static_cast<char *>(st->dev) + st->off_y, y, sizeof(float) * (size_t)n,
                               cudaMemcpyHostToDevice);
    if (cur != st->dev_id) cudaSetDevice(cur);
    GCNN_CUDA_TRY(e);
  }
  return GCNN_OK;
}

}  // namespace gcnn
