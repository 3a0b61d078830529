// Per-graph files and the packed store built from them (Sec. 4: the paper
// replaces one file per molecule by one global array per graph attribute,
// written in parallel, to cut the cost of loading the data; Table 1 lists the
// arrays).  Host code only.
//
// Per-graph file: "GCNNGRF1", int32 n, int32 e, int32 F, float32 y, then
// uint8 types[n], uint8 edges[e][2] (local source, destination), zero padding
// to a multiple of 4 bytes, float32 edge_attr[e][F].
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "store.h"

namespace gcnn {

int read_graph_file(const char *path, GraphFile *g) {
  FILE *f = fopen(path, "rb");
  if (!f) return set_error(GCNN_EINVAL, "cannot open graph file %s", path);
  fseek(f, 0, SEEK_END);
  const long size = ftell(f);
  fseek(f, 0, SEEK_SET);
  if (size < 24) {
    fclose(f);
    return set_error(GCNN_EFORMAT, "%s: not a graph file", path);
  }
  g->buf.resize((size_t)size);
  const size_t got = fread(g->buf.data(), 1, (size_t)size, f);
  fclose(f);
  const uint8_t *b = g->buf.data();
  int32_t hdr[3];
  memcpy(hdr, b + 8, sizeof(hdr));
  memcpy(&g->y, b + 20, sizeof(float));
  g->n = hdr[0];
  g->e = hdr[1];
  g->F = hdr[2];
  if (got != (size_t)size || memcmp(b, "GCNNGRF1", 8) != 0 || g->n < 1 || g->n > kMaxGraphNodes || g->e < 0 ||
      g->e > kMaxGraphEdges || g->F < 0 || g->F > 16)
    return set_error(GCNN_EFORMAT, "%s: bad graph file header", path);
  const size_t o_attr = (24 + (size_t)g->n + 2 * (size_t)g->e + 3) / 4 * 4;
  if ((size_t)size != o_attr + 4 * (size_t)g->e * g->F) return set_error(GCNN_EFORMAT, "%s: size mismatch", path);
  g->types = b + 24;
  g->edges = b + 24 + g->n;
  g->attr = reinterpret_cast<const float *>(b + o_attr);
  for (int k = 0; k < 2 * g->e; ++k)
    if (g->edges[k] >= g->n) return set_error(GCNN_EFORMAT, "%s: edge %d names node %d >= %d", path, k / 2,
                                              g->edges[k], g->n);
  return GCNN_OK;
}

namespace {

size_t align64(size_t v) { return (v + 63) / 64 * 64; }

// Run body(t, first, last) on n_threads threads over [0, n) in contiguous ranges.
template <class Body>
void parallel_ranges(int64_t n, int n_threads, Body body) {
  const int T = (int)std::max<int64_t>(1, std::min<int64_t>(n_threads, n));
  std::vector<std::thread> pool;
  for (int t = 0; t < T; ++t) {
    const int64_t a = n * t / T, b = n * (t + 1) / T;
    pool.emplace_back([=, &body] { body(t, a, b); });
  }
  for (auto &th : pool) th.join();
}

}  // namespace

int store_pack(const char *const *paths, int64_t n_files, const char *out_path, int n_threads) {
  std::vector<GraphFile> g((size_t)n_files);
  std::vector<int> rc((size_t)std::max(n_threads, 1), GCNN_OK);
  std::vector<std::string> msg((size_t)std::max(n_threads, 1));
  std::mutex mu;
  // 1. read and check every file (parallel)
  parallel_ranges(n_files, n_threads, [&](int t, int64_t a, int64_t b) {
    for (int64_t q = a; q < b && rc[t] == GCNN_OK; ++q) {
      const int r = read_graph_file(paths[q], &g[(size_t)q]);
      if (r != GCNN_OK) {
        std::lock_guard<std::mutex> lock(mu);
        rc[t] = r;
        msg[t] = last_error();
      }
    }
  });
  for (size_t t = 0; t < rc.size(); ++t)
    if (rc[t] != GCNN_OK) return set_error(rc[t], "%s", msg[t].c_str());
  const int F = n_files > 0 ? g[0].F : 0;
  int n_types = 7;
  for (int64_t q = 0; q < n_files; ++q) {
    if (g[(size_t)q].F != F) return set_error(GCNN_EFORMAT, "%s: %d bond features, the first file %d", paths[q],
                                              g[(size_t)q].F, F);
    for (int v = 0; v < g[(size_t)q].n; ++v) n_types = std::max(n_types, (int)g[(size_t)q].types[v] + 1);
  }
  if (n_types > 16) return set_error(GCNN_EFORMAT, "atom types above 15");
  // 2. offsets of every graph in the global arrays
  std::vector<int64_t> node_ptr((size_t)n_files + 1, 0), edge_ptr((size_t)n_files + 1, 0);
  for (int64_t q = 0; q < n_files; ++q) {
    node_ptr[(size_t)q + 1] = node_ptr[(size_t)q] + g[(size_t)q].n;
    edge_ptr[(size_t)q + 1] = edge_ptr[(size_t)q] + g[(size_t)q].e;
  }
  const int64_t G = n_files, N = node_ptr[(size_t)G], E = edge_ptr[(size_t)G];
  // 3. layout: 128-byte header, then each array on a 64-byte boundary
  int64_t off[6];
  size_t pos = 128;
  const size_t bytes[6] = {8 * (size_t)(G + 1), 8 * (size_t)(G + 1), (size_t)N, 2 * (size_t)E, 4 * (size_t)G,
                           4 * (size_t)E * F};
  const int n_arrays = F > 0 ? 6 : 5;
  for (int a = 0; a < n_arrays; ++a) {
    pos = align64(pos);
    off[a] = (int64_t)pos;
    pos += bytes[a];
  }
  const size_t total = align64(pos);
  std::vector<uint8_t> out(total, 0);
  memcpy(out.data(), "GCNNPKD1", 8);
  const uint32_t ver[2] = {F > 0 ? 2u : 1u, (uint32_t)n_types};
  memcpy(out.data() + 8, ver, sizeof(ver));
  const int64_t h1[9] = {G, N, E, off[0], off[1], off[2], off[3], off[4], (int64_t)total};
  memcpy(out.data() + 16, h1, sizeof(h1));
  if (F > 0) {
    const int64_t h2[2] = {F, off[5]};
    memcpy(out.data() + 88, h2, sizeof(h2));
  }
  memcpy(out.data() + off[0], node_ptr.data(), bytes[0]);
  memcpy(out.data() + off[1], edge_ptr.data(), bytes[1]);
  // 4. every graph's slices into the global arrays (parallel, disjoint ranges)
  parallel_ranges(n_files, n_threads, [&](int, int64_t a, int64_t b) {
    for (int64_t q = a; q < b; ++q) {
      const GraphFile &f = g[(size_t)q];
      memcpy(out.data() + off[2] + node_ptr[(size_t)q], f.types, (size_t)f.n);
      memcpy(out.data() + off[3] + 2 * edge_ptr[(size_t)q], f.edges, 2 * (size_t)f.e);
      memcpy(out.data() + off[4] + 4 * q, &f.y, 4);
      if (F > 0) memcpy(out.data() + off[5] + 4 * (size_t)edge_ptr[(size_t)q] * F, f.attr, 4 * (size_t)f.e * F);
    }
  });
  const std::string tmp = std::string(out_path) + ".tmp";
  FILE *fo = fopen(tmp.c_str(), "wb");
  if (!fo) return set_error(GCNN_EINVAL, "cannot write %s", tmp.c_str());
  const size_t put = fwrite(out.data(), 1, total, fo);
  const int cl = fclose(fo);
  if (put != total || cl != 0 || std::rename(tmp.c_str(), out_path) != 0)
    return set_error(GCNN_EINVAL, "writing %s failed", out_path);
  return GCNN_OK;
}

}  // namespace gcnn
