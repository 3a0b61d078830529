// Packed graph store (host side).
#pragma once

#include <vector>

#include "kernels.cuh"

struct gcnn_store {
  void *host = nullptr;  // whole file (pinned when possible)
  bool pinned = false;
  size_t bytes = 0;
  int64_t G = 0, N = 0, E = 0;
  uint32_t n_types = 0;
  int32_t F = 0;  // bond features per edge (version 2)
  int64_t off_node_ptr = 0, off_edge_ptr = 0, off_types = 0, off_edges = 0, off_y = 0, off_eattr = 0;
  int64_t off_ynode = 0;  // 0: no node-level targets
  const int64_t *node_ptr = nullptr;
  const int64_t *edge_ptr = nullptr;
  const uint8_t *types = nullptr;
  const uint8_t *edges = nullptr;
  float *y = nullptr;
  const float *eattr = nullptr;  // [E][F]
  float *ynode = nullptr;        // [N] node-level targets or nullptr
  void *dev = nullptr;  // device mirror of the whole file, or nullptr
  int dev_id = -1;
};

namespace gcnn {
// One graph read from a per-graph file (gcnn_store_pack's input format).
struct GraphFile {
  std::vector<uint8_t> buf;  // the whole file
  int n = 0, e = 0, F = 0;
  float y = 0.f;
  const uint8_t *types = nullptr, *edges = nullptr;
  const float *attr = nullptr;
};
int read_graph_file(const char *path, GraphFile *out);
int store_pack(const char *const *paths, int64_t n_files, const char *out_path, int n_threads);

const char *last_error();
int store_open(const char *path, gcnn_store **out);
int store_close(gcnn_store *st);
int store_to_device(gcnn_store *st);
StoreView store_device_view(const gcnn_store *st);
int store_batch_size(const gcnn_store *st, const int64_t *ids, int64_t n, int64_t *nn, int64_t *ne);
int store_delta(const gcnn_store *st, const int64_t *ids, int64_t n, double *delta);
int store_set_targets(gcnn_store *st, const float *y, int64_t n);
}  // namespace gcnn
