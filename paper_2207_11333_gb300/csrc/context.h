// Training context: parameters, optimiser state, batch and activation arena.
#pragma once

#include <map>
#include <tuple>
#include <vector>

#include "store.h"

struct gcnn_ctx {
  gcnn_config cfg{};
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;  // private stream used only for graph capture
  cudaStream_t side = nullptr;        // BF16 backward: weight-gradient work off the critical path
  std::vector<cudaEvent_t> side_ev;   // 3 per layer: fork, aggregate gradient done, side work done;
                                      // then one for the head gradients
  cudaStream_t opt = nullptr;         // train step: early AdamW updates of layers L-1 .. 1
  cudaEvent_t opt_ev = nullptr;       // their completion
  int device = 0;
  int H = 0, L = 0, T = 0, Hh = 0;
  int64_t P = 0;       // parameter count
  int64_t layer_size = 0;
  int Gc = 0, Nc = 0, Ec = 0;  // capacities

  char *dmem = nullptr;  // one device allocation for everything below
  size_t dbytes = 0;

  float *params = nullptr, *grads = nullptr, *adam_m = nullptr, *adam_v = nullptr;
  int *opt_state = nullptr;  // [0] step, [1..2] bias-correction factors (float bits)
  float *lr_dev = nullptr;
  float *loss_scale = nullptr;  // [0] graph-level, [1] node-level loss-gradient scale (1, 1)
  std::vector<cudaEvent_t> grad_ev;  // L + 1: layer l's gradients final; [L]: every gradient
  float *scal_tab = nullptr;  // 2 * (kMaxGraphEdges + 1)
  unsigned *err = nullptr;

  gcnn::BatchBuf bb{};
  int64_t *ids_dev = nullptr;
  char *stage_dev = nullptr;
  size_t stage_bytes = 0;
  char *stage_host[2] = {nullptr, nullptr};
  cudaEvent_t stage_ev[2] = {nullptr, nullptr};
  bool stage_used[2] = {false, false};
  int stage_i = 0;

  int64_t *order_dev = nullptr;  // gcnn_set_order
  std::vector<int64_t> order_host;
  const gcnn_store *order_store = nullptr;

  // activations
  float *xs = nullptr;   // (L+1) x Nc x H
  float *PQ = nullptr;   // L x Nc x 2H
  float *agg = nullptr;  // (recompute ? 1 : L) x Nc x 5H
  float *pooled = nullptr, *z1 = nullptr, *pred = nullptr, *dpred = nullptr, *dz1 = nullptr;
  float *dg = nullptr;
  float *dH = nullptr, *dX = nullptr, *dagg = nullptr, *dPQ = nullptr, *dm = nullptr;
  int *chunks = nullptr;  // work partition of the fused aggregation backward
  // node-level head: pre-activations, their gradient, outputs, output
  // gradients and the gradient it sends to the last layer's atoms
  float *zn = nullptr, *dzn = nullptr, *predn = nullptr, *dpredn = nullptr, *dxn = nullptr;
  float *dPQ2 = nullptr;  // BF16: second [dP | dQ] buffer, alternating by layer
  unsigned *tickets = nullptr;  // zero-initialised completion counters of single-launch reductions

  // BF16 operands of the tensor-core GEMMs (precision == GCNN_PREC_BF16)
  uint16_t *wb = nullptr;     // parameters cast to BF16 after every update (same layout)
  uint16_t *wpack = nullptr;  // per layer: Wd [5H][3H] then Wx [H][3H] (backward B operands)
  uint16_t *U = nullptr;      // (recompute ? 1 : L) x Nc x 16H: [x_l | agg | amp*agg | att*agg]
  uint16_t *Xb = nullptr;     // recompute only: L x Nc x H layer inputs (copied into U when needed)
  uint16_t *G5[2] = {nullptr, nullptr};  // Nc x 5H: [amp*g | att*g | g | dP | dQ]
  gcnn::GemmWorkspace ws{};
  gcnn::GemmWorkspace ws_side{};  // split-K partials of the GEMMs on the side stream

  // host-side state
  bool have_fwd = false;
  int fwd_G = 0, fwd_N = 0, fwd_E = 0;
  float lr_host = -1.f;
  float *lr_pinned = nullptr;
  float scale_host[2] = {1.f, 1.f};
  float *scale_pinned = nullptr;  // 2 floats
  struct ProfEvent {
    int phase;
    cudaEvent_t a, b;
  };
  struct Graph {
    cudaGraphExec_t exec;
    int kernels;
    std::vector<ProfEvent> ev;  // profiling graphs: event-record nodes around each phase
    // graphs that begin with the collation of a range of the device-resident
    // order: the captured graph (its nodes address the instantiated one), the
    // collation's kernel nodes, and the store and id list they were last set to
    cudaGraph_t graph = nullptr;
    cudaGraphNode_t scan_node = nullptr, graph_node = nullptr;
    const gcnn_store *range_store = nullptr;
    const int64_t *range_ids = nullptr;
  };
  // key: grid (graphs, node bucket, edge bucket), loss accumulator, profiling
  // graph, whether the graph ends with the optimizer step, and whether it
  // begins with the collation of a range of the device-resident order
  std::map<std::tuple<int, int, int, const double *, bool, bool, bool>, Graph> graphs;
  bool cap_grad_events = false;  // capturing forward + backward: record the bucket events externally
  int last_step_kernels = 0;
  bool capturing = false;
  bool fuse_head = false;  // train step: head backward runs inside the forward's head kernel
  bool fuse_step = false;  // train step: the optimiser follows the backward in the same graph

  // per-phase event timing (gcnn_profile_enable)
  bool prof_on = false;
  std::vector<cudaEvent_t> prof_ev;  // eager launches: pairs [2k] start, [2k+1] end
  std::vector<int> prof_cls;
  size_t prof_used = 0;
  std::vector<ProfEvent> cap_ev;     // events recorded into the graph being captured
  double prof_ms[GCNN_NPHASE] = {};  // accumulated from profiling-graph replays
  int64_t prof_n[GCNN_NPHASE] = {};
};

namespace gcnn {
// Refresh the BF16 copies of the parameters (BF16 precision; no-op otherwise).
int ctx_refresh_bf16(gcnn_ctx *c);

// Event pair around the kernels launched in its lifetime (no-op unless
// profiling is on and the stream is not being captured).
class PhaseScope {
 public:
  PhaseScope(gcnn_ctx *c, int phase);
  ~PhaseScope();

 private:
  gcnn_ctx *c_;
  long idx_;
};

int ctx_collate(gcnn_ctx *c, const gcnn_store *st, const int64_t *ids, int32_t n, gcnn_batch *out);
int ctx_collate_files(gcnn_ctx *c, const char *const *paths, int32_t n, gcnn_batch *out);
int ctx_collate_range(gcnn_ctx *c, const gcnn_store *st, int64_t first, int32_t count, gcnn_batch *out);
// gcnn_collate_range in parts: checks and host-side sizes of the range (out
// receives the batch views), the collation launches on c->stream, and the
// update of a captured collation's two kernel nodes to another range of the
// same graph count
int ctx_range_prepare(gcnn_ctx *c, const gcnn_store *st, int64_t first, int32_t count, gcnn_batch *out);
int ctx_range_launch(gcnn_ctx *c, const gcnn_store *st, int64_t first, int32_t count);
int ctx_range_update(gcnn_ctx *c, const gcnn_store *st, int64_t first, int32_t count, cudaGraphExec_t exec,
                     cudaGraphNode_t scan_node, cudaGraphNode_t graph_node);
int ctx_forward(gcnn_ctx *c, int G, int Ngrid, int Egrid, bool train);
int ctx_backward(gcnn_ctx *c, int G, int Ngrid, int Egrid, const float *dpred, double *loss_accum);
int ctx_step(gcnn_ctx *c);
}  // namespace gcnn
