// Inference server: continuous batching of screening requests (Sec. 1 and
// Sec. 6: the trained GCNN as a fast surrogate over streams of molecules).
//
// submit() validates a request, reserves room for its atoms and edges in a
// device-resident request pool (two FIFO rings in device memory, sized at
// creation from queue_nodes and from the free device memory reported by
// cudaMemGetInfo once the slots' arenas are allocated), copies its atom types
// and bonds there and queues it.  Admission is refused (GCNN_EAGAIN) while
// the pool has no contiguous room for the request: admission is by device
// memory.  A request's room is released once all its molecules are done,
// in submission order.  One scheduler thread loops over the slots:
//   - a busy slot whose completion event fired is retired: its predictions
//     (pinned memory) are scattered to their requests, finished requests are
//     stamped and waiters woken;
//   - a free slot takes queued molecules in FIFO order (splitting requests
//     across batches) up to the largest bucket and the slot's molecule and
//     edge capacities, and only while they lie contiguously in the pool,
//     picks the smallest bucket that fits, writes the molecules' atom and
//     edge offsets into pinned memory, and enqueues on its own stream: one
//     host-to-device copy of the offsets, the device collator reading the
//     molecules straight from the pool, the forward graph
//     of that bucket (captured for every slot and bucket at creation), and one
//     device-to-host copy of the predictions, followed by its completion
//     event.
// Slots run with GCNN_FLAG_ROW_INVARIANT, so results do not depend on which
// molecules share a batch.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "context.h"

using namespace gcnn;
using Clock = std::chrono::steady_clock;

namespace {

struct Request {
  uint64_t ticket = 0;
  int n_mol = 0;
  std::vector<int32_t> n_nodes, n_edges;
  std::vector<int64_t> node_off, edge_off;  // prefix sums into types / edges
  int64_t pool_a = 0, pool_e = 0;            // first atom / edge of the request in the pool
  std::vector<float> out;
  int next = 0;          // first molecule not yet placed in a batch
  int remaining = 0;     // molecules not yet finished
  int status = GCNN_OK;  // sticky failure
  bool done = false;
  Clock::time_point t_submit, t_done;
};

struct Piece {
  Request *r;
  int first, count;
};

struct Slot {
  gcnn_ctx *ctx = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t start = nullptr, done = nullptr;  // around the batch's device work (timed)
  float *pin_out = nullptr;
  bool busy = false;
  std::vector<Piece> pieces;
  int graphs = 0;
  int64_t atoms = 0;
  std::vector<cudaGraphExec_t> exec;  // per bucket, captured at creation
};

// A FIFO ring over [0, cap) of one pool array: allocations are contiguous,
// taken at the head (skipping the end of the array when a request does not
// fit before it) and released from the tail in allocation order.
struct Ring {
  int64_t cap = 0, head = 0, tail = 0, used = 0;
  // start of `need` contiguous free units, and the units skipped at the end
  // of the array to reach it; false when there is no room
  bool fits(int64_t need, int64_t *start, int64_t *skip) const {
    if (need > cap) return false;
    if (used == 0) {
      *start = 0;
      *skip = 0;
      return true;
    }
    if (head > tail || (head == tail && used == 0)) {  // live [tail, head)
      if (cap - head >= need) { *start = head; *skip = 0; return true; }
      if (tail >= need) { *start = 0; *skip = cap - head; return true; }
      return false;
    }
    if (head < tail && tail - head >= need) { *start = head; *skip = 0; return true; }  // live wraps
    return false;
  }
  void take(int64_t start, int64_t skip, int64_t need) {
    if (used == 0) tail = start;
    used += skip + need;
    head = start + need;
  }
  void release(int64_t units, int64_t next_tail) {
    used -= units;
    tail = next_tail;
    if (used == 0) head = tail = 0;
  }
};

// One request's room in both rings: each region starts where the ring's head
// stood (so it includes the units skipped to reach the array's start).
struct Alloc {
  uint64_t ticket;  // the request's (requests are freed once polled)
  int64_t a_region, a_units, e_region, e_units;
  bool done;
};

}  // namespace

struct gcnn_server {
  gcnn_serve_config cfg{};
  std::vector<Slot> slots;
  int max_edges = 0;
  std::mutex mu;
  std::condition_variable work_cv, done_cv;
  std::deque<Request *> pending;
  std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
  // device request pool: atom types and local edge pairs of admitted requests
  uint8_t *pool_types = nullptr, *pool_edges = nullptr;
  float *zeros = nullptr;  // [max_graphs] targets of the collator (unused by serving)
  Ring ring_a, ring_e;     // atoms, edges
  std::deque<Alloc> allocs;
  cudaStream_t copy_stream = nullptr;
  std::mutex copy_mu;
  uint64_t next_ticket = 1;
  int64_t queued_nodes = 0;
  std::atomic<bool> stop{false};
  int fatal = GCNN_OK;
  char fatal_msg[256] = "";
  int64_t n_requests = 0, n_molecules = 0, n_batches = 0, n_refused = 0;
  // scheduler time forming and launching batches (host), device time from the
  // batch's input copy to its output copy, and atoms, summed over batches
  double host_us = 0.0, device_us = 0.0, atoms = 0.0;
  std::thread worker;
  int device = 0;
};

namespace {

size_t align16(size_t v) { return (v + 15) / 16 * 16; }

int capture_forward(gcnn_ctx *c, int G, int Ngrid, int Egrid, cudaGraphExec_t *out) {
  cudaGraph_t graph = nullptr;
  cudaStream_t user = c->stream;
  c->stream = c->cap_stream;
  c->capturing = true;
  cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
  int rc = e == cudaSuccess ? ctx_forward(c, G, Ngrid, Egrid, false)
                            : set_error(GCNN_ECUDA, "begin capture: %s", cudaGetErrorString(e));
  if (e == cudaSuccess) {
    cudaError_t e2 = cudaStreamEndCapture(c->stream, &graph);
    if (rc == GCNN_OK && e2 != cudaSuccess) rc = set_error(GCNN_ECUDA, "end capture: %s", cudaGetErrorString(e2));
  }
  c->stream = user;
  c->capturing = false;
  if (rc == GCNN_OK) {
    e = cudaGraphInstantiate(out, graph, 0);
    if (e != cudaSuccess) rc = set_error(GCNN_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
  }
  if (graph) cudaGraphDestroy(graph);
  return rc;
}

void fail_all(gcnn_server *s, int code) {
  // caller holds s->mu
  for (auto &kv : s->reqs) {
    Request *r = kv.second.get();
    if (!r->done) {
      r->status = code;
      r->done = true;
      r->t_done = Clock::now();
    }
  }
  s->pending.clear();
  s->done_cv.notify_all();
}

// Take molecules for one batch from the queue (caller holds s->mu).
void form_batch(gcnn_server *s, Slot &sl, int64_t *nodes, int64_t *edges) {
  const int64_t cap_nodes = s->cfg.bucket_nodes[s->cfg.n_buckets - 1];
  int64_t N = 0, E = 0;
  int G = 0;
  sl.pieces.clear();
  int64_t next_a = -1, next_e = -1;  // where the batch's next molecule must lie in the pool
  while (!s->pending.empty() && G < s->cfg.max_graphs) {
    Request *r = s->pending.front();
    const int64_t a0 = r->pool_a + r->node_off[r->next], e0 = r->pool_e + r->edge_off[r->next];
    if (next_a >= 0 && (a0 != next_a || e0 != next_e)) break;  // not contiguous (the pool wrapped)
    int take = 0;
    while (r->next + take < r->n_mol && G + take < s->cfg.max_graphs) {
      const int m = r->next + take;
      if (N + r->n_nodes[m] > cap_nodes || E + r->n_edges[m] > s->max_edges) break;
      N += r->n_nodes[m];
      E += r->n_edges[m];
      ++take;
    }
    if (take == 0) break;
    sl.pieces.push_back(Piece{r, r->next, take});
    for (int m = r->next; m < r->next + take; ++m) s->queued_nodes -= r->n_nodes[m];
    r->next += take;
    const int last = r->next - 1;
    next_a = r->pool_a + r->node_off[last] + r->n_nodes[last];
    next_e = r->pool_e + r->edge_off[last] + r->n_edges[last];
    G += take;
    if (r->next == r->n_mol) s->pending.pop_front();
    else break;  // batch full
  }
  sl.graphs = G;
  *nodes = N;
  *edges = E;
}

// Edge grid of bucket b: the slot's edge capacity in proportion to the
// bucket's node capacity (at least 512)
int bucket_edges(const gcnn_server *s, const gcnn_ctx *c, int b) {
  const int64_t top = s->cfg.bucket_nodes[s->cfg.n_buckets - 1];
  const int Eg = std::min(c->Ec, (int)((int64_t)s->cfg.bucket_nodes[b] * s->max_edges / top + 512));
  return std::max(Eg, 512);
}

int launch_batch(gcnn_server *s, Slot &sl, int64_t N, int64_t E) {
  gcnn_ctx *c = sl.ctx;
  const int G = sl.graphs;
  int b = 0;
  while (b < s->cfg.n_buckets - 1 && s->cfg.bucket_nodes[b] < N) ++b;
  // the batch's molecules lie contiguously in the pool: only their atom and
  // edge offsets (relative to the first molecule) go to the device, through
  // the slot context's pinned staging buffer (free: its previous batch has
  // completed)
  char *h = c->stage_host[0];
  size_t o = 0;
  const size_t o_np = o; o = align16(o + 8 * (size_t)(G + 1));
  const size_t o_ep = o; o = align16(o + 8 * (size_t)(G + 1));
  if (o > c->stage_bytes) return set_error(GCNN_EINVAL, "serve: staging too small");
  int64_t *np = reinterpret_cast<int64_t *>(h + o_np), *ep = reinterpret_cast<int64_t *>(h + o_ep);
  const Request *r0 = sl.pieces.front().r;
  const int64_t base_a = r0->pool_a + r0->node_off[sl.pieces.front().first];
  const int64_t base_e = r0->pool_e + r0->edge_off[sl.pieces.front().first];
  int g = 0;
  for (const Piece &p : sl.pieces) {
    const Request *r = p.r;
    for (int m = p.first; m < p.first + p.count; ++m, ++g) {
      np[g] = r->pool_a + r->node_off[m] - base_a;
      ep[g] = r->pool_e + r->edge_off[m] - base_e;
    }
  }
  np[G] = N;
  ep[G] = E;
  GCNN_CUDA_TRY(cudaEventRecord(sl.start, sl.stream));
  GCNN_CUDA_TRY(cudaMemcpyAsync(c->stage_dev, h, o, cudaMemcpyHostToDevice, sl.stream));
  const char *d = c->stage_dev;
  StoreView v{reinterpret_cast<const int64_t *>(d + o_np), reinterpret_cast<const int64_t *>(d + o_ep),
              s->pool_types + base_a, s->pool_edges + 2 * base_e, s->zeros};
  GCNN_TRY(launch_collate(G, nullptr, v, c->bb, c->scal_tab, c->Nc, c->Ec, c->err, sl.stream));
  GCNN_CUDA_TRY(cudaGraphLaunch(sl.exec[b], sl.stream));
  GCNN_CUDA_TRY(cudaMemcpyAsync(sl.pin_out, c->pred, sizeof(float) * G, cudaMemcpyDeviceToHost, sl.stream));
  GCNN_CUDA_TRY(cudaEventRecord(sl.done, sl.stream));
  sl.busy = true;
  sl.atoms = N;
  return GCNN_OK;
}

// Mark request r's pool room free and return every free room at the front
// of the allocation order to the rings (caller holds s->mu).
void release_pool(gcnn_server *s, Request *r) {
  for (Alloc &a : s->allocs)
    if (a.ticket == r->ticket) a.done = true;
  while (!s->allocs.empty() && s->allocs.front().done) {
    const Alloc a = s->allocs.front();
    s->allocs.pop_front();
    const Alloc *next = s->allocs.empty() ? nullptr : &s->allocs.front();
    s->ring_a.release(a.a_units, next ? next->a_region : 0);
    s->ring_e.release(a.e_units, next ? next->e_region : 0);
  }
}

void retire(gcnn_server *s, Slot &sl) {
  // caller holds s->mu
  int g = 0;
  const auto now = Clock::now();
  for (const Piece &p : sl.pieces) {
    Request *r = p.r;
    for (int m = p.first; m < p.first + p.count; ++m, ++g) r->out[m] = sl.pin_out[g];
    r->remaining -= p.count;
    s->n_molecules += p.count;
    if (r->remaining == 0 && !r->done) {
      r->done = true;
      r->t_done = now;
      s->n_requests += 1;
    }
    if (r->remaining == 0) release_pool(s, r);
  }
  sl.pieces.clear();
  sl.busy = false;
  s->n_batches += 1;
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, sl.start, sl.done) == cudaSuccess) s->device_us += 1e3 * ms;
  s->atoms += (double)sl.atoms;
  s->done_cv.notify_all();
}

void worker_loop(gcnn_server *s) {
  cudaSetDevice(s->device);
  for (;;) {
    bool progressed = false;
    for (Slot &sl : s->slots) {
      if (!sl.busy) continue;
      const cudaError_t q = cudaEventQuery(sl.done);
      if (q == cudaSuccess) {
        std::lock_guard<std::mutex> lock(s->mu);
        retire(s, sl);
        progressed = true;
      } else if (q != cudaErrorNotReady) {
        std::lock_guard<std::mutex> lock(s->mu);
        s->fatal = GCNN_ECUDA;
        snprintf(s->fatal_msg, sizeof(s->fatal_msg), "serve: batch failed: %s", cudaGetErrorString(q));
        fail_all(s, GCNN_ECUDA);
        sl.busy = false;
      }
    }
    for (Slot &sl : s->slots) {
      if (sl.busy) continue;
      int64_t N = 0, E = 0;
      {
        std::lock_guard<std::mutex> lock(s->mu);
        if (s->fatal != GCNN_OK || s->pending.empty()) break;
        form_batch(s, sl, &N, &E);
      }
      if (sl.graphs == 0) break;
      const auto t0 = Clock::now();
      const int rc = launch_batch(s, sl, N, E);
      const double us = std::chrono::duration<double, std::micro>(Clock::now() - t0).count();
      {
        std::lock_guard<std::mutex> lock(s->mu);
        s->host_us += us;
      }
      progressed = true;
      if (rc != GCNN_OK) {
        std::lock_guard<std::mutex> lock(s->mu);
        s->fatal = rc;
        snprintf(s->fatal_msg, sizeof(s->fatal_msg), "%s", gcnn_last_error());
        fail_all(s, rc);
      }
    }
    bool any_busy = false;
    for (Slot &sl : s->slots) any_busy |= sl.busy;
    if (s->stop.load() && !any_busy) break;
    if (!progressed) {
      if (any_busy) {
        std::this_thread::sleep_for(std::chrono::microseconds(20));
      } else {
        std::unique_lock<std::mutex> lock(s->mu);
        s->work_cv.wait_for(lock, std::chrono::milliseconds(2),
                            [s] { return s->stop.load() || (!s->pending.empty() && s->fatal == GCNN_OK); });
      }
    }
  }
}

int validate(const gcnn_server *s, const gcnn_request *q, int64_t *nodes) {
  if (!q || q->n_mol < 1 || !q->n_nodes || !q->n_edges || !q->types || !q->edges)
    return set_error(GCNN_EINVAL, "serve_submit: empty or null request");
  if (q->n_mol > (1 << 24)) return set_error(GCNN_EINVAL, "serve_submit: too many molecules");
  int64_t nn = 0, ne = 0;
  for (int m = 0; m < q->n_mol; ++m) {
    if (q->n_nodes[m] < 1 || q->n_nodes[m] > kMaxGraphNodes || q->n_edges[m] < 0 ||
        q->n_edges[m] > kMaxGraphEdges || q->n_edges[m] > s->max_edges)
      return set_error(GCNN_EINVAL, "serve_submit: molecule %d has %d atoms / %d edges (1..%d / 0..%d)", m,
                       q->n_nodes[m], q->n_edges[m], kMaxGraphNodes, kMaxGraphEdges);
    for (int v = 0; v < q->n_nodes[m]; ++v)
      if (q->types[nn + v] >= s->slots[0].ctx->T)
        return set_error(GCNN_EINVAL, "serve_submit: molecule %d has an atom type out of range", m);
    for (int k = 0; k < q->n_edges[m]; ++k) {
      const uint8_t *e = q->edges + 2 * (ne + k);
      if (e[0] >= q->n_nodes[m] || e[1] >= q->n_nodes[m])
        return set_error(GCNN_EINVAL, "serve_submit: molecule %d has an edge to a missing atom", m);
    }
    nn += q->n_nodes[m];
    ne += q->n_edges[m];
  }
  *nodes = nn;
  return GCNN_OK;
}

void destroy_server(gcnn_server *s) {
  if (s->pool_types) cudaFree(s->pool_types);
  if (s->pool_edges) cudaFree(s->pool_edges);
  if (s->zeros) cudaFree(s->zeros);
  if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
  for (Slot &sl : s->slots) {
    for (auto e : sl.exec)
      if (e) cudaGraphExecDestroy(e);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.start) cudaEventDestroy(sl.start);
    if (sl.pin_out) cudaFreeHost(sl.pin_out);
    if (sl.ctx) gcnn_destroy(sl.ctx);
    if (sl.stream) cudaStreamDestroy(sl.stream);
  }
  delete s;
}

}  // namespace

extern "C" {

int gcnn_serve_create(const gcnn_ctx *model, const gcnn_serve_config *cfg, gcnn_server **out) {
  if (!model || !cfg || !out) return set_error(GCNN_EINVAL, "serve_create: null argument");
  *out = nullptr;
  if (cfg->n_slots < 1 || cfg->n_slots > 16 || cfg->n_buckets < 1 || cfg->n_buckets > 8 || cfg->max_graphs < 1 ||
      cfg->queue_nodes < 1 || (cfg->precision != GCNN_PREC_FP32 && cfg->precision != GCNN_PREC_BF16))
    return set_error(GCNN_EINVAL, "serve_create: bad configuration");
  if (model->cfg.edge_features != 0)
    return set_error(GCNN_EINVAL, "serve_create: requests carry no bond features (model has %d)",
                     model->cfg.edge_features);
  for (int b = 0; b < cfg->n_buckets; ++b)
    if (cfg->bucket_nodes[b] < kMaxGraphNodes || (b > 0 && cfg->bucket_nodes[b] <= cfg->bucket_nodes[b - 1]))
      return set_error(GCNN_EINVAL, "serve_create: buckets must ascend and hold at least %d atoms", kMaxGraphNodes);
  gcnn_server *s = new gcnn_server();
  s->cfg = *cfg;
  cudaGetDevice(&s->device);
  const int max_nodes = cfg->bucket_nodes[cfg->n_buckets - 1];
  s->max_edges = (int)std::min<int64_t>((int64_t)max_nodes * 4 + kMaxGraphEdges, (int64_t)1 << 30);
  gcnn_config sc = model->cfg;
  sc.max_graphs = cfg->max_graphs;
  sc.max_nodes = max_nodes;
  sc.max_edges = s->max_edges;
  sc.precision = cfg->precision;
  sc.recompute = 1;  // inference: one aggregate buffer is enough
  sc.flags |= GCNN_FLAG_ROW_INVARIANT;
  sc.node_head = 0;  // screening serves the graph-level prediction; the node head's
                     // parameters follow all others, so the prefix is the graph model
  s->slots.resize(cfg->n_slots);
  int rc = GCNN_OK;
  for (Slot &sl : s->slots) {
    if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&sl.done) != cudaSuccess || cudaEventCreate(&sl.start) != cudaSuccess ||
        cudaMallocHost(&sl.pin_out, sizeof(float) * cfg->max_graphs) != cudaSuccess) {
      rc = set_error(GCNN_ENOMEM, "serve_create: stream / event / pinned allocation failed");
      break;
    }
    rc = gcnn_create(&sc, sl.stream, &sl.ctx);
    if (rc != GCNN_OK) break;
    rc = gcnn_set_params(sl.ctx, model->params, sl.ctx->P, 1);
    if (rc != GCNN_OK) break;
    // every bucket's forward graph is captured now, so that no request
    // waits for a capture
    sl.exec.assign(cfg->n_buckets, nullptr);
    for (int b = 0; b < cfg->n_buckets && rc == GCNN_OK; ++b)
      rc = capture_forward(sl.ctx, cfg->max_graphs, cfg->bucket_nodes[b], bucket_edges(s, sl.ctx, b), &sl.exec[b]);
    if (rc != GCNN_OK) break;
  }
  // the request pool: queue_nodes atoms and four edges per atom (plus one
  // largest molecule), within half of the device memory left once the slots'
  // arenas are allocated
  if (rc == GCNN_OK) {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) rc = set_error(GCNN_ECUDA, "serve_create: cudaMemGetInfo");
    int64_t atoms = cfg->queue_nodes;
    const int64_t budget = (int64_t)(free_b / 2);
    if (rc == GCNN_OK && atoms + 2 * (4 * atoms + kMaxGraphEdges) > budget) atoms = (budget - 2 * kMaxGraphEdges) / 9;
    if (rc == GCNN_OK && atoms < kMaxGraphNodes)
      rc = set_error(GCNN_ENOMEM, "serve_create: no device memory left for the request pool");
    if (rc == GCNN_OK) {
      s->ring_a.cap = atoms;
      s->ring_e.cap = 4 * atoms + kMaxGraphEdges;
      s->cfg.queue_nodes = atoms;
      if (cudaMalloc(&s->pool_types, (size_t)s->ring_a.cap) != cudaSuccess ||
          cudaMalloc(&s->pool_edges, 2 * (size_t)s->ring_e.cap) != cudaSuccess ||
          cudaMalloc(&s->zeros, sizeof(float) * cfg->max_graphs) != cudaSuccess ||
          cudaMemset(s->zeros, 0, sizeof(float) * cfg->max_graphs) != cudaSuccess ||
          cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking) != cudaSuccess)
        rc = set_error(GCNN_ENOMEM, "serve_create: request pool allocation failed");
    }
  }
  if (rc != GCNN_OK) {
    destroy_server(s);
    return rc;
  }
  s->worker = std::thread(worker_loop, s);
  *out = s;
  return GCNN_OK;
}

int gcnn_serve_submit(gcnn_server *s, const gcnn_request *q, uint64_t *ticket) {
  if (!s || !ticket) return set_error(GCNN_EINVAL, "serve_submit: null argument");
  int64_t nodes = 0;
  GCNN_TRY(validate(s, q, &nodes));
  if (nodes > s->cfg.queue_nodes)
    return set_error(GCNN_EINVAL, "serve_submit: request of %lld atoms exceeds the pool's %lld", (long long)nodes,
                     (long long)s->cfg.queue_nodes);
  auto r = std::make_unique<Request>();
  r->n_mol = q->n_mol;
  r->n_nodes.assign(q->n_nodes, q->n_nodes + q->n_mol);
  r->n_edges.assign(q->n_edges, q->n_edges + q->n_mol);
  r->node_off.resize(q->n_mol);
  r->edge_off.resize(q->n_mol);
  int64_t nn = 0, ne = 0;
  for (int m = 0; m < q->n_mol; ++m) {
    r->node_off[m] = nn;
    r->edge_off[m] = ne;
    nn += q->n_nodes[m];
    ne += q->n_edges[m];
  }
  if (ne > s->ring_e.cap)
    return set_error(GCNN_EINVAL, "serve_submit: request of %lld edges exceeds the pool's %lld", (long long)ne,
                     (long long)s->ring_e.cap);
  r->out.assign(q->n_mol, 0.f);
  r->remaining = q->n_mol;
  r->t_submit = Clock::now();
  Request *rp = r.get();
  {
    // room in the device pool (admission by device memory)
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->fatal != GCNN_OK) return set_error(s->fatal, "%s", s->fatal_msg);
    if (s->stop.load()) return set_error(GCNN_ESTATE, "serve_submit: server is stopping");
    int64_t a0 = 0, askip = 0, e0 = 0, eskip = 0;
    if (!s->ring_a.fits(nn, &a0, &askip) || !s->ring_e.fits(ne, &e0, &eskip)) {
      s->n_refused += 1;
      return set_error(GCNN_EAGAIN, "serve_submit: request pool full (%lld of %lld atoms held)",
                       (long long)s->ring_a.used, (long long)s->ring_a.cap);
    }
    r->ticket = s->next_ticket++;
    *ticket = r->ticket;
    s->allocs.push_back(Alloc{r->ticket, s->ring_a.head, askip + nn, s->ring_e.head, eskip + ne, false});
    s->ring_a.take(a0, askip, nn);
    s->ring_e.take(e0, eskip, ne);
    rp->pool_a = a0;
    rp->pool_e = e0;
    s->reqs.emplace(r->ticket, std::move(r));
  }
  // the atom types and bonds go to the reserved room before the scheduler can
  // see the request (the room belongs to no batch until then)
  cudaError_t ce;
  {
    std::lock_guard<std::mutex> lock(s->copy_mu);
    ce = cudaMemcpyAsync(s->pool_types + rp->pool_a, q->types, (size_t)nn, cudaMemcpyHostToDevice, s->copy_stream);
    if (ce == cudaSuccess && ne > 0)
      ce = cudaMemcpyAsync(s->pool_edges + 2 * rp->pool_e, q->edges, 2 * (size_t)ne, cudaMemcpyHostToDevice,
                           s->copy_stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s->copy_stream);
  }
  {
    std::lock_guard<std::mutex> lock(s->mu);
    if (ce != cudaSuccess) {
      s->fatal = GCNN_ECUDA;
      snprintf(s->fatal_msg, sizeof(s->fatal_msg), "serve: request copy failed: %s", cudaGetErrorString(ce));
      fail_all(s, GCNN_ECUDA);
      return set_error(GCNN_ECUDA, "%s", s->fatal_msg);
    }
    s->queued_nodes += nodes;
    s->pending.push_back(rp);
  }
  s->work_cv.notify_one();
  return GCNN_OK;
}

static int take_result(gcnn_server *s, std::unordered_map<uint64_t, std::unique_ptr<Request>>::iterator it, float *out,
                       double *latency_us) {
  Request *r = it->second.get();
  const int st = r->status;
  if (st == GCNN_OK && out) memcpy(out, r->out.data(), sizeof(float) * r->n_mol);
  if (latency_us) latency_us[0] = std::chrono::duration<double, std::micro>(r->t_done - r->t_submit).count();
  s->reqs.erase(it);
  return st == GCNN_OK ? GCNN_OK : set_error(st, "serve: request failed: %s", s->fatal_msg);
}

int gcnn_serve_poll(gcnn_server *s, uint64_t ticket, float *out, double *latency_us) {
  if (!s) return set_error(GCNN_EINVAL, "serve_poll: null server");
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return set_error(GCNN_EINVAL, "serve_poll: unknown ticket %llu", (unsigned long long)ticket);
  if (!it->second->done) return set_error(GCNN_EAGAIN, "serve_poll: not ready");
  return take_result(s, it, out, latency_us);
}

int gcnn_serve_wait(gcnn_server *s, uint64_t ticket, float *out, double *latency_us, int64_t timeout_us) {
  if (!s) return set_error(GCNN_EINVAL, "serve_wait: null server");
  std::unique_lock<std::mutex> lock(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return set_error(GCNN_EINVAL, "serve_wait: unknown ticket %llu", (unsigned long long)ticket);
  Request *r = it->second.get();
  if (!s->done_cv.wait_for(lock, std::chrono::microseconds(std::max<int64_t>(timeout_us, 0)), [r] { return r->done; }))
    return set_error(GCNN_ETIMEDOUT, "serve_wait: timed out");
  return take_result(s, s->reqs.find(ticket), out, latency_us);
}

int gcnn_serve_stats(gcnn_server *s, int64_t *requests, int64_t *molecules, int64_t *batches, int64_t *refused) {
  if (!s) return set_error(GCNN_EINVAL, "serve_stats: null server");
  std::lock_guard<std::mutex> lock(s->mu);
  if (requests) *requests = s->n_requests;
  if (molecules) *molecules = s->n_molecules;
  if (batches) *batches = s->n_batches;
  if (refused) *refused = s->n_refused;
  return GCNN_OK;
}

int gcnn_serve_timing(gcnn_server *s, double *host_us, double *device_us, double *atoms, int64_t *batches) {
  if (!s) return set_error(GCNN_EINVAL, "serve_timing: null server");
  std::lock_guard<std::mutex> lock(s->mu);
  if (host_us) *host_us = s->host_us;
  if (device_us) *device_us = s->device_us;
  if (atoms) *atoms = s->atoms;
  if (batches) *batches = s->n_batches;
  return GCNN_OK;
}

int gcnn_serve_destroy(gcnn_server *s) {
  if (!s) return GCNN_OK;
  s->stop.store(true);
  s->work_cv.notify_all();
  if (s->worker.joinable()) s->worker.join();
  {
    std::lock_guard<std::mutex> lock(s->mu);
    fail_all(s, GCNN_ESTATE);
  }
  destroy_server(s);
  return GCNN_OK;
}

}  // extern "C"
