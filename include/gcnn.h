/*
 * gcnn.h -- C ABI of the GB300 (sm_103a) GCNN training / inference library.
 *
 * The library implements one training step of the graph convolutional neural
 * network of HydraGNN (Choi et al., arXiv 2207.11333) over a collated batch
 * of molecular graphs: data loading from a packed store (Sec. 4, Table 1),
 * batch collation, PNA graph convolutions (Sec. 3.1; 6 layers in Sec. 5.1),
 * global mean pooling (Sec. 3.1), a fully connected head (Sec. 3.1), the MSE
 * loss, the backward pass and the optimizer step (Sec. 3.2, Fig. 3; AdamW with
 * learning rate 1e-3 in Sec. 5.1), plus an inference server for the paper's
 * screening use (Sec. 1, Sec. 6).
 *
 * Conventions
 *   - Every function returns an int status: GCNN_OK (0) or a negative GCNN_E*
 *     code; gcnn_last_error() gives a message for the calling thread.  No
 *     function aborts, traps or throws across this boundary.
 *   - "stream" arguments are cudaStream_t values passed as void*; NULL is the
 *     legacy default stream.  GPU work is asynchronous on the stream unless a
 *     function says otherwise.
 *   - Pointers marked (device) are CUDA device pointers; (host) pointers are
 *     ordinary host memory.  The caller owns every buffer it passes; the
 *     library owns the objects it creates until the matching destroy call.
 *   - Matrices are row-major.  H = hidden width, Hh = head hidden width,
 *     T = number of atom types, L = number of convolution layers,
 *     G / N / E = graphs / nodes / directed edges of a batch.
 *
 * Model (PNA layer, the published definition with one linear message layer
 * and one linear update layer; the paper names PNA without printing it):
 *   x0_i          = emb[type_i]
 *   m_ij          = W_M [x_i ; x_j ; e_ij] + b_M        for each edge j -> i
 *                   (e_ij: the bond's F features, Sec. 3.1 and Table 1's
 *                   edge attributes; F = 0: no bond term)
 *   a_i           = sum, mean, min, max, std of m_ij over j in N(i)   (5H)
 *   s_i           = [1, log(d_i+1)/delta, delta/log(d_i+1)]          (scalers)
 *   x_i'          = ReLU(W_U [x_i ; s_i (x) a_i] + b_U)               (16H -> H)
 *   g             = mean of x^L over the graph's nodes
 *   yhat          = w2 . ReLU(W1 g + b1) + b2
 *   loss          = (1/G) sum_g (yhat_g - y_g)^2
 *   optional node-level head (config node_head), on every atom of x^L:
 *   yhat_i        = w2n . ReLU(W1n x_i + b1n) + b2n
 *   loss         += node_loss_weight (1/N) sum_i (yhat_i - y_i)^2
 * with std = sqrt(ReLU(var) + std_eps), var two-pass; d_i = 0 gives zero
 * aggregates; the scalers use max(d_i, 1); min/max ties share the gradient
 * equally; ReLU'(0) = 0.
 *
 * Flat parameter layout (float32), in this order:
 *   emb[T][H]
 *   per layer: msg_w[H][2H] (columns 0..H-1 act on x_i, H..2H-1 on x_j),
 *              msg_b[H],
 *              upd_w[16H][H] (rows 0..H-1 act on x_i, then 15 blocks of H
 *                 rows, scaler-major: identity{sum,mean,min,max,std},
 *                 amplification{...}, attenuation{...}),
 *              upd_b[H]
 *   head: w1[H][Hh], b1[Hh], w2[Hh], b2[1]
 *   with F bond features: 0..3 unused floats up to the next multiple of 4,
 *   then per layer edge_w[F][H] (the bond rows of W_M)
 *   with the node head: 0..3 unused floats up to the next multiple of 4,
 *   then w1n[H][Hh], b1n[Hh], w2n[Hh], b2n[1]
 */
#ifndef GCNN_H_
#define GCNN_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GCNN_OK 0
#define GCNN_EINVAL (-1)    /* bad argument or unsupported size               */
#define GCNN_ENOMEM (-2)    /* host or device allocation failed               */
#define GCNN_ECUDA (-3)     /* a CUDA runtime call failed                     */
#define GCNN_EFORMAT (-4)   /* the store file is malformed                    */
#define GCNN_EDEVICE (-5)   /* a device-side bounds check fired               */
#define GCNN_ETIMEDOUT (-6) /* a bounded wait ran out                         */
#define GCNN_EAGAIN (-7)    /* result not ready / queue full: call again      */
#define GCNN_ESTATE (-8)    /* call out of order (e.g. backward w/o forward)  */

#define GCNN_PREC_FP32 0    /* FP32 everywhere (SIMT FFMA GEMMs)              */
#define GCNN_PREC_BF16 1    /* BF16 tensor-core GEMMs, FP32 accumulate        */

/* Row-invariant arithmetic: no split-K in the GEMMs, so each node's and each
 * graph's results depend only on its own graph, never on its batch-mates
 * (bit-identical alone and in any batch).  Used by the inference server. */
#define GCNN_FLAG_ROW_INVARIANT 1
/* One stream for the whole step.  By default the BF16 backward (without
 * recompute) runs each layer's weight- and bias-gradient GEMMs and sums on a
 * second stream, overlapped with the data-gradient chain of the layers below
 * (same kernels, same results bit for bit); this flag keeps every kernel on
 * the caller's stream, in order, e.g. to time kernels one by one. */
#define GCNN_FLAG_SERIAL 2

/* Message for the last failing call on this thread (never NULL). */
const char *gcnn_last_error(void);
/* Library version, major * 10000 + minor * 100 + patch. */
int gcnn_version(void);

/* ------------------------------------------------------------------ store
 * Packed graph store: one file holding every graph attribute as a global
 * array (the single-file analogue of the paper's schema, Sec. 4, Table 1):
 * node_ptr[G+1], edge_ptr[G+1] (int64 offsets), types[N] (uint8 atom type),
 * edges[E][2] (uint8 local source, destination), y[G] (float32 target);
 * version-2 files may add edge_attr[E][F] (float32 bond features, F <= 16;
 * both directions of a bond must carry bitwise-equal features) and node_y[N]
 * (float32 node-level targets).
 * Graphs must have 1..255 nodes and at most 1024 directed edges, local ids
 * < n; each undirected bond is stored as two directed edges.  The file is
 * validated once at open (GCNN_EFORMAT on any violation).  A store is
 * read-only after open except for gcnn_store_set_targets, and may be shared
 * by several contexts on one device.
 */
typedef struct gcnn_store gcnn_store;

/* Open and validate a store file; *out owns a host copy in pinned memory. */
int gcnn_store_open(const char *path, gcnn_store **out);
int gcnn_store_close(gcnn_store *st);
/* Totals of the whole store. */
int gcnn_store_info(const gcnn_store *st, int64_t *n_graphs, int64_t *n_nodes, int64_t *n_edges);
/* Bond features per edge, 0 for a version-1 store (Table 1's edge
 * attributes).  Never fails on a valid store. */
int gcnn_store_edge_features(const gcnn_store *st, int32_t *n_features);
/* Whether the store carries node-level targets, 1, or not, 0 (Table 1's
 * node-level y).  Never fails on a valid store. */
int gcnn_store_has_node_targets(const gcnn_store *st, int32_t *has);
/* Node and edge totals of the batch graph_ids[0..n) (host ids). */
int gcnn_store_batch_size(const gcnn_store *st, const int64_t *graph_ids, int64_t n,
                          int64_t *n_nodes, int64_t *n_edges);
/* PNA degree normaliser delta = mean over all nodes of graphs ids[0..n)
 * (ids NULL: every graph) of log(in-degree + 1), in FP64. */
int gcnn_store_delta(const gcnn_store *st, const int64_t *graph_ids, int64_t n, double *delta);
/* Replace the targets y[0..n) (host, n = number of graphs); updates the
 * device copy too when one exists (synchronously). */
int gcnn_store_set_targets(gcnn_store *st, const float *y, int64_t n);
/* Copy the store's arrays into device memory of the current device so that
 * collation reads them there (the "resident" mode).  Synchronous. */
int gcnn_store_to_device(gcnn_store *st);

/* Per-graph files: one molecule per file, the layout the packed store
 * replaces (Sec. 4: global arrays instead of one file per sample, to cut the
 * data-loading time of Fig. 5).  Format: "GCNNGRF1", int32 n (atoms, 1..255),
 * int32 e (directed edges, <= 1024), int32 F (bond features, 0..16),
 * float32 y, uint8 types[n], uint8 edges[e][2] (local source, destination),
 * zero padding to a multiple of 4 bytes, float32 edge_attr[e][F];
 * little-endian.
 * gcnn_store_pack reads paths[0..n_files) (host strings) with n_threads
 * threads, checks each file (GCNN_EFORMAT names the first bad one; every file
 * must have the same F), and writes one packed store to out_path (version 1,
 * or 2 when F > 0; atom-type count max(7, largest type + 1)): graph q of the
 * store is file q.  The bytes do not depend on n_threads.  Bond symmetry is
 * checked when the store is opened. */
int gcnn_store_pack(const char *const *paths, int64_t n_files, const char *out_path, int32_t n_threads);

/* ------------------------------------------------------------------ context */
typedef struct gcnn_config {
  int32_t hidden;       /* H, a multiple of 8, 8..1024                         */
  int32_t layers;       /* L >= 1 convolution layers                           */
  int32_t n_types;      /* T atom types (7)                                    */
  int32_t head_hidden;  /* Hh, 1..1024                                         */
  int32_t max_graphs;   /* batch capacity: graphs                              */
  int32_t max_nodes;    /* batch capacity: nodes                               */
  int32_t max_edges;    /* batch capacity: directed edges                      */
  int32_t precision;    /* GCNN_PREC_FP32 or GCNN_PREC_BF16                    */
  int32_t recompute;    /* 1: do not keep aggregates in forward; recompute
                           them per layer in backward (saves 5*N*H floats per
                           layer)                                              */
  int32_t flags;        /* GCNN_FLAG_* bits                                    */
  double delta;         /* PNA degree normaliser (gcnn_store_delta)            */
  double std_eps;       /* epsilon inside the std aggregator (1e-5)            */
  double beta1, beta2;  /* Adam moment decays (0.9, 0.999)                     */
  double adam_eps;      /* Adam epsilon (1e-8)                                 */
  double weight_decay;  /* decoupled (AdamW) weight decay (0)                  */
  int32_t edge_features;  /* F bond features per edge, 0..16 (0); a store fed
                             to the context must carry exactly F           */
  int32_t reserved0;
  int32_t node_head;      /* 1: add the node-level head (Sec. 3.1 node-level
                             properties; Table 1 node-level y); the store
                             must carry node targets; head_hidden % 4 == 0 */
  int32_t reserved1;
  double node_loss_weight;  /* weight of the node-level MSE in the loss (1) */
} gcnn_config;

typedef struct gcnn_ctx gcnn_ctx;

/* Fill *cfg with the defaults above for the given sizes. */
int gcnn_config_default(gcnn_config *cfg, int32_t hidden, int32_t layers, int32_t max_graphs,
                        int32_t max_nodes, int32_t max_edges);
/* Create a context on the current device: allocates parameters (zeroed),
 * gradients, Adam moments and an activation arena sized by the capacities.
 * All later GPU work of this context runs on `stream`. */
int gcnn_create(const gcnn_config *cfg, void *stream, gcnn_ctx **out);
int gcnn_destroy(gcnn_ctx *ctx);
/* Number of float32 parameters (layout in the file header). */
int gcnn_param_count(const gcnn_ctx *ctx, int64_t *n);
/* Copy n = gcnn_param_count floats in or out; on_device says whether the
 * caller's pointer is device (1) or host (0) memory.  Synchronous. */
int gcnn_set_params(gcnn_ctx *ctx, const float *src, int64_t n, int on_device);
int gcnn_get_params(gcnn_ctx *ctx, float *dst, int64_t n, int on_device);
int gcnn_get_grads(gcnn_ctx *ctx, float *dst, int64_t n, int on_device);
/* Zero Adam's moments and step counter. */
int gcnn_reset_optimizer(gcnn_ctx *ctx);
/* Checkpoint: parameters, Adam moments and step counter in one binary file. */
int gcnn_save(gcnn_ctx *ctx, const char *path);
int gcnn_load(gcnn_ctx *ctx, const char *path);
/* Device error word (bounds checks in kernels); synchronises the stream.
 * Returns GCNN_EDEVICE and clears the word if a check fired. */
int gcnn_check(gcnn_ctx *ctx);

/* ------------------------------------------------------------------ batches
 * A collated batch: device views into the context's arena, valid until the
 * next collate on the same context.  Edges are grouped by destination in
 * CSR form (row_ptr/col, col = source node), each row sorted by source.
 */
typedef struct gcnn_batch {
  int32_t n_graphs, n_nodes, n_edges, reserved;
  const int32_t *node_off;  /* (device) [G+1] first node of each graph         */
  const int32_t *edge_off;  /* (device) [G+1] first edge slot of each graph    */
  const int32_t *graph_id;  /* (device) [N]   graph of each node               */
  const int32_t *row_ptr;   /* (device) [N+1] CSR offsets by destination       */
  const int32_t *col;       /* (device) [E]   source node of each edge slot    */
  const int32_t *rev;       /* (device) [E]   slot of the reverse edge         */
  const int32_t *deg;       /* (device) [N]   in-degree                        */
  const float *amp;         /* (device) [N]   log(max(d,1)+1)/delta as float   */
  const float *att;         /* (device) [N]   delta/log(max(d,1)+1) as float   */
  const uint8_t *types;     /* (device) [N]   atom type                        */
  const float *y;           /* (device) [G]   target                           */
  const float *edge_attr;   /* (device) [E] rows of bond features per edge
                               slot, row stride F rounded up to a multiple
                               of 4 floats (NULL when F = 0)                  */
  const float *node_y;      /* (device) [N] node-level targets (NULL without
                               the node head)                                 */
} gcnn_batch;

/* Collate graphs graph_ids[0..n_graphs) (host ids) of `st` on the device: the
 * disjoint union of the molecules as one graph (Sec. 3.2: a mini-batch of
 * graphs; Sec. 4, Table 1: per-graph slices of the global arrays).
 * Resident store: the collator reads the device copy; otherwise the graphs'
 * slices are gathered into pinned staging memory and copied in one transfer.
 * GCNN_EINVAL if the batch exceeds the context's capacities. */
int gcnn_collate(gcnn_ctx *ctx, const gcnn_store *st, const int64_t *graph_ids, int32_t n_graphs,
                 gcnn_batch *out);
/* Collate graphs straight from per-graph files (host paths, read one after
 * another into pinned staging memory, then one copy): the per-file loading
 * path that the packed store replaces, kept for comparison.  Same batch as
 * gcnn_collate on a store packed from the same files. */
int gcnn_collate_files(gcnn_ctx *ctx, const char *const *paths, int32_t n_graphs, gcnn_batch *out);
/* Upload an order of graph ids (host, n) once; gcnn_collate_range then
 * collates order[first .. first+count) reading the ids on the device
 * (resident stores only). */
int gcnn_set_order(gcnn_ctx *ctx, const gcnn_store *st, const int64_t *order, int64_t n);
int gcnn_collate_range(gcnn_ctx *ctx, const gcnn_store *st, int64_t first, int32_t count,
                       gcnn_batch *out);
/* Copy a batch's arrays to host buffers (any may be NULL).  Synchronous. */
int gcnn_batch_export(gcnn_ctx *ctx, const gcnn_batch *b, int32_t *node_off, int32_t *graph_id,
                      int32_t *row_ptr, int32_t *col, int32_t *rev, int32_t *deg, float *amp,
                      float *att, uint8_t *types, float *y);

/* ------------------------------------------------------------------ training */
/* Forward pass (Sec. 3.1: embedding, L PNA message-passing layers, global
 * mean pooling, FC head; Fig. 3's forward phase); pred (device, G floats) may
 * be NULL.  train = 1 keeps what backward needs (with the node head it also
 * forms the node-level loss gradient from the batch's node targets). */
int gcnn_forward(gcnn_ctx *ctx, const gcnn_batch *b, float *pred, int train);
/* Backward of the last forward(train = 1) on the same batch (Sec. 3.2, Fig. 3:
 * the MSE loss and its gradients w.r.t. every parameter).  dpred (device,
 * G) = dL/dyhat, or NULL for the MSE loss against the batch targets.
 * Gradients overwrite the context's gradient buffer.  loss_accum (device,
 * 3 doubles, 5 with the node head, may be NULL): += sum (yhat-y)^2,
 * += sum |yhat-y|, += G, then += sum over atoms (yhat_i-y_i)^2, += N.  The
 * node-level loss always uses the batch's node targets (dpred is graph-level). */
int gcnn_backward(gcnn_ctx *ctx, const gcnn_batch *b, const float *dpred, double *loss_accum);
/* AdamW step over all parameters with learning rate lr (Sec. 3.2, Fig. 3: the
 * optimizer update of one training iteration; Sec. 5.1: AdamW). */
int gcnn_step(gcnn_ctx *ctx, float lr);

/* ------------------------------------------------------- data parallelism
 * Sec. 4 (Fig. 4): distributed data parallelism replicates the model on every
 * GPU, gives each process its own graphs and averages the gradients with an
 * all-reduce before every optimizer step.  The library does not talk to other
 * processes; these calls let the caller run that exchange with its own
 * communicator (NCCL through torch.distributed in the Python package), bucket
 * by bucket while the backward is still running.
 *
 * gcnn_set_loss_scale: multiply dL/dyhat of the graph-level MSE by graph_scale
 * and the node-level loss gradient by node_scale in every later backward and
 * train step (both 1 after gcnn_create).  With graph_scale = G_r / G (this
 * process's graphs over all processes' graphs of the step) and node_scale =
 * N_r / N (atoms likewise), the sum over processes of the gradients is the
 * gradient of the whole step's mean loss.  Not applied to a caller-given dpred.
 * Synchronises the context's stream when a value changes.  GCNN_EINVAL for a
 * negative or non-finite scale. */
int gcnn_set_loss_scale(gcnn_ctx *ctx, float graph_scale, float node_scale);
/* Number of gradient buckets: L + 2.  Bucket l < L is conv layer l's
 * parameters; bucket L the head, bond rows and node head; bucket L + 1 the
 * embedding table.  Buckets are disjoint and together cover the flat buffer. */
int gcnn_grad_buckets(const gcnn_ctx *ctx, int32_t *n_buckets);
/* Float offset and count of bucket k in the flat gradient buffer. */
int gcnn_grad_bucket(const gcnn_ctx *ctx, int32_t k, int64_t *offset, int64_t *count);
/* Make `stream` (a caller's cudaStream_t) wait until bucket k's gradients of
 * the last backward are final.  Layer buckets complete during the backward,
 * from the last layer to the first; buckets L and L + 1 when it ends.  Valid
 * after gcnn_backward, not after gcnn_train_step (whose graph
 * applies AdamW itself); after gcnn_forward_backward too.  Enqueues a wait
 * only; never blocks the host. */
int gcnn_grad_wait(gcnn_ctx *ctx, int32_t k, void *stream);
/* Device address of the flat FP32 gradient buffer (gcnn_param_count floats,
 * owned by the context, valid until gcnn_destroy).  A caller that reduces the
 * gradients in place does so between gcnn_backward and gcnn_step, on streams
 * ordered after gcnn_grad_wait and before the context's stream resumes. */
int gcnn_grads_device(gcnn_ctx *ctx, float **grads);
/* forward(train) + backward(MSE) + step (Sec. 3.2, Fig. 3: one training
 * iteration); replays a captured CUDA graph per batch graph count after the
 * first call with that count.  With BF16 GEMMs and the overlapped backward, the
 * graph runs the weight gradients on a second stream and each layer's AdamW
 * update on a third as soon as that layer's gradients are complete; the result
 * equals forward + backward + step bit for bit. */
int gcnn_train_step(gcnn_ctx *ctx, const gcnn_batch *b, float lr, double *loss_accum);
/* gcnn_collate_range(first, count) + gcnn_train_step in one captured CUDA
 * graph (Sec. 3.2, Fig. 3: loading, forward, backward and optimizer of one
 * training iteration): the collation of order[first .. first+count) (the
 * order set by gcnn_set_order, resident store) is the graph's first launch,
 * so the device goes from batch assembly into the forward without a host
 * round trip between two submissions.  The graph is captured per graph count
 * and size bucket on first use; a later call with another `first` updates the
 * collation's arguments in the instantiated graph (launches already queued
 * keep theirs).  Results equal gcnn_collate_range + gcnn_train_step bit for
 * bit.  out (nullable) receives the batch's device views, valid as after
 * gcnn_collate_range.  GCNN_ESTATE without gcnn_set_order on `st`,
 * GCNN_EINVAL for a range outside the order or beyond the capacities. */
int gcnn_train_step_range(gcnn_ctx *ctx, const gcnn_store *st, int64_t first, int32_t count, float lr,
                          double *loss_accum, gcnn_batch *out);
/* forward(train) + backward(MSE) without the optimizer step, replayed from a
 * captured CUDA graph per batch graph count like gcnn_train_step: the first
 * half of a data-parallel step.  The graph records the gradient buckets'
 * completion events (gcnn_grad_wait works on them after this call returns);
 * the caller exchanges the gradients and then calls gcnn_step.  Results equal
 * gcnn_forward + gcnn_backward. */
int gcnn_forward_backward(gcnn_ctx *ctx, const gcnn_batch *b, double *loss_accum);
/* Copy x^l (l = 0..L, N x H floats) of the last forward to host.  Sync. */
int gcnn_get_activation(gcnn_ctx *ctx, int32_t layer, float *dst, int64_t n);
/* Copy the node-level predictions (Sec. 3.1 atom-level properties; N floats,
 * atom order of the batch) of the last forward to host memory dst (caller-
 * owned); GCNN_ESTATE without the node head, GCNN_EINVAL unless n = N.
 * Synchronous. */
int gcnn_get_node_predictions(gcnn_ctx *ctx, float *dst, int64_t n);

/* ------------------------------------------------------------------ timing
 * Per-phase device time of the step (the paper's load / forward / backward /
 * optimizer breakdown, Fig. 5, at kernel granularity).  While enabled, the
 * library records a CUDA event pair on the context's stream around every
 * kernel it launches outside graph capture, and gcnn_train_step runs eagerly.
 */
enum {
  GCNN_PHASE_COLLATE = 0,   /* device collation                         */
  GCNN_PHASE_EMBED = 1,     /* embedding lookup                         */
  GCNN_PHASE_GEMM = 2,      /* dense node-wise GEMMs (fwd and bwd)      */
  GCNN_PHASE_AGG_FWD = 3,   /* gather + aggregate (fwd, and recompute)  */
  GCNN_PHASE_AGG_BWD = 4,   /* aggregate backward                       */
  GCNN_PHASE_HEAD = 5,      /* pooling, head, loss (fwd and bwd)        */
  GCNN_PHASE_EMBED_BWD = 6, /* embedding gradient                       */
  GCNN_PHASE_ADAM = 7,      /* optimizer                                */
  GCNN_NPHASE = 8
};
/* With profiling on, gcnn_train_step replays a separately captured graph that
 * carries event-record nodes around every phase (so the kernels are timed as
 * they run inside a graph) and synchronises the stream after each step;
 * other calls time their launches with eager events. */
int gcnn_profile_enable(gcnn_ctx *ctx, int enable);
/* Synchronises the stream; returns per-phase milliseconds and numbers of
 * timed launches since the last read (host arrays of GCNN_NPHASE), then
 * resets the counters. */
int gcnn_profile_read(gcnn_ctx *ctx, double *ms, int64_t *launches);
/* Device bytes held by the context (parameters, optimiser state, batch,
 * activations and workspace; one allocation made by gcnn_create). */
int gcnn_memory(const gcnn_ctx *ctx, int64_t *arena_bytes);
/* Kernels in the CUDA graph of the most recent gcnn_train_step or
 * gcnn_train_step_range (0 if it ran eagerly; the latter's count includes its
 * collation); a separate collation of a batch adds 1 more launch for at most
 * 1024 graphs, 2 beyond. */
int gcnn_step_kernel_count(gcnn_ctx *ctx, int32_t *n);

/* Kernel timeline.  While enabled, block 0 of every kernel of the library
 * appends one record (kernel id, device clock in ns) right after the kernel's
 * dependency on the previous work in its stream is satisfied.  Inside a
 * serial stream or graph that moment is the completion of the previous
 * kernel, so consecutive records give each kernel's in-stream duration.  The
 * timeline is process-wide on the calling thread's device (every context's
 * kernels append) and holds at most `capacity` records; records past it are
 * dropped.  Not a paper operation: measurement support.
 *   gcnn_timeline_enable: capacity > 0 allocates (or resizes) the device
 *     buffer and clears it; 0 disables recording and frees it.  Call it with
 *     no library kernel in flight.
 *   gcnn_timeline_read: synchronises the device, copies up to `max` records
 *     (ids into `ids`, times into `t_ns`, both host arrays) in append order,
 *     sets *n to the number copied and clears the buffer.  GCNN_ESTATE when
 *     the timeline is not enabled. */
enum {
  GCNN_K_COLLATE_SCAN = 1,
  GCNN_K_COLLATE_GRAPH = 2,
  GCNN_K_EMBED = 3,
  GCNN_K_EMBED_BWD = 4,
  GCNN_K_AGG_FWD = 5,
  GCNN_K_AGG_BWD_EDGE = 6,
  GCNN_K_AGG_BWD_GATHER = 7,
  GCNN_K_GEMM_TC_PARTIAL = 8,   /* tensor-core GEMM writing split-K partials   */
  GCNN_K_GEMM_TC_C = 9,         /* tensor-core GEMM, C / C16 epilogue          */
  GCNN_K_GEMM_TC_D3 = 10,       /* tensor-core GEMM, masked gradient epilogue  */
  GCNN_K_GEMM_TC_REDUCE = 11,   /* split-K reduction and epilogue              */
  GCNN_K_GEMM_SIMT = 12,
  GCNN_K_GEMM_SIMT_REDUCE = 13,
  GCNN_K_POOL_FWD = 14,
  GCNN_K_POOL_BWD = 15,
  GCNN_K_HEAD_GRAPH = 16,
  GCNN_K_HEAD_GRAD = 17,
  GCNN_K_COLSUM = 18,
  GCNN_K_ADAM = 19,
  GCNN_K_CAST_BF16 = 20,
  GCNN_K_PACK_LAYER = 21,
  GCNN_K_STEP_END = 22,         /* marker after a train step (timeline on only) */
  GCNN_K_AGG_BWD_FUSED = 23,    /* aggregation backward over whole graphs      */
  GCNN_K_AGG_BWD_CHUNKS = 24,   /* its partition of the batch into chunks      */
  GCNN_K_NODE_PRED = 25,        /* node-level head: outputs and loss gradient  */
  GCNN_K_NODE_GRAD = 26,        /* node-level head: w2n, b2n and loss sums     */
  GCNN_K_BOND_GRAD = 27,        /* gradient of the bond rows of W_M            */
  GCNN_K_COLLATE = 28,          /* collation of <= 1024 graphs in one launch   */
  GCNN_NKERNEL = 28
};
int gcnn_timeline_enable(gcnn_ctx *ctx, int32_t capacity);
int gcnn_timeline_read(gcnn_ctx *ctx, int32_t *ids, int64_t *t_ns, int32_t max, int32_t *n);

/* FP32 FFMA throughput of the calling thread's device, in TFLOP/s: a kernel
 * of independent fused multiply-add chains over every SM (full occupancy),
 * timed with CUDA events over `iters` loop trips per thread after a warm-up
 * launch; synchronous.  The roofline of the FP32 (CUDA-core) GEMM path.  Not a
 * paper operation: measurement support.  GCNN_EINVAL for iters < 1. */
int gcnn_ffma_peak(int32_t iters, double *tflops);

/* Timing study of the BF16 tensor-core GEMMs of one training step, for a
 * batch of n_atoms atoms and hidden width `hidden` (a multiple of 8, at most
 * 256), on the calling thread's device; synchronous.  Six shapes: 0 message
 * (x [A | B]), 1 update (U W_U), 2 dW_U, 3 dagg, 4 dW_M, 5 dx (dW_U and dW_M
 * with the CTA limit of the backward's second stream).
 * Each time is the best of five replays of a CUDA graph of 20 launches, in
 * microseconds per launch.  mode 0: per shape, the planner's own plan (flag
 * 1), then every plan of its search space: tile width BN (16..128), K-splits,
 * cluster or partial buffer, up to two CTAs per SM.  mode 1: the update shape
 * at K = 64 .. 16 hidden without split-K, at tile widths 32, 64, 112 and 128.
 * Each result row is 8
 * doubles: shape, BN, n-tiles, splits, cluster (0/1), K, microseconds, planner
 * flag; rows beyond max_rows are dropped.  Not a paper operation: measurement
 * support.  GCNN_EINVAL for bad sizes; GCNN_EDEVICE if a wait timed out. */
int gcnn_gemm_study(int32_t n_atoms, int32_t hidden, int32_t mode, double *rows, int32_t max_rows,
                    int32_t *n_rows);

/* ------------------------------------------------------------------ serving
 * Inference server for the screening use of the trained model (Sec. 1:
 * surrogate screening over streaming molecules; Sec. 6).  Requests of any
 * number of molecules are queued on submit; a scheduler thread packs queued
 * molecules (splitting requests when needed) into batches of the smallest
 * node-count bucket that fits, and runs each batch on one of n_slots
 * in-flight slots -- each with its own CUDA stream, device-resident copy of
 * the weights and arena, and one captured CUDA graph per bucket -- so that
 * batches overlap on the device and requests that arrive while others run
 * are admitted as soon as a slot frees up (continuous batching).  Admission
 * is by memory: submit returns GCNN_EAGAIN while the queued molecules would
 * exceed queue_nodes.  Slots use GCNN_FLAG_ROW_INVARIANT, so a molecule's
 * prediction is bit-identical alone and in any mix.
 */
typedef struct gcnn_server gcnn_server;

typedef struct gcnn_serve_config {
  int32_t n_slots;            /* batches in flight (1..16)                       */
  int32_t n_buckets;          /* node-count buckets (1..8)                       */
  int32_t bucket_nodes[8];    /* ascending node capacities, e.g. 1k,4k,16k,64k   */
  int32_t max_graphs;         /* molecules per batch                             */
  int32_t precision;          /* GCNN_PREC_FP32 or GCNN_PREC_BF16                */
  int64_t queue_nodes;        /* atoms of the device request pool: admission is
                                 refused while admitted requests hold it (their
                                 atoms and four edges per atom, until all their
                                 molecules are done); clamped to half of the
                                 device memory left after the slots' arenas   */
} gcnn_serve_config;

typedef struct gcnn_request {
  int32_t n_mol;              /* molecules in the request                        */
  int32_t reserved;
  const int32_t *n_nodes;     /* (host) [n_mol] atoms per molecule (1..255)      */
  const int32_t *n_edges;     /* (host) [n_mol] directed edges per molecule      */
  const uint8_t *types;       /* (host) atom types, molecules concatenated       */
  const uint8_t *edges;       /* (host) local (src, dst) pairs, concatenated;
                                 each bond stored in both directions             */
} gcnn_request;

/* Create a server for the model in `model` (its current parameters are copied
 * to every slot; later changes to `model` are not seen).  Captures every
 * slot's forward graph for every bucket, then starts the scheduler thread.  Requests carry no bond features: a model with
 * edge_features > 0 is refused (GCNN_EINVAL). */
int gcnn_serve_create(const gcnn_ctx *model, const gcnn_serve_config *cfg, gcnn_server **out);
/* Queue a request: its atom types and bonds are copied into the server's
 * device request pool before this returns (the caller may free it then).
 * GCNN_EAGAIN: admission refused (no room in the pool), retry later;
 * GCNN_EINVAL: malformed, or larger than the whole pool. */
int gcnn_serve_submit(gcnn_server *srv, const gcnn_request *req, uint64_t *ticket);
/* Non-blocking: GCNN_EAGAIN until every molecule of the request is done;
 * then writes n_mol predictions to out (host), the latency from submit to
 * completion in microseconds to latency_us (may be NULL), and forgets the
 * ticket. */
int gcnn_serve_poll(gcnn_server *srv, uint64_t ticket, float *out, double *latency_us);
/* Blocking variant with a timeout (GCNN_ETIMEDOUT when it expires). */
int gcnn_serve_wait(gcnn_server *srv, uint64_t ticket, float *out, double *latency_us, int64_t timeout_us);
/* Counters since creation: requests done, molecules done, batches run,
 * submissions refused. */
int gcnn_serve_stats(gcnn_server *srv, int64_t *requests, int64_t *molecules, int64_t *batches,
                     int64_t *refused);
/* Time spent since creation, summed over batches: host_us, the scheduler's
 * time forming and launching batches (packing, copies, graph launches);
 * device_us, each batch's device time from its input copy to its output copy
 * (batches on different slots overlap, so this can exceed wall time); atoms,
 * the batches' atoms; batches, their number.  Measurement support: it says
 * whether the host or the device limits a saturated server. */
int gcnn_serve_timing(gcnn_server *srv, double *host_us, double *device_us, double *atoms, int64_t *batches);
/* Stop the scheduler (finishing batches in flight) and free everything. */
int gcnn_serve_destroy(gcnn_server *srv);

/* ------------------------------------------------------------------ operators
 * Single steps of the path on caller-owned device buffers, for composing the
 * layer from PyTorch (torch.autograd.Function) and for unit tests.
 */
/* agg[i] = [sum, mean, min, max, std] over edges j->i of m_ij = P_i + Q_j,
 * where PQ (N x 2H) holds P in columns 0..H-1 and Q in H..2H-1.
 * agg is N x 5H.  (Sec. 3.1 message passing; PNA aggregators.) */
int gcnn_op_aggregate_fwd(int32_t n_nodes, int32_t hidden, const int32_t *row_ptr,
                          const int32_t *col, const float *PQ, float *agg, float std_eps,
                          void *stream);
/* Gradient of gcnn_op_aggregate_fwd: from dagg (N x 5H) and the forward's
 * PQ and agg, writes dPQ (N x 2H: dP = sum over the row, dQ_j = sum over the
 * edges leaving j).  scratch (device) holds n_edges * hidden floats.  Min/max
 * ties share the gradient equally; no atomics (deterministic). */
int gcnn_op_aggregate_bwd(int32_t n_nodes, int32_t n_edges, int32_t hidden, const int32_t *row_ptr,
                          const int32_t *col, const int32_t *rev, const float *PQ,
                          const float *agg, const float *dagg, float *dPQ, float *scratch,
                          float std_eps, void *stream);
/* Same result as gcnn_op_aggregate_bwd (bitwise) for a batch of n_graphs whole
 * graphs: node_off (device, n_graphs + 1 int32) gives each graph's first node,
 * and no edge may leave its graph (as after gcnn_collate).  Batches of at
 * least 2 x (SM count) x 128 edges run one fused kernel: the batch is cut into
 * chunks of about 128 edges of whole graphs, and each block keeps its chunk's
 * per-edge gradients in shared memory, so they never travel to device memory
 * (graphs too large for that use scratch).  Smaller batches run the kernel
 * pair of gcnn_op_aggregate_bwd.  scratch (device) holds
 * n_edges * hidden + n_edges + 2 floats.  The operators carry no device
 * error flag: an edge that leaves its graph, or an index out of range, is
 * skipped (its gradient is lost) rather than read or written out of bounds.
 * (Sec. 3.1 message passing; PNA aggregators; backward.) */
int gcnn_op_aggregate_bwd_graphs(int32_t n_graphs, int32_t n_nodes, int32_t n_edges, int32_t hidden,
                                 const int32_t *node_off, const int32_t *row_ptr, const int32_t *col,
                                 const int32_t *rev, const float *PQ, const float *agg, const float *dagg,
                                 float *dPQ, float *scratch, float std_eps, void *stream);
/* Same result as gcnn_op_aggregate_bwd, for callers that cannot allocate
 * device memory where they need this gradient (a host framework whose caching
 * allocator already holds the device's memory, or a latency-critical loop in
 * which cudaMalloc/cudaFree, which can synchronise the device, are not
 * allowed).  It allocates nothing: the per-edge scratch is a fixed array of
 * 2^22 floats (16 MiB) inside the library, which every GPU that loads the
 * library holds until the process exits.  n_edges * hidden above 2^22 returns
 * GCNN_EINVAL.  The first call on each device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture.  All calls share the one array and each
 * clears the part it uses, so calls whose GPU work overlaps (on different
 * streams or host threads) race and must be serialised by the caller.  The
 * paper has no counterpart of this entry point; it is a deployment variant. */
int gcnn_op_aggregate_bwd_noalloc(int32_t n_nodes, int32_t n_edges, int32_t hidden, const int32_t *row_ptr,
                                  const int32_t *col, const int32_t *rev, const float *PQ,
                                  const float *agg, const float *dagg, float *dPQ, float std_eps,
                                  void *stream);
/* pooled[g] = mean of x over nodes node_off[g]..node_off[g+1]-1 (Sec. 3.1). */
int gcnn_op_pool_fwd(int32_t n_graphs, int32_t hidden, const int32_t *node_off, const float *x,
                     float *pooled, void *stream);
/* dx[i] = dpooled[graph_id[i]] / n_graph. */
int gcnn_op_pool_bwd(int32_t n_graphs, int32_t n_nodes, int32_t hidden, const int32_t *node_off,
                     const int32_t *graph_id, const float *dpooled, float *dx, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* GCNN_H_ */
