/*
 * FP64 CPU oracle for the GCNN (PNA) training step of HydraGNN
 * (Choi et al., "Scalable training of graph convolutional neural networks for
 * fast and accurate predictions of HOMO-LUMO gap in molecules").
 *
 * TEST INFRASTRUCTURE ONLY.  It is called by the test suite, by the smoke
 * check and by the benchmark's CPU-baseline leg, never by the library.  It
 * shares no code with the CUDA path: it reads the same packed inputs and the
 * same flat parameter layout, and restates every step from its definition,
 * with plain loops and no blocking, fusion or reordering.
 *
 * What it computes (paper sections in brackets):
 *   batch collation of graphs into one disjoint-union graph         [Sec. 1, 4]
 *   atom-type embedding as node features                            [Sec. 3.1]
 *   L PNA graph-convolution layers (message passing)                [Sec. 3.1, 5.1]
 *       message     m_ij = W_M [x_i ; x_j ; e_ij] + b_M   on each edge j->i
 *                   (e_ij: the edge's F bond features, F = 0 without them)
 *       aggregators sum, mean, min, max, std over j in N(i)
 *       scalers     identity, amplification log(d+1)/delta,
 *                   attenuation delta/log(d+1)
 *       update      x_i' = ReLU(W_U [x_i ; scalers (x) aggregators] + b_U)
 *   global mean pooling per graph                                   [Sec. 3.1]
 *   fully connected head  y = W2 ReLU(W1 g + b1) + b2                [Sec. 3.1]
 *   optional node-level head (no pooling)                           [Sec. 3.1, Table 1]
 *       yn_i = w2n . ReLU(W1n^T x_i + b1n) + b2n on the last layer
 *   MSE loss (+ node_weight times the node-level MSE)               [Sec. 3.2]
 *   gradients of the loss w.r.t. every parameter (by hand)          [Sec. 3.2]
 *   Adam / AdamW update                                             [Sec. 3.2, 5.1]
 * The paper names PNA (Corso et al. 2020) but does not print its equations;
 * the layer above is the published PNA definition with one linear message
 * layer (over the two atoms' features and, when the data carry them, the
 * bond's features: Sec. 3.1 and Table 1 name edge attributes), one linear
 * update layer and no towers.
 *
 * Readings where the paper is silent (the same ones the library documents):
 *   std    = sqrt(ReLU(var) + eps), var = (1/d) sum_j (m_ij - mean)^2
 *   d = 0  -> every aggregator is 0; the scalers use max(d, 1)
 *   delta  = mean over the training nodes of log(d + 1)
 *   amp/att are computed in FP64 and rounded once to float32
 *   min/max ties share the gradient equally among all tied entries
 *   ReLU'(0) = 0
 *
 * Parameter layout (float32 in the library, double here), in order:
 *   emb[T][H]
 *   per layer: msg_w[H][2H] (columns 0..H-1 act on x_i, H..2H-1 on x_j),
 *              msg_b[H], upd_w[16H][H] (rows: x_i, then scaler-major blocks
 *              id{sum,mean,min,max,std}, amp{...}, att{...}), upd_b[H]
 *   head: w1[H][Hh], b1[Hh], w2[Hh], b2
 *   with F bond features: 0..3 unused floats up to the next multiple of 4,
 *   then per layer edge_w[F][H] (the bond rows of W_M)
 *   with the node head: 0..3 unused floats up to the next multiple of 4,
 *   then w1n[H][Hh], b1n[Hh], w2n[Hh], b2n
 * so that W_M(k, c) for the stacked input [x_i ; x_j ; e_ij] is msg_w[k][c]
 * for k < H, msg_w[k-H][H+c] for H <= k < 2H and edge_w[k-2H][c] after.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NAGG 5
#define NSCL 3

/* ------------------------------------------------------------ collation */

/*
 * Disjoint union of graphs ids[0..G) from a packed store (global arrays).
 * Outputs (caller-allocated, N and E = total nodes / edges of the batch):
 *   node_off[G+1], edge_off[G+1]   prefix sums of node / edge counts
 *   graph_id[N]                    graph of each node
 *   row_ptr[N+1], col[E]           in-edges grouped by destination, each
 *                                  group sorted by source (col = source)
 *   rev[E]                         position of the reverse edge
 *   deg[N]                         in-degree
 *   amp[N], att[N]                 degree scalers (FP64, rounded to float)
 *   types[N], y[G]                 gathered node types and targets
 *   eattr[E][F]                    bond features of each edge, in the order
 *                                  of col (F = 0: not used)
 *   ynode[N]                       node-level targets (when st_ynode != NULL)
 */
int oracle_collate(int64_t G, const int64_t *ids, const int64_t *st_node_ptr,
                   const int64_t *st_edge_ptr, const uint8_t *st_types,
                   const uint8_t *st_edges, const float *st_y, double delta,
                   int64_t *node_off, int64_t *edge_off, int32_t *graph_id,
                   int32_t *row_ptr, int32_t *col, int32_t *rev, int32_t *deg,
                   float *amp, float *att, uint8_t *types, float *y, int F,
                   const float *st_eattr, float *eattr, const float *st_ynode, float *ynode) {
  node_off[0] = 0;
  edge_off[0] = 0;
  for (int64_t g = 0; g < G; ++g) {
    int64_t id = ids[g];
    node_off[g + 1] = node_off[g] + (st_node_ptr[id + 1] - st_node_ptr[id]);
    edge_off[g + 1] = edge_off[g] + (st_edge_ptr[id + 1] - st_edge_ptr[id]);
  }
  int64_t N = node_off[G], E = edge_off[G];
  int64_t *src = (int64_t *)malloc(sizeof(int64_t) * (E + 1));
  int64_t *dst = (int64_t *)malloc(sizeof(int64_t) * (E + 1));
  int64_t *sid = (int64_t *)malloc(sizeof(int64_t) * (E + 1));  /* store index of each edge */
  if (!src || !dst || !sid) { free(src); free(dst); free(sid); return -1; }

  /* global node ids and node attributes */
  for (int64_t g = 0; g < G; ++g) {
    int64_t id = ids[g];
    int64_t n = node_off[g + 1] - node_off[g];
    for (int64_t v = 0; v < n; ++v) {
      graph_id[node_off[g] + v] = (int32_t)g;
      types[node_off[g] + v] = st_types[st_node_ptr[id] + v];
      if (st_ynode) ynode[node_off[g] + v] = st_ynode[st_node_ptr[id] + v];
    }
    int64_t e = edge_off[g + 1] - edge_off[g];
    for (int64_t k = 0; k < e; ++k) {
      const uint8_t *pair = st_edges + 2 * (st_edge_ptr[id] + k);
      src[edge_off[g] + k] = node_off[g] + pair[0];
      dst[edge_off[g] + k] = node_off[g] + pair[1];
      sid[edge_off[g] + k] = st_edge_ptr[id] + k;
    }
    y[g] = st_y[id];
  }

  /* in-degree and row offsets */
  for (int64_t i = 0; i < N; ++i) deg[i] = 0;
  for (int64_t k = 0; k < E; ++k) deg[dst[k]] += 1;
  row_ptr[0] = 0;
  for (int64_t i = 0; i < N; ++i) row_ptr[i + 1] = row_ptr[i] + deg[i];

  /* place each edge in its destination's row, then sort the row by source
     (a stable sort: edges with the same source keep their store order) */
  int32_t *fill = (int32_t *)calloc((size_t)(N + 1), sizeof(int32_t));
  int64_t *pos_sid = (int64_t *)malloc(sizeof(int64_t) * (E + 1));
  if (!fill || !pos_sid) { free(src); free(dst); free(sid); free(fill); free(pos_sid); return -1; }
  for (int64_t k = 0; k < E; ++k) {
    int64_t i = dst[k];
    col[row_ptr[i] + fill[i]] = (int32_t)src[k];
    pos_sid[row_ptr[i] + fill[i]] = sid[k];
    fill[i] += 1;
  }
  for (int64_t i = 0; i < N; ++i) {
    for (int32_t a = row_ptr[i] + 1; a < row_ptr[i + 1]; ++a) { /* insertion sort */
      int32_t v = col[a];
      int64_t vs = pos_sid[a];
      int32_t b = a - 1;
      while (b >= row_ptr[i] && col[b] > v) { col[b + 1] = col[b]; pos_sid[b + 1] = pos_sid[b]; --b; }
      col[b + 1] = v;
      pos_sid[b + 1] = vs;
    }
  }
  for (int64_t p = 0; p < E; ++p)
    for (int f = 0; f < F; ++f) eattr[p * F + f] = st_eattr[pos_sid[p] * F + f];
  /* reverse edge: the edge i -> j sits in row j with source i */
  for (int64_t i = 0; i < N; ++i) {
    for (int32_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
      int32_t j = col[p];
      rev[p] = -1;
      for (int32_t q = row_ptr[j]; q < row_ptr[j + 1]; ++q)
        if (col[q] == (int32_t)i) { rev[p] = q; break; }
    }
  }
  /* degree scalers */
  for (int64_t i = 0; i < N; ++i) {
    double d = deg[i] > 1 ? (double)deg[i] : 1.0;
    amp[i] = (float)(log(d + 1.0) / delta);
    att[i] = (float)(delta / log(d + 1.0));
  }
  free(fill);
  free(pos_sid);
  free(src);
  free(dst);
  free(sid);
  return 0;
}

/* delta = (1/N) sum_i log(d_i + 1) over the given in-degrees. */
double oracle_delta(int64_t N, const int32_t *deg) {
  double s = 0.0;
  for (int64_t i = 0; i < N; ++i) s += log((double)deg[i] + 1.0);
  return N > 0 ? s / (double)N : 1.0;
}

/* ------------------------------------------------------------ model */

typedef struct {
  int H, L, T, Hh, F, NH;  /* NH: node-level head present (0/1) */
  int64_t G, N, E;
  const float *eattr;  /* E x F bond features in col order */
  const float *ynode;  /* N node-level targets (NH = 1) */
  double node_weight;  /* weight of the node-level MSE in the loss */
  const int64_t *node_off;
  const int32_t *graph_id, *row_ptr, *col, *deg;
  const float *amp, *att;
  const uint8_t *types;
  double eps;
} net_t;

typedef struct {
  const double *msg_w, *msg_b, *upd_w, *upd_b, *edge_w;
} layer_t;

static int64_t layer_size(int H) {
  return (int64_t)H * 2 * H + H + (int64_t)16 * H * H + H;
}

static int64_t head_size(int H, int Hh) { return (int64_t)H * Hh + Hh + Hh + 1; }

/* first bond row: after the head, rounded up to a multiple of 4 floats */
static int64_t bonds_offset(int H, int L, int T, int Hh) {
  return ((int64_t)T * H + L * layer_size(H) + head_size(H, Hh) + 3) / 4 * 4;
}

static int64_t trunk_end(int H, int L, int T, int Hh, int F) {
  if (F == 0) return (int64_t)T * H + L * layer_size(H) + head_size(H, Hh);
  return bonds_offset(H, L, T, Hh) + (int64_t)L * F * H;
}

/* node head: after the bond rows (or the head), from the next multiple of 4 */
static int64_t node_head_offset(int H, int L, int T, int Hh, int F) {
  return (trunk_end(H, L, T, Hh, F) + 3) / 4 * 4;
}

int64_t oracle_param_count(int H, int L, int T, int Hh, int F, int NH) {
  if (!NH) return trunk_end(H, L, T, Hh, F);
  return node_head_offset(H, L, T, Hh, F) + head_size(H, Hh);
}

static layer_t layer_at(const net_t *n, const double *p, int l) {
  layer_t w;
  const double *b = p + (int64_t)n->T * n->H + l * layer_size(n->H);
  w.msg_w = b;
  w.msg_b = w.msg_w + (int64_t)n->H * 2 * n->H;
  w.upd_w = w.msg_b + n->H;
  w.upd_b = w.upd_w + (int64_t)16 * n->H * n->H;
  w.edge_w = p + bonds_offset(n->H, n->L, n->T, n->Hh) + (int64_t)l * n->F * n->H;
  return w;
}

static int64_t head_offset(const net_t *n) {
  return (int64_t)n->T * n->H + n->L * layer_size(n->H);
}

/* W_M(k, c) of the stacked input [x_i ; x_j] (2H x H). */
static double wm(const net_t *n, const double *msg_w, int k, int c) {
  int H = n->H;
  return k < H ? msg_w[(int64_t)k * 2 * H + c] : msg_w[(int64_t)(k - H) * 2 * H + H + c];
}

/* scaler s (0 identity, 1 amplification, 2 attenuation) of node i */
static double scaler(const net_t *n, int64_t i, int s) {
  return s == 0 ? 1.0 : (s == 1 ? (double)n->amp[i] : (double)n->att[i]);
}

/* m[e][c] = b_M[c] + sum_k W_M(k,c) [x_i ; x_j ; e_ij]_k for the edge e = (j -> i) */
static void messages(const net_t *n, const layer_t *w, const double *x, double *m) {
  int H = n->H;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n->N; ++i) {
    for (int32_t e = n->row_ptr[i]; e < n->row_ptr[i + 1]; ++e) {
      int64_t j = n->col[e];
      for (int c = 0; c < H; ++c) {
        double acc = w->msg_b[c];
        for (int k = 0; k < H; ++k) acc += wm(n, w->msg_w, k, c) * x[i * H + k];
        for (int k = 0; k < H; ++k) acc += wm(n, w->msg_w, H + k, c) * x[j * H + k];
        for (int f = 0; f < n->F; ++f) acc += w->edge_w[(int64_t)f * H + c] * (double)n->eattr[(int64_t)e * n->F + f];
        m[(int64_t)e * H + c] = acc;
      }
    }
  }
}

/* agg[i] = [sum, mean, min, max, std] over the messages into node i */
static void aggregate(const net_t *n, const double *m, double *agg) {
  int H = n->H;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n->N; ++i) {
    int32_t r0 = n->row_ptr[i], r1 = n->row_ptr[i + 1];
    double d = (double)(r1 - r0);
    double *a = agg + i * NAGG * H;
    for (int c = 0; c < H; ++c) {
      if (r1 == r0) {
        for (int q = 0; q < NAGG; ++q) a[q * H + c] = 0.0;
        continue;
      }
      double sum = 0.0, mn = INFINITY, mx = -INFINITY;
      for (int32_t e = r0; e < r1; ++e) {
        double v = m[(int64_t)e * H + c];
        sum += v;
        if (v < mn) mn = v;
        if (v > mx) mx = v;
      }
      double mean = sum / d;
      double var = 0.0;
      for (int32_t e = r0; e < r1; ++e) {
        double t = m[(int64_t)e * H + c] - mean;
        var += t * t;
      }
      var /= d;
      a[0 * H + c] = sum;
      a[1 * H + c] = mean;
      a[2 * H + c] = mn;
      a[3 * H + c] = mx;
      a[4 * H + c] = sqrt((var > 0.0 ? var : 0.0) + n->eps);
    }
  }
}

/*
 * Backward of the five aggregators (Sec. 3.1): the gradient dm[e] of the
 * loss w.r.t. every message m[e] into node i, given the forward's agg[i]
 * (sum, mean, min, max, std) and the incoming dagg[i]:
 *   sum: 1 ; mean: 1/d ; min / max: 1 / (number of tied extrema) at each
 *   extremum, 0 elsewhere ; std = sqrt(var + eps): (m - mean) / (d std)
 *   (0 when var = 0, where the derivative of the ReLU is taken as 0).
 */
static void aggregate_backward(const net_t *n, const double *msg, const double *agg, const double *dagg,
                               double *dm) {
  int H = n->H;
  const int32_t *row_ptr = n->row_ptr;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n->N; ++i) {
    int32_t r0 = row_ptr[i], r1 = row_ptr[i + 1];
    if (r1 == r0) continue;
    double d = (double)(r1 - r0);
    const double *a = agg + i * NAGG * H;
    const double *da = dagg + i * NAGG * H;
    for (int c = 0; c < H; ++c) {
      double mean = a[1 * H + c], mn = a[2 * H + c], mx = a[3 * H + c], sd = a[4 * H + c];
      double var = 0.0;
      int nmin = 0, nmax = 0;
      for (int32_t e = r0; e < r1; ++e) {
        double v = msg[(int64_t)e * H + c];
        var += (v - mean) * (v - mean);
        nmin += (v == mn);
        nmax += (v == mx);
      }
      var /= d;
      for (int32_t e = r0; e < r1; ++e) {
        double v = msg[(int64_t)e * H + c];
        double g = da[0 * H + c] + da[1 * H + c] / d;      /* sum, mean */
        if (v == mn) g += da[2 * H + c] / nmin;            /* min, ties share */
        if (v == mx) g += da[3 * H + c] / nmax;            /* max, ties share */
        if (var > 0.0) g += da[4 * H + c] * (v - mean) / (d * sd);  /* std */
        dm[(int64_t)e * H + c] = g;
      }
    }
  }
}

/* u_i = [x_i ; id*agg_i ; amp_i*agg_i ; att_i*agg_i]  (16H) */
static void update_input(const net_t *n, const double *x, const double *agg, int64_t i, double *u) {
  int H = n->H;
  for (int k = 0; k < H; ++k) u[k] = x[i * H + k];
  for (int s = 0; s < NSCL; ++s)
    for (int r = 0; r < NAGG * H; ++r)
      u[H + s * NAGG * H + r] = scaler(n, i, s) * agg[i * NAGG * H + r];
}

/* pre_i = b_U + W_U^T u_i ; h_i = ReLU(pre_i) */
static void update(const net_t *n, const layer_t *w, const double *x, const double *agg,
                   double *pre, double *h) {
  int H = n->H;
#pragma omp parallel
  {
    double *u = (double *)malloc(sizeof(double) * 16 * H);
#pragma omp for schedule(static)
    for (int64_t i = 0; i < n->N; ++i) {
      update_input(n, x, agg, i, u);
      for (int c = 0; c < H; ++c) {
        double acc = w->upd_b[c];
        for (int k = 0; k < 16 * H; ++k) acc += u[k] * w->upd_w[(int64_t)k * H + c];
        pre[i * H + c] = acc;
        h[i * H + c] = acc > 0.0 ? acc : 0.0;
      }
    }
    free(u);
  }
}

/* g[gr] = mean of x over the nodes of graph gr */
static void mean_pool(const net_t *n, const double *x, double *g) {
  int H = n->H;
  for (int64_t gr = 0; gr < n->G; ++gr) {
    int64_t a = n->node_off[gr], b = n->node_off[gr + 1];
    for (int k = 0; k < H; ++k) {
      double s = 0.0;
      for (int64_t i = a; i < b; ++i) s += x[i * H + k];
      g[gr * H + k] = b > a ? s / (double)(b - a) : 0.0;
    }
  }
}

/* z1 = W1^T g + b1 ; y = w2 . ReLU(z1) + b2 */
static void head(const net_t *n, const double *p, const double *g, double *z1, double *pred) {
  int H = n->H, Hh = n->Hh;
  const double *w1 = p + head_offset(n), *b1 = w1 + (int64_t)H * Hh, *w2 = b1 + Hh, *b2 = w2 + Hh;
  for (int64_t gr = 0; gr < n->G; ++gr) {
    double out = b2[0];
    for (int c = 0; c < Hh; ++c) {
      double acc = b1[c];
      for (int k = 0; k < H; ++k) acc += g[gr * H + k] * w1[(int64_t)k * Hh + c];
      z1[gr * Hh + c] = acc;
      out += (acc > 0.0 ? acc : 0.0) * w2[c];
    }
    pred[gr] = out;
  }
}

/* node-level head on the last layer: zn_i = W1n^T x_i + b1n ;
   predn_i = w2n . ReLU(zn_i) + b2n  (no pooling: one output per atom) */
static void node_head(const net_t *n, const double *p, const double *x, double *zn, double *predn) {
  int H = n->H, Hh = n->Hh;
  const double *w1 = p + node_head_offset(H, n->L, n->T, Hh, n->F), *b1 = w1 + (int64_t)H * Hh;
  const double *w2 = b1 + Hh, *b2 = w2 + Hh;
  for (int64_t i = 0; i < n->N; ++i) {
    double out = b2[0];
    for (int c = 0; c < Hh; ++c) {
      double z = b1[c];
      for (int k = 0; k < H; ++k) z += x[i * H + k] * w1[(int64_t)k * Hh + c];
      zn[i * Hh + c] = z;
      out += (z > 0.0 ? z : 0.0) * w2[c];
    }
    predn[i] = out;
  }
}

static void embed(const net_t *n, const double *p, double *x0) {
  int H = n->H;
  for (int64_t i = 0; i < n->N; ++i)
    for (int k = 0; k < H; ++k) x0[i * H + k] = p[(int64_t)n->types[i] * H + k];
}

static void net_init(net_t *n, int H, int L, int T, int Hh, int F, int NH, int64_t G, int64_t N, int64_t E,
                     const int64_t *node_off, const int32_t *graph_id, const int32_t *row_ptr,
                     const int32_t *col, const int32_t *deg, const float *amp, const float *att,
                     const uint8_t *types, const float *eattr, const float *ynode, double node_weight,
                     double eps) {
  n->H = H; n->L = L; n->T = T; n->Hh = Hh; n->F = F; n->eattr = eattr;
  n->NH = NH; n->ynode = ynode; n->node_weight = node_weight;
  n->G = G; n->N = N; n->E = E;
  n->node_off = node_off; n->graph_id = graph_id; n->row_ptr = row_ptr; n->col = col;
  n->deg = deg; n->amp = amp; n->att = att; n->types = types; n->eps = eps;
}

/* Forward pass state: xs[(L+1)][N][H], pre[L][N][H], agg[L][N][5H], g, z1. */
typedef struct {
  double *xs, *pre, *agg, *msg, *g, *z1, *zn, *predn;
} fwd_t;

static int fwd_alloc(const net_t *n, fwd_t *f) {
  int H = n->H;
  f->xs = (double *)calloc((size_t)((n->L + 1) * n->N * H + 1), sizeof(double));
  f->pre = (double *)calloc((size_t)(n->L * n->N * H + 1), sizeof(double));
  f->agg = (double *)calloc((size_t)(n->L * n->N * NAGG * H + 1), sizeof(double));
  f->msg = (double *)calloc((size_t)(n->E * H + 1), sizeof(double));
  f->g = (double *)calloc((size_t)(n->G * H + 1), sizeof(double));
  f->z1 = (double *)calloc((size_t)(n->G * n->Hh + 1), sizeof(double));
  f->zn = (double *)calloc((size_t)(n->NH ? n->N * n->Hh + 1 : 1), sizeof(double));
  f->predn = (double *)calloc((size_t)(n->N + 1), sizeof(double));
  return (f->xs && f->pre && f->agg && f->msg && f->g && f->z1 && f->zn && f->predn) ? 0 : -1;
}

static void fwd_free(fwd_t *f) {
  free(f->xs); free(f->pre); free(f->agg); free(f->msg); free(f->g); free(f->z1); free(f->zn); free(f->predn);
}

static void forward(const net_t *n, const double *p, const double *x0_in, fwd_t *f, double *pred) {
  int64_t NH = n->N * n->H;
  if (x0_in) memcpy(f->xs, x0_in, sizeof(double) * NH);
  else embed(n, p, f->xs);
  for (int l = 0; l < n->L; ++l) {
    layer_t w = layer_at(n, p, l);
    messages(n, &w, f->xs + l * NH, f->msg);
    aggregate(n, f->msg, f->agg + l * NH * NAGG);
    update(n, &w, f->xs + l * NH, f->agg + l * NH * NAGG, f->pre + l * NH, f->xs + (l + 1) * NH);
  }
  mean_pool(n, f->xs + n->L * NH, f->g);
  head(n, p, f->g, f->z1, pred);
  if (n->NH) node_head(n, p, f->xs + n->L * NH, f->zn, f->predn);
}

/*
 * Forward pass.  x0_in (N x H) replaces the embedding when not NULL.
 * Optional outputs: xs_out ((L+1) x N x H, layer inputs/outputs),
 * agg_out (L x N x 5H), pooled_out (G x H).
 */
int oracle_forward(int H, int L, int T, int Hh, int F, int NH, const double *params, int64_t G, int64_t N,
                   int64_t E, const int64_t *node_off, const int32_t *graph_id,
                   const int32_t *row_ptr, const int32_t *col, const int32_t *deg,
                   const float *amp, const float *att, const uint8_t *types, const float *eattr,
                   const float *ynode, const double *x0_in, double eps, double node_weight, double *pred,
                   double *xs_out, double *agg_out, double *pooled_out, double *predn_out) {
  net_t n;
  fwd_t f;
  net_init(&n, H, L, T, Hh, F, NH, G, N, E, node_off, graph_id, row_ptr, col, deg, amp, att, types, eattr, ynode,
           node_weight, eps);
  if (fwd_alloc(&n, &f)) { fwd_free(&f); return -1; }
  forward(&n, params, x0_in, &f, pred);
  if (predn_out && NH) memcpy(predn_out, f.predn, sizeof(double) * (size_t)N);
  if (xs_out) memcpy(xs_out, f.xs, sizeof(double) * (size_t)((L + 1) * N * H));
  if (agg_out) memcpy(agg_out, f.agg, sizeof(double) * (size_t)(L * N * NAGG * H));
  if (pooled_out) memcpy(pooled_out, f.g, sizeof(double) * (size_t)(G * H));
  fwd_free(&f);
  return 0;
}

/*
 * Loss and gradients.  With dpred_in == NULL the loss is the MSE
 * (1/G) sum_g (pred_g - y_g)^2 and dL/dpred_g = 2 (pred_g - y_g) / G;
 * otherwise dpred_in is used as dL/dpred and *loss is not written.
 * grad has the parameter layout; dx0 (N x H, optional) receives dL/dx0.
 */
int oracle_backward(int H, int L, int T, int Hh, int F, int NHd, const double *params, int64_t G, int64_t N,
                    int64_t E, const int64_t *node_off, const int32_t *graph_id,
                    const int32_t *row_ptr, const int32_t *col, const int32_t *deg,
                    const float *amp, const float *att, const uint8_t *types, const float *eattr,
                    const float *ynode, const double *x0_in, double eps, double node_weight, const float *y,
                    const double *dpred_in, double *grad, double *dx0, double *loss, double *pred_out) {
  net_t n;
  fwd_t f;
  net_init(&n, H, L, T, Hh, F, NHd, G, N, E, node_off, graph_id, row_ptr, col, deg, amp, att, types, eattr, ynode,
           node_weight, eps);
  int64_t NH = N * H;
  int64_t P = oracle_param_count(H, L, T, Hh, F, NHd);
  double *pred = (double *)calloc((size_t)(G + 1), sizeof(double));
  double *dpred = (double *)calloc((size_t)(G + 1), sizeof(double));
  double *dx = (double *)calloc((size_t)(NH + 1), sizeof(double));      /* dL/dx_l   */
  double *dxn = (double *)calloc((size_t)(NH + 1), sizeof(double));     /* dL/dx_l-1 */
  double *dpre = (double *)calloc((size_t)(NH + 1), sizeof(double));
  double *dagg = (double *)calloc((size_t)(NH * NAGG + 1), sizeof(double));
  double *dm = (double *)calloc((size_t)(E * H + 1), sizeof(double));
  double *dg = (double *)calloc((size_t)(G * H + 1), sizeof(double));
  double *tsrc = (double *)calloc((size_t)(E * H + 1), sizeof(double));
  if (fwd_alloc(&n, &f) || !pred || !dpred || !dx || !dxn || !dpre || !dagg || !dm || !dg || !tsrc) {
    fwd_free(&f); free(pred); free(dpred); free(dx); free(dxn); free(dpre); free(dagg); free(dm); free(dg); free(tsrc);
    return -1;
  }
  forward(&n, params, x0_in, &f, pred);
  if (pred_out) memcpy(pred_out, pred, sizeof(double) * G);
  for (int64_t k = 0; k < P; ++k) grad[k] = 0.0;

  /* MSE loss */
  if (dpred_in) {
    for (int64_t g = 0; g < G; ++g) dpred[g] = dpred_in[g];
  } else {
    double l = 0.0;
    for (int64_t g = 0; g < G; ++g) {
      double r = pred[g] - (double)y[g];
      l += r * r;
      dpred[g] = G > 0 ? 2.0 * r / (double)G : 0.0;
    }
    if (loss) *loss = G > 0 ? l / (double)G : 0.0;
  }
  /* node-level MSE, weighted: node_weight (1/N) sum_i (predn_i - yn_i)^2 */
  double *dpredn = (double *)calloc((size_t)(N + 1), sizeof(double));
  if (!dpredn) { fwd_free(&f); free(pred); free(dpred); free(dx); free(dxn); free(dpre); free(dagg); free(dm); free(dg); free(tsrc); return -1; }
  if (NHd) {
    double l = 0.0;
    for (int64_t i = 0; i < N; ++i) {
      double r = f.predn[i] - (double)ynode[i];
      l += r * r;
      dpredn[i] = N > 0 ? node_weight * 2.0 * r / (double)N : 0.0;
    }
    if (loss && !dpred_in) *loss += N > 0 ? node_weight * l / (double)N : 0.0;
  }

  /* head */
  {
    const double *w1 = params + head_offset(&n), *w2 = w1 + (int64_t)H * Hh + Hh;
    double *gw1 = grad + head_offset(&n), *gb1 = gw1 + (int64_t)H * Hh, *gw2 = gb1 + Hh, *gb2 = gw2 + Hh;
    for (int64_t g = 0; g < G; ++g) {
      gb2[0] += dpred[g];
      for (int c = 0; c < Hh; ++c) {
        double z = f.z1[g * Hh + c];
        double a = z > 0.0 ? z : 0.0;
        gw2[c] += a * dpred[g];
        double dz = z > 0.0 ? dpred[g] * w2[c] : 0.0;
        gb1[c] += dz;
        for (int k = 0; k < H; ++k) {
          gw1[(int64_t)k * Hh + c] += f.g[g * H + k] * dz;
          dg[g * H + k] += w1[(int64_t)k * Hh + c] * dz;
        }
      }
    }
  }

  /* mean pool: every node of graph g receives dg / n_g */
  for (int64_t g = 0; g < G; ++g) {
    int64_t a = node_off[g], b = node_off[g + 1];
    for (int64_t i = a; i < b; ++i)
      for (int k = 0; k < H; ++k) dx[i * H + k] = dg[g * H + k] / (double)(b - a);
  }

  /* node head: predn_i = b2n + w2n . ReLU(zn_i), zn_i = b1n + W1n^T x_i */
  if (NHd) {
    const int64_t o = node_head_offset(H, L, T, Hh, F);
    const double *w1 = params + o, *w2 = w1 + (int64_t)H * Hh + Hh;
    double *gw1 = grad + o, *gb1 = gw1 + (int64_t)H * Hh, *gw2 = gb1 + Hh, *gb2 = gw2 + Hh;
    const double *xl = f.xs + (int64_t)L * NH;
    for (int64_t i = 0; i < N; ++i) {
      gb2[0] += dpredn[i];
      for (int c = 0; c < Hh; ++c) {
        double z = f.zn[i * Hh + c];
        gw2[c] += (z > 0.0 ? z : 0.0) * dpredn[i];
        double dz = z > 0.0 ? dpredn[i] * w2[c] : 0.0;
        gb1[c] += dz;
        for (int k = 0; k < H; ++k) {
          gw1[(int64_t)k * Hh + c] += xl[i * H + k] * dz;
          dx[i * H + k] += w1[(int64_t)k * Hh + c] * dz;
        }
      }
    }
  }

  /* conv layers, last to first */
  for (int l = L - 1; l >= 0; --l) {
    layer_t w = layer_at(&n, params, l);
    const double *x = f.xs + l * NH;
    const double *pre = f.pre + l * NH;
    const double *agg = f.agg + l * NH * NAGG;
    double *gbase = grad + (int64_t)T * H + l * layer_size(H);
    double *g_msg_w = gbase, *g_msg_b = g_msg_w + (int64_t)H * 2 * H;
    double *g_upd_w = g_msg_b + H, *g_upd_b = g_upd_w + (int64_t)16 * H * H;

    /* ReLU */
    for (int64_t q = 0; q < NH; ++q) dpre[q] = pre[q] > 0.0 ? dx[q] : 0.0;

    /* update layer: pre_i = b_U + W_U^T u_i */
    for (int c = 0; c < H; ++c) {
      double s = 0.0;
      for (int64_t i = 0; i < N; ++i) s += dpre[i * H + c];
      g_upd_b[c] += s;
    }
#pragma omp parallel for schedule(static)
    for (int k = 0; k < 16 * H; ++k) {           /* dW_U[k][c] = sum_i u_i[k] dpre_i[c] */
      for (int64_t i = 0; i < N; ++i) {
        double uk;
        if (k < H) uk = x[i * H + k];
        else uk = scaler(&n, i, (k - H) / (NAGG * H)) * agg[i * NAGG * H + (k - H) % (NAGG * H)];
        for (int c = 0; c < H; ++c) g_upd_w[(int64_t)k * H + c] += uk * dpre[i * H + c];
      }
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {           /* du_i = W_U dpre_i, split into dx_i and da_i */
      for (int q = 0; q < H; ++q) dxn[i * H + q] = 0.0;
      for (int q = 0; q < NAGG * H; ++q) dagg[i * NAGG * H + q] = 0.0;
      for (int k = 0; k < 16 * H; ++k) {
        double s = 0.0;
        for (int c = 0; c < H; ++c) s += w.upd_w[(int64_t)k * H + c] * dpre[i * H + c];
        if (k < H) {
          dxn[i * H + k] += s;
        } else {
          int sc = (k - H) / (NAGG * H), r = (k - H) % (NAGG * H);
          dagg[i * NAGG * H + r] += scaler(&n, i, sc) * s;
        }
      }
    }

    /* aggregators -> per-edge message gradients */
    messages(&n, &w, x, f.msg);
    aggregate_backward(&n, f.msg, agg, dagg, dm);

    /* message layer: m_ij = b_M + W_M^T [x_i ; x_j ; e_ij], edge e = (j -> i) in row i */
    for (int c = 0; c < H; ++c) {
      double s = 0.0;
      for (int64_t e = 0; e < E; ++e) s += dm[e * H + c];
      g_msg_b[c] += s;
    }
    if (F > 0) {                                  /* bond rows: dW_E[f][c] = sum_e e_ij[f] dm_ij[c] */
      double *g_edge_w = grad + (w.edge_w - params);
      for (int fi = 0; fi < F; ++fi)
        for (int c = 0; c < H; ++c) {
          double s = 0.0;
          for (int64_t e = 0; e < E; ++e) s += (double)eattr[e * F + fi] * dm[e * H + c];
          g_edge_w[(int64_t)fi * H + c] += s;
        }
    }
#pragma omp parallel for schedule(static)
    for (int k = 0; k < H; ++k) {                /* dW_M over all edges */
      for (int64_t i = 0; i < N; ++i) {
        for (int32_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
          int64_t j = col[e];
          for (int c = 0; c < H; ++c) {
            double d = dm[(int64_t)e * H + c];
            g_msg_w[(int64_t)k * 2 * H + c] += x[i * H + k] * d;
            g_msg_w[(int64_t)k * 2 * H + H + c] += x[j * H + k] * d;
          }
        }
      }
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {           /* destination side: dx_i += W_M[:H] dm_ij */
      for (int32_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
        for (int k = 0; k < H; ++k) {
          double s = 0.0;
          for (int c = 0; c < H; ++c) s += wm(&n, w.msg_w, k, c) * dm[(int64_t)e * H + c];
          dxn[i * H + k] += s;
        }
    }
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < E; ++e) {           /* source side: t_e = W_M[H:] dm_ij */
      for (int k = 0; k < H; ++k) {
        double s = 0.0;
        for (int c = 0; c < H; ++c) s += wm(&n, w.msg_w, H + k, c) * dm[e * H + c];
        tsrc[e * H + k] = s;
      }
    }
    for (int64_t e = 0; e < E; ++e) {           /* ... scattered to the source x_j */
      int64_t j = col[e];
      for (int k = 0; k < H; ++k) dxn[j * H + k] += tsrc[e * H + k];
    }
    double *t = dx; dx = dxn; dxn = t;
  }

  /* embedding (or the continuous node input) */
  if (dx0) memcpy(dx0, dx, sizeof(double) * NH);
  if (!x0_in)
    for (int64_t i = 0; i < N; ++i)
      for (int k = 0; k < H; ++k) grad[(int64_t)types[i] * H + k] += dx[i * H + k];

  fwd_free(&f);
  free(pred); free(dpred); free(dx); free(dxn); free(dpre); free(dagg); free(dm); free(dg); free(tsrc); free(dpredn);
  return 0;
}

/* ------------------------------------------------------------ operators */

/*
 * The aggregation step alone (Sec. 3.1), on given messages: m[E][H] holds
 * the message of every edge slot, the slots of node i being
 * row_ptr[i]..row_ptr[i+1]-1.  agg[N][5H] receives [sum, mean, min, max,
 * std] per node (all 0 for a node without in-edges).
 */
void oracle_aggregate_op(int64_t N, int H, const int32_t *row_ptr, const double *m, double eps, double *agg) {
  net_t n;
  memset(&n, 0, sizeof(n));
  n.N = N; n.H = H; n.row_ptr = row_ptr; n.eps = eps;
  aggregate(&n, m, agg);
}

/*
 * Its backward: dm[E][H] = dL/dm for every edge slot from dagg[N][5H] and
 * the forward's agg (oracle_aggregate_op of the same messages).
 */
void oracle_aggregate_bwd_op(int64_t N, int H, const int32_t *row_ptr, const double *m, const double *agg,
                             const double *dagg, double *dm) {
  net_t n;
  memset(&n, 0, sizeof(n));
  n.N = N; n.H = H; n.row_ptr = row_ptr;
  aggregate_backward(&n, m, agg, dagg, dm);
}

/*
 * Adam with decoupled weight decay (AdamW), step number t >= 1:
 *   theta <- theta - lr * wd * theta
 *   m <- b1 m + (1 - b1) g ;  v <- b2 v + (1 - b2) g^2
 *   theta <- theta - lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)
 */
void oracle_adam(int64_t P, double *theta, const double *grad, double *m, double *v, int64_t t,
                 double lr, double b1, double b2, double eps, double wd) {
  double c1 = 1.0 - pow(b1, (double)t), c2 = 1.0 - pow(b2, (double)t);
  for (int64_t k = 0; k < P; ++k) {
    if (wd > 0.0) theta[k] -= lr * wd * theta[k];
    m[k] = b1 * m[k] + (1.0 - b1) * grad[k];
    v[k] = b2 * v[k] + (1.0 - b2) * grad[k] * grad[k];
    theta[k] -= lr * (m[k] / c1) / (sqrt(v[k] / c2) + eps);
  }
}
