/*
 * Seeded synthetic inputs for the GCNN training step: molecule-shaped graphs,
 * atom types, targets drawn at random, and the initial parameter vector.
 *
 * This module is shared by the FP64 oracle and the CUDA path as their common
 * source of inputs.  It holds none of the method's arithmetic (no message,
 * aggregation, scaler, pooling, loss or optimiser code): only random numbers
 * and graph topology.
 *
 * Random numbers: splitmix64 (Steele, Lea & Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014), used as a counter-based
 * generator: every (seed, graph, purpose) triple owns an independent stream,
 * so any subset of a data set can be regenerated without the rest.
 * Normal variates: Box-Muller (Box & Muller, 1958).
 *
 * Graph recipe (stands in for the molecular graphs of PCQM4Mv2 / AISD, which
 * are not available):
 *   - n nodes (atoms, hydrogens included);
 *   - a random spanning tree built by attaching node v to a uniformly chosen
 *     earlier node whose degree is below max_deg;
 *   - extra uniformly random non-edges between nodes of degree < max_deg until
 *     the undirected edge count reaches floor(edge_factor * n + 0.5), with a
 *     bounded number of attempts;
 *   - each undirected bond stored as two directed edges (u->v, v->u), in
 *     generation order (not sorted: sorting is the collator's job);
 *   - atom types i.i.d. over {H,C,N,O,F,S,Cl} with probabilities
 *     {.45,.33,.08,.08,.02,.02,.02}.
 */
#include <stdint.h>
#include <string.h>
#include <math.h>

#define SYNTH_MAX_NODES 255

/* ---- splitmix64 ------------------------------------------------------- */

static uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

static uint64_t next64(uint64_t *s) {
  *s += 0x9E3779B97F4A7C15ULL;
  return mix64(*s);
}

/* Independent stream for (seed, index, purpose). */
static uint64_t stream_state(uint64_t seed, uint64_t index, uint64_t purpose) {
  uint64_t s = mix64(seed ^ 0x6A09E667F3BCC909ULL);
  s = mix64(s ^ (index * 0xD1B54A32D192ED03ULL + 0x3C6EF372FE94F82BULL));
  s = mix64(s ^ (purpose * 0x8CB92BA72F3D8DD7ULL + 0xA54FF53A5F1D36F1ULL));
  return s;
}

/* Uniform double in [0, 1) with 53 random bits. */
static double u01(uint64_t *s) { return (double)(next64(s) >> 11) * 0x1.0p-53; }

/* Uniform integer in [0, n), n >= 1, unbiased (rejection on the top bits). */
static uint32_t below(uint64_t *s, uint32_t n) {
  uint64_t lim = UINT64_MAX - (UINT64_MAX % n);
  uint64_t x;
  do { x = next64(s); } while (x >= lim);
  return (uint32_t)(x % n);
}

/* Standard normal by Box-Muller (cosine branch only). */
static double normal(uint64_t *s) {
  double u1 = 1.0 - u01(s); /* (0, 1] */
  double u2 = u01(s);
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586476925286766559 * u2);
}

/* Exported so both sides can check they agree on the stream definition. */
uint64_t synth_stream_first(uint64_t seed, uint64_t index, uint64_t purpose) {
  uint64_t s = stream_state(seed, index, purpose);
  return next64(&s);
}

/* ---- node counts ------------------------------------------------------ */

enum { SYNTH_N_UNIFORM = 0, SYNTH_N_LOGNORMAL = 1 };

/*
 * Node count of graphs [g0, g0+G) of a data set with the given seed.
 *   kind 0: uniform integer in [lo, hi]
 *   kind 1: round(exp(mu + sigma*z)), z ~ N(0,1), redrawn until in [lo, hi]
 */
int synth_node_counts(uint64_t seed, int64_t g0, int64_t G, int kind, int lo, int hi,
                      double mu, double sigma, int32_t *n_out) {
  if (lo < 1 || hi < lo || hi > SYNTH_MAX_NODES) return -1;
  for (int64_t g = 0; g < G; ++g) {
    uint64_t s = stream_state(seed, (uint64_t)(g0 + g), 0);
    int n;
    if (kind == SYNTH_N_UNIFORM) {
      n = lo + (int)below(&s, (uint32_t)(hi - lo + 1));
    } else if (kind == SYNTH_N_LOGNORMAL) {
      for (;;) {
        double v = exp(mu + sigma * normal(&s));
        double r = floor(v + 0.5);
        if (r >= lo && r <= hi) { n = (int)r; break; }
      }
    } else {
      return -2;
    }
    n_out[g] = n;
  }
  return 0;
}

/* Upper bound on the directed edge count of an n-node graph. */
int64_t synth_max_directed_edges(int n, double edge_factor) {
  int64_t m = (int64_t)floor(edge_factor * n + 0.5);
  int64_t full = (int64_t)n * (n - 1) / 2;
  if (m > full) m = full;
  if (m < n - 1) m = n - 1;
  return 2 * m;
}

/* ---- topology and atom types ----------------------------------------- */

static const double k_type_cdf[7] = {0.45, 0.78, 0.86, 0.94, 0.96, 0.98, 1.0};

/*
 * Topology and atom types of graphs [g0, g0+G) with node counts n[].
 * Writes node_ptr[G+1], edge_ptr[G+1] (offsets into types / edges, starting
 * at 0), types[sum n] and edges[2 * sum e] as (src, dst) local byte pairs.
 * edges_cap bounds the directed edges written.  Returns the total number of
 * directed edges, or a negative value on error.
 */
int64_t synth_topology(uint64_t seed, int64_t g0, int64_t G, const int32_t *n,
                       int max_deg, double edge_factor, int64_t *node_ptr,
                       int64_t *edge_ptr, uint8_t *types, uint8_t *edges,
                       int64_t edges_cap) {
  static uint8_t adj[SYNTH_MAX_NODES][SYNTH_MAX_NODES];
  int deg[SYNTH_MAX_NODES];
  int cand[SYNTH_MAX_NODES];
  int64_t nn = 0, ne = 0;
  node_ptr[0] = 0;
  edge_ptr[0] = 0;
  for (int64_t g = 0; g < G; ++g) {
    int nv = n[g];
    if (nv < 1 || nv > SYNTH_MAX_NODES) return -1;
    uint64_t s = stream_state(seed, (uint64_t)(g0 + g), 1);
    for (int i = 0; i < nv; ++i) { deg[i] = 0; memset(adj[i], 0, (size_t)nv); }
    int64_t m_target = synth_max_directed_edges(nv, edge_factor) / 2;
    int64_t e0 = ne;
    int64_t m = 0;
    /* random spanning tree */
    for (int v = 1; v < nv; ++v) {
      int c = 0;
      for (int u = 0; u < v; ++u) if (deg[u] < max_deg) cand[c++] = u;
      if (c == 0) return -3;
      int u = cand[below(&s, (uint32_t)c)];
      if (ne + 2 > edges_cap) return -4;
      edges[2 * ne + 0] = (uint8_t)u; edges[2 * ne + 1] = (uint8_t)v; ++ne;
      edges[2 * ne + 0] = (uint8_t)v; edges[2 * ne + 1] = (uint8_t)u; ++ne;
      adj[u][v] = adj[v][u] = 1; ++deg[u]; ++deg[v]; ++m;
    }
    /* extra bonds up to the target mean degree */
    for (int64_t tries = 0; m < m_target && tries < 50 * (int64_t)nv; ++tries) {
      int u = (int)below(&s, (uint32_t)nv), v = (int)below(&s, (uint32_t)nv);
      if (u == v || adj[u][v] || deg[u] >= max_deg || deg[v] >= max_deg) continue;
      if (ne + 2 > edges_cap) return -4;
      edges[2 * ne + 0] = (uint8_t)u; edges[2 * ne + 1] = (uint8_t)v; ++ne;
      edges[2 * ne + 0] = (uint8_t)v; edges[2 * ne + 1] = (uint8_t)u; ++ne;
      adj[u][v] = adj[v][u] = 1; ++deg[u]; ++deg[v]; ++m;
    }
    (void)e0;
    /* atom types */
    for (int i = 0; i < nv; ++i) {
      double r = u01(&s);
      int t = 0;
      while (t < 6 && r >= k_type_cdf[t]) ++t;
      types[nn + i] = (uint8_t)t;
    }
    nn += nv;
    node_ptr[g + 1] = nn;
    edge_ptr[g + 1] = ne;
  }
  return ne;
}

/* ---- scalar draws ----------------------------------------------------- */

/* out[g] = lo + (hi - lo) * U[0,1) for graphs [g0, g0+G) (purpose 3). */
void synth_uniform_targets(uint64_t seed, int64_t g0, int64_t G, double lo, double hi,
                           float *out) {
  for (int64_t g = 0; g < G; ++g) {
    uint64_t s = stream_state(seed, (uint64_t)(g0 + g), 3);
    out[g] = (float)(lo + (hi - lo) * u01(&s));
  }
}

/* out[i] = sigma * N(0,1) for items [i0, i0+n) (purpose 4). */
void synth_normal(uint64_t seed, int64_t i0, int64_t n, double sigma, double *out) {
  for (int64_t i = 0; i < n; ++i) {
    uint64_t s = stream_state(seed, (uint64_t)(i0 + i), 4);
    out[i] = sigma * normal(&s);
  }
}

/* out[i] = lo + (hi - lo) * U[0,1) for items [i0, i0+n) (purpose 5). */
void synth_uniform(uint64_t seed, int64_t i0, int64_t n, double lo, double hi, double *out) {
  for (int64_t i = 0; i < n; ++i) {
    uint64_t s = stream_state(seed, (uint64_t)(i0 + i), 5);
    out[i] = lo + (hi - lo) * u01(&s);
  }
}

/* ---- initial parameters ---------------------------------------------- */

/*
 * Initial flat parameter vector (float32) in the library's documented layout:
 *   emb[T][H]
 *   for each conv layer: msg_w[H][2H], msg_b[H], upd_w[16H][H], upd_b[H]
 *   head: w1[H][Hh], b1[Hh], w2[Hh], b2[1]
 * Weights and biases of a linear layer with fan-in f are U(-1/sqrt f, 1/sqrt f)
 * (msg: f = 2H; upd: f = 16H; w1/b1: f = H; w2/b2: f = Hh); the embedding is
 * N(0, 1).  Element k of the vector uses stream (seed, k, purpose 6).
 */
int64_t synth_param_count(int H, int L, int T, int Hh) {
  int64_t per_layer = (int64_t)H * 2 * H + H + (int64_t)16 * H * H + H;
  return (int64_t)T * H + L * per_layer + (int64_t)H * Hh + Hh + Hh + 1;
}

void synth_init_params(uint64_t seed, int H, int L, int T, int Hh, float *out) {
  int64_t k = 0;
  for (int64_t i = 0; i < (int64_t)T * H; ++i, ++k) {
    uint64_t s = stream_state(seed, (uint64_t)k, 6);
    out[k] = (float)normal(&s);
  }
  struct { int64_t count; double fan_in; } seg[4 + 4];
  int ns;
  for (int l = 0; l <= L; ++l) {
    if (l < L) {
      seg[0].count = (int64_t)H * 2 * H; seg[0].fan_in = 2.0 * H;
      seg[1].count = H;                  seg[1].fan_in = 2.0 * H;
      seg[2].count = (int64_t)16 * H * H; seg[2].fan_in = 16.0 * H;
      seg[3].count = H;                  seg[3].fan_in = 16.0 * H;
      ns = 4;
    } else {
      seg[0].count = (int64_t)H * Hh; seg[0].fan_in = H;
      seg[1].count = Hh;              seg[1].fan_in = H;
      seg[2].count = Hh;              seg[2].fan_in = Hh;
      seg[3].count = 1;               seg[3].fan_in = Hh;
      ns = 4;
    }
    for (int q = 0; q < ns; ++q) {
      double b = 1.0 / sqrt(seg[q].fan_in);
      for (int64_t i = 0; i < seg[q].count; ++i, ++k) {
        uint64_t s = stream_state(seed, (uint64_t)k, 6);
        out[k] = (float)(-b + 2.0 * b * u01(&s));
      }
    }
  }
}
