// Gather + multi-aggregator message passing of the PNA layer (Sec. 3.1, the
// graph-convolution step), and its backward.
//
// By linearity of the one-layer message function, m_ij = W_M [x_i ; x_j] + b_M
// equals P_i + Q_j with P = x A + b_M and Q = x B (A, B the two halves of
// W_M), so the per-edge message never has to be stored: the forward kernel
// gathers Q rows over each destination's CSR row and reduces them on the fly.
//
// Forward:  one thread per (node, 4 channels); FP32; the row's messages stay
//           in registers (first 4 edges) for the two-pass variance; all of a
//           row's loads are issued before its arithmetic, so a thread has its
//           P row and up to four Q rows in flight at once.
// Backward: kernel 1, one thread per (node i, 4 channels), recomputes m_ij,
//           routes dagg to every edge (sum: 1, mean: 1/d, min/max: shared
//           equally among exact ties, std: (m - mean) / (d std)), writes
//           dP_i and stores each dm_ij at the slot of the reverse edge;
//           kernel 2, one thread per (node j, 4 channels), sums its own row of
//           that buffer into dQ_j.  No atomics: the result is deterministic.
#include <algorithm>
#include <cfloat>
#include <mutex>

#include "kernels.cuh"

namespace gcnn {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void flag(unsigned *err, unsigned bits) {
  if (err) atomicOr(err, bits);
}
__device__ __forceinline__ void st4(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }
__device__ __forceinline__ float4 add4(float4 a, float4 b) {
  return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}

// Messages of a row are kept in registers for its first kCache edges (the
// degree of a molecule's atom is at most 4 in practice), so each Q row is
// gathered once per pass structure; longer rows re-read the tail.
constexpr int kCache = 4;

// source of edge e, or -1 (and the error flag) when it is out of range
__device__ __forceinline__ int source(const int *__restrict__ col, int e, int N, unsigned *err) {
  const int j = col[e];
  if (j < 0 || j >= N) {
    flag(err, kErrIndex);
    return -1;
  }
  return j;
}

// The bond term of the message (Sec. 3.1 bond properties; Table 1 edge
// attributes): R_e = sum_f e_e[f] W_E[f] for edge slot e, with the edge
// features in slot order (attr, E rows of round_up(F, 4) floats) and the
// layer's bond rows of W_M (w, F x H).  F = 0 (EDGE = false) drops the term.
struct Bonds {
  const float *attr, *w;
  int F;
};

// rows of attr are round_up(F, 4) floats apart
__device__ __forceinline__ float4 bond_term(const Bonds &b, int H, int e, int c) {
  float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
  const size_t row = (size_t)e * ((b.F + 3) & ~3);
  for (int f = 0; f < b.F; ++f) {
    const float a = b.attr[row + f];
    const float4 w = ld4(b.w + (size_t)f * H + c);
    r.x = fmaf(a, w.x, r.x); r.y = fmaf(a, w.y, r.y); r.z = fmaf(a, w.z, r.z); r.w = fmaf(a, w.w, r.w);
  }
  return r;
}

// m_ij = (P_i + Q_j) + R_e for the 4 channels at c, edge slot e (Q taken as 0
// for an invalid source)
template <bool EDGE>
__device__ __forceinline__ float4 message(const float *__restrict__ PQ, int j, int H, int c, float4 P, const Bonds &b,
                                          int e) {
  const float4 m = j >= 0 ? add4(P, ld4(PQ + (size_t)j * 2 * H + H + c)) : P;
  return EDGE ? add4(m, bond_term(b, H, e, c)) : m;
}

// Messages of the first kCache edges (slots r0 + k, clamped into the row) of
// node i's row from their sources j[]: every Q row is loaded unconditionally
// (row i stands in for a source out of range, whose message is then P alone,
// plus its bond term), so the loads are all in flight at once; returns
// whether a source was out of range.
template <bool EDGE>
__device__ __forceinline__ bool gather_first(const float *__restrict__ PQ, const int (&j)[kCache], int i, int N, int H,
                                             int c, float4 P, float4 (&mc)[kCache], const Bonds &b, int r0, int r1) {
  bool bad = false;
#pragma unroll
  for (int k = 0; k < kCache; ++k) {
    const bool ok = j[k] >= 0 && j[k] < N;
    bad |= !ok;
    const float4 q = ld4(PQ + (size_t)(ok ? j[k] : i) * 2 * H + H + c);
    mc[k] = ok ? add4(P, q) : P;
  }
  if (EDGE) {  // bond_term for the kCache edges, each W_E row loaded once
    const int ld = (b.F + 3) & ~3;
    float4 r[kCache];
#pragma unroll
    for (int k = 0; k < kCache; ++k) r[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int f = 0; f < b.F; ++f) {
      const float4 w = ld4(b.w + (size_t)f * H + c);
#pragma unroll
      for (int k = 0; k < kCache; ++k) {
        const float a = b.attr[(size_t)min(r0 + k, r1 - 1) * ld + f];
        r[k].x = fmaf(a, w.x, r[k].x); r[k].y = fmaf(a, w.y, r[k].y);
        r[k].z = fmaf(a, w.z, r[k].z); r[k].w = fmaf(a, w.w, r[k].w);
      }
    }
#pragma unroll
    for (int k = 0; k < kCache; ++k) mc[k] = add4(mc[k], r[k]);
  }
  return bad;
}

__device__ __forceinline__ void acc_sq(float4 &v, float4 m, float4 mean) {
  const float tx = m.x - mean.x, ty = m.y - mean.y, tz = m.z - mean.z, tw = m.w - mean.w;
  v.x += tx * tx; v.y += ty * ty; v.z += tz * tz; v.w += tw * tw;
}

// F32 / B16: whether the FP32 aggregates / the BF16 scaled operand are
// written (one instantiation per output set keeps the other's code out)
template <bool F32, bool B16, bool EDGE>
__global__ void __launch_bounds__(kThreads, 4)
aggregate_fwd_kernel(int n_cap, int H, DevDims dims, const int *__restrict__ row_ptr,
                     const int *__restrict__ col, const float *__restrict__ PQ,
                     float *__restrict__ agg, float eps, unsigned *err, uint16_t *__restrict__ S16, int ld16,
                     const float *__restrict__ amp, const float *__restrict__ att, Bonds bonds, int early) {
  const int H4 = H >> 2;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  // the batch's sizes, the row's CSR range and its first sources (and the
  // degree scalers) come from the collator; with `early` they are read
  // before the dependency wait, overlapping the previous kernel's tail
  int N = 0, i = 0, c = 0, r0 = 0, r1 = 0;
  int j[kCache];
  float s_amp = 0.f, s_att = 0.f;
  auto load_row = [&]() {
    N = min(n_cap, dims.nodes(n_cap));
    if (t >= (long long)N * H4) return;
    i = (int)(t / H4);
    c = (int)(t % H4) * 4;
    r0 = row_ptr[i];
    r1 = row_ptr[i + 1];
    if (r1 > r0 && r0 >= 0)
#pragma unroll
      for (int k = 0; k < kCache; ++k) j[k] = col[min(r0 + k, r1 - 1)];
    if (B16) {
      s_amp = amp[i];
      s_att = att[i];
    }
  };
  if (early) load_row();
  pdl_entry(GCNN_K_AGG_FWD);
  if (!early) load_row();
  if (t >= (long long)N * H4) return;
  const int d = r1 - r0;
  float *out = F32 ? agg + (size_t)i * kAgg * H + c : nullptr;
  const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
  if (d <= 0 || r0 < 0) {
    if (d < 0 || r0 < 0) flag(err, kErrIndex);
    if (F32)
#pragma unroll
      for (int a = 0; a < kAgg; ++a) st4(out + a * H, z);
    if (B16)
      for (int a = 0; a < kScalers * kAgg; ++a) st_bf16x4(S16 + (size_t)i * ld16 + a * H + c, 0.f, 0.f, 0.f, 0.f);
    return;
  }
  // every load of the row is issued before the arithmetic: the first kCache
  // sources (indices clamped into the row, so short rows repeat their last
  // edge and use only the first d; read above), then P and the gathered Q rows
  const float4 P = ld4(PQ + (size_t)i * 2 * H + c);
  float4 mc[kCache];
  if (gather_first<EDGE>(PQ, j, i, N, H, c, P, mc, bonds, r0, r1)) flag(err, kErrIndex);
  float4 s = z;
  float4 mn = make_float4(FLT_MAX, FLT_MAX, FLT_MAX, FLT_MAX);
  float4 mx = make_float4(-FLT_MAX, -FLT_MAX, -FLT_MAX, -FLT_MAX);
  auto take = [&](float4 m) {
    s = add4(s, m);
    mn.x = fminf(mn.x, m.x); mn.y = fminf(mn.y, m.y); mn.z = fminf(mn.z, m.z); mn.w = fminf(mn.w, m.w);
    mx.x = fmaxf(mx.x, m.x); mx.y = fmaxf(mx.y, m.y); mx.z = fmaxf(mx.z, m.z); mx.w = fmaxf(mx.w, m.w);
  };
#pragma unroll
  for (int k = 0; k < kCache; ++k)
    if (k < d) take(mc[k]);
  for (int e = r0 + kCache; e < r1; ++e) take(message<EDGE>(PQ, source(col, e, N, err), H, c, P, bonds, e));
  const float df = (float)d;
  const float4 mean = make_float4(s.x / df, s.y / df, s.z / df, s.w / df);
  float4 v = z;  // two-pass variance
#pragma unroll
  for (int k = 0; k < kCache; ++k)
    if (k < d) acc_sq(v, mc[k], mean);
  for (int e = r0 + kCache; e < r1; ++e)
    acc_sq(v, message<EDGE>(PQ, source(col, e, N, err), H, c, P, bonds, e), mean);
  float4 sd;
  sd.x = sqrtf(fmaxf(v.x / df, 0.f) + eps);
  sd.y = sqrtf(fmaxf(v.y / df, 0.f) + eps);
  sd.z = sqrtf(fmaxf(v.z / df, 0.f) + eps);
  sd.w = sqrtf(fmaxf(v.w / df, 0.f) + eps);
  if (F32) {
    st4(out + 0 * H, s);
    st4(out + 1 * H, mean);
    st4(out + 2 * H, mn);
    st4(out + 3 * H, mx);
    st4(out + 4 * H, sd);
  }
  if (B16) {  // scaler-major: identity, amplification, attenuation
    const float4 vv[kAgg] = {s, mean, mn, mx, sd};
    const float sc[kScalers] = {1.f, s_amp, s_att};
    uint16_t *o = S16 + (size_t)i * ld16 + c;
#pragma unroll
    for (int q = 0; q < kScalers; ++q)
#pragma unroll
      for (int a = 0; a < kAgg; ++a)
        st_bf16x4(o + (q * kAgg + a) * H, sc[q] * vv[a].x, sc[q] * vv[a].y, sc[q] * vv[a].z, sc[q] * vv[a].w);
  }
}

// dL/dm for one channel of one edge from its node's routing coefficients
__device__ __forceinline__ float route(float m, float base, float mn, float cmin, float mx, float cmax, float mean,
                                       float cstd) {
  float g = base;
  if (m == mn) g += cmin;
  if (m == mx) g += cmax;
  return g + cstd * (m - mean);
}

constexpr int kEdgeThreads = 128;  // five blocks of 128 per SM at this kernel's register count

// CSR range of node i's row and the sources and reverse slots of its first
// kCache edges (clamped into the row); the slots are read only for a valid range.
struct RowIdx {
  int r0, r1;
  int j[kCache], re[kCache];
};

__device__ __forceinline__ RowIdx load_row_idx(int i, int E, const int *__restrict__ row_ptr,
                                               const int *__restrict__ col, const int *__restrict__ rev) {
  RowIdx x;
  x.r0 = row_ptr[i];
  x.r1 = row_ptr[i + 1];
  if (x.r1 > x.r0 && x.r0 >= 0 && x.r1 <= E)
#pragma unroll
    for (int k = 0; k < kCache; ++k) {
      x.j[k] = col[min(x.r0 + k, x.r1 - 1)];
      x.re[k] = rev[min(x.r0 + k, x.r1 - 1)];
    }
  return x;
}

// Backward of one (node i, 4 channels at c): recomputes the row's messages,
// takes the forward's statistics (stored in agg, or recomputed in the
// forward's order when agg is null), routes dagg to every edge of the row
// and hands each edge's gradient to to_slot(reverse slot, g); returns dP_i.
// STATS: 1 = statistics stored in agg, 0 = recomputed, -1 = decided at run
// time by agg != null (one code path for both, fewer registers)
template <int STATS, bool EDGE, class ToSlot>
__device__ __forceinline__ float4 node_backward(int i, int c, int H, int N, int E, const RowIdx &ix,
                                                const int *__restrict__ col, const int *__restrict__ rev,
                                                const float *__restrict__ PQ, const float *__restrict__ agg,
                                                const float *__restrict__ dagg, float eps, unsigned *err,
                                                const Bonds &bonds, ToSlot to_slot) {
  const bool STORED = STATS < 0 ? agg != nullptr : STATS == 1;
  const int r0 = ix.r0, r1 = ix.r1;
  const int d = r1 - r0;
  float4 dP = make_float4(0.f, 0.f, 0.f, 0.f);
  if (d <= 0 || r0 < 0 || r1 > E) {
    if (d < 0 || r0 < 0 || r1 > E) flag(err, kErrIndex);
    return dP;
  }
  const float df = (float)d;
  // all loads of the row first (as in the forward): sources and reverse slots
  // of the first kCache edges (clamped into the row; in ix), P, the stored
  // statistics, the incoming gradient and the gathered Q rows
  const int(&j)[kCache] = ix.j;
  const int(&re)[kCache] = ix.re;
  const float4 P = ld4(PQ + (size_t)i * 2 * H + c);
  float4 mean, mn, mx, sd;
  if (STORED) {
    const float *a = agg + (size_t)i * kAgg * H + c;
    mean = ld4(a + 1 * H); mn = ld4(a + 2 * H); mx = ld4(a + 3 * H); sd = ld4(a + 4 * H);
  }
  const float *da = dagg + (size_t)i * kAgg * H + c;
  const float4 dsum = ld4(da + 0 * H), dmean = ld4(da + 1 * H), dmin = ld4(da + 2 * H);
  const float4 dmax = ld4(da + 3 * H), dstd = ld4(da + 4 * H);
  float4 mc[kCache];
  if (gather_first<EDGE>(PQ, j, i, N, H, c, P, mc, bonds, r0, r1)) flag(err, kErrIndex);
  // the forward's statistics: stored, or recomputed in the forward's order
  if (!STORED) {
    float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
    mn = make_float4(FLT_MAX, FLT_MAX, FLT_MAX, FLT_MAX);
    mx = make_float4(-FLT_MAX, -FLT_MAX, -FLT_MAX, -FLT_MAX);
    auto take = [&](float4 m) {
      s = add4(s, m);
      mn.x = fminf(mn.x, m.x); mn.y = fminf(mn.y, m.y); mn.z = fminf(mn.z, m.z); mn.w = fminf(mn.w, m.w);
      mx.x = fmaxf(mx.x, m.x); mx.y = fmaxf(mx.y, m.y); mx.z = fmaxf(mx.z, m.z); mx.w = fmaxf(mx.w, m.w);
    };
#pragma unroll
    for (int k = 0; k < kCache; ++k)
      if (k < d) take(mc[k]);
    for (int e = r0 + kCache; e < r1; ++e) take(message<EDGE>(PQ, source(col, e, N, err), H, c, P, bonds, e));
    mean = make_float4(s.x / df, s.y / df, s.z / df, s.w / df);
  }
  float4 nmin = make_float4(0.f, 0.f, 0.f, 0.f), nmax = nmin, var = nmin;
  auto count = [&](float4 m) {
    nmin.x += (m.x == mn.x); nmin.y += (m.y == mn.y); nmin.z += (m.z == mn.z); nmin.w += (m.w == mn.w);
    nmax.x += (m.x == mx.x); nmax.y += (m.y == mx.y); nmax.z += (m.z == mx.z); nmax.w += (m.w == mx.w);
    acc_sq(var, m, mean);
  };
#pragma unroll
  for (int k = 0; k < kCache; ++k)
    if (k < d) count(mc[k]);
  for (int e = r0 + kCache; e < r1; ++e) count(message<EDGE>(PQ, source(col, e, N, err), H, c, P, bonds, e));
  var.x /= df; var.y /= df; var.z /= df; var.w /= df;
  if (!STORED) {
    sd.x = sqrtf(fmaxf(var.x, 0.f) + eps);
    sd.y = sqrtf(fmaxf(var.y, 0.f) + eps);
    sd.z = sqrtf(fmaxf(var.z, 0.f) + eps);
    sd.w = sqrtf(fmaxf(var.w, 0.f) + eps);
  }
  // per-node routing coefficients: every edge gets base = dsum + dmean / d,
  // plus dmin / (number of minima) at a minimum, dmax / (number of maxima) at
  // a maximum and dstd (m - mean) / (d std) where the variance is positive
  const float4 base = make_float4(dsum.x + dmean.x / df, dsum.y + dmean.y / df, dsum.z + dmean.z / df,
                                  dsum.w + dmean.w / df);
  const float4 cmin = make_float4(dmin.x / nmin.x, dmin.y / nmin.y, dmin.z / nmin.z, dmin.w / nmin.w);
  const float4 cmax = make_float4(dmax.x / nmax.x, dmax.y / nmax.y, dmax.z / nmax.z, dmax.w / nmax.w);
  const float4 cstd = make_float4(var.x > 0.f ? dstd.x / (df * sd.x) : 0.f, var.y > 0.f ? dstd.y / (df * sd.y) : 0.f,
                                  var.z > 0.f ? dstd.z / (df * sd.z) : 0.f, var.w > 0.f ? dstd.w / (df * sd.w) : 0.f);
  auto emit = [&](int r, float4 m) {  // r: the reverse slot of the edge
    float4 g;
    g.x = route(m.x, base.x, mn.x, cmin.x, mx.x, cmax.x, mean.x, cstd.x);
    g.y = route(m.y, base.y, mn.y, cmin.y, mx.y, cmax.y, mean.y, cstd.y);
    g.z = route(m.z, base.z, mn.z, cmin.z, mx.z, cmax.z, mean.z, cstd.z);
    g.w = route(m.w, base.w, mn.w, cmin.w, mx.w, cmax.w, mean.w, cstd.w);
    dP = add4(dP, g);
    to_slot(r, g);
  };
#pragma unroll
  for (int k = 0; k < kCache; ++k)
    if (k < d) emit(re[k], mc[k]);
  for (int e = r0 + kCache; e < r1; ++e)
    emit(rev[e], message<EDGE>(PQ, source(col, e, N, err), H, c, P, bonds, e));
  return dP;
}

template <bool EDGE>
__global__ void __launch_bounds__(kEdgeThreads)
aggregate_bwd_edge_kernel(int n_cap, int e_cap, int H, DevDims dims, const int *__restrict__ row_ptr,
                          const int *__restrict__ col, const int *__restrict__ rev,
                          const float *__restrict__ PQ, const float *__restrict__ agg,
                          const float *__restrict__ dagg, float *__restrict__ dPQ,
                          float *__restrict__ dm, unsigned *err, uint16_t *__restrict__ dPQ16, int ld16, float eps,
                          Bonds bonds, int early) {
  const int H4 = H >> 2;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  // sizes and the row's indices (collator) before the dependency wait with `early`
  int N = 0, E = 0;
  RowIdx ix{};
  auto load = [&]() {
    N = min(n_cap, dims.nodes(n_cap));
    E = min(e_cap, dims.edges(e_cap));
    if (t < (long long)N * H4) ix = load_row_idx((int)(t / H4), E, row_ptr, col, rev);
  };
  if (early) load();
  pdl_entry(GCNN_K_AGG_BWD_EDGE);
  if (!early) load();
  if (t >= (long long)N * H4) return;
  const int i = (int)(t / H4), c = (int)(t % H4) * 4;
  const float4 dP = node_backward<-1, EDGE>(i, c, H, N, E, ix, col, rev, PQ, agg, dagg, eps, err, bonds,
                                             [&](int r, float4 g) {
    if (r >= 0 && r < E) st4(dm + (size_t)r * H + c, g);
    else flag(err, kErrIndex);
  });
  st4(dPQ + (size_t)i * 2 * H + c, dP);
  if (dPQ16) st_bf16x4(dPQ16 + (size_t)i * ld16 + c, dP.x, dP.y, dP.z, dP.w);
}

// Fused backward over whole graphs: block (x, y) takes the graphs of chunk x
// (a node range closed under the edges, since edges stay inside a graph) and
// the channel slice of cs4 float4 columns starting at y cs4.  Pass 1 is
// node_backward for every (node, channel) of the range with each edge's
// gradient kept at its reverse slot in shared memory (in the global scratch
// dm when the range has more than emax edges); after a block barrier pass 2
// sums each node's own row of slots into dQ.  Same arithmetic and order as
// the edge + gather pair, without the per-edge round trip through memory.
constexpr int kFusedThreads = 512;
constexpr int kChunkEdges = 128;  // edges per chunk on average (one window)
constexpr int kChunkSlots = 192;  // edges a chunk keeps in shared memory (more costs L1)
constexpr int kFusedSmem = 160 * 1024;  // shared-memory budget of one block

// Work partition of the fused backward: chunk k holds the graphs whose first
// edge lies in [k T, (k + 1) T); chunk_first[k] is its first graph (G when it
// is empty), for k = 0..n_chunks.  Thread g (g = 0..G) is the first graph of
// every window that starts after graph g - 1's first edge and no later than
// its own, so each entry is written by exactly one thread.
__global__ void __launch_bounds__(kThreads)
aggregate_chunk_kernel(int g_cap, int n_cap, int n_chunks, int T, DevDims dims, const int *__restrict__ node_off,
                       const int *__restrict__ row_ptr, int *__restrict__ chunk_first, unsigned *err) {
  pdl_entry(GCNN_K_AGG_BWD_CHUNKS);
  const int G = min(g_cap, dims.graphs(g_cap));
  const int N = min(n_cap, dims.nodes(n_cap));
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g > G) return;
  auto first_edge = [&](int h) {
    const int n = node_off[h];
    if (n < 0 || n > N) {
      flag(err, kErrIndex);
      return 0;
    }
    return row_ptr[n];
  };
  // the sentinel entry n_chunks is always G (a trailing graph without edges
  // then belongs to the last chunk)
  const int k0 = min(g == 0 ? 0 : first_edge(g - 1) / T + 1, n_chunks);
  const int k1 = g == G ? n_chunks : min(n_chunks - 1, first_edge(g) / T);
  for (int k = k0; k <= k1; ++k) chunk_first[k] = g;
}

template <bool STORED>
__global__ void __launch_bounds__(kFusedThreads, 1)
aggregate_bwd_fused_kernel(int g_cap, int n_cap, int e_cap, const int *__restrict__ chunk_first, int cs4, int emax,
                           int H, DevDims dims, const int *__restrict__ node_off, const int *__restrict__ row_ptr,
                           const int *__restrict__ col, const int *__restrict__ rev, const float *__restrict__ PQ,
                           const float *__restrict__ agg, const float *__restrict__ dagg, float *__restrict__ dPQ,
                           float *__restrict__ dm, unsigned *err, uint16_t *__restrict__ dPQ16, int ld16, float eps) {
  extern __shared__ float4 s_dm[];
  pdl_entry(GCNN_K_AGG_BWD_FUSED);
  const int G = min(g_cap, dims.graphs(g_cap));
  const int N = min(n_cap, dims.nodes(n_cap));
  const int E = min(e_cap, dims.edges(e_cap));
  const int g0 = chunk_first[blockIdx.x], g1 = min(chunk_first[blockIdx.x + 1], G);
  if (g0 < 0 || g0 >= g1) return;
  const int n0 = node_off[g0], n1 = node_off[g1];
  if (n0 < 0 || n1 < n0 || n1 > N) {
    flag(err, kErrIndex);
    return;
  }
  const int e0 = row_ptr[n0], e1 = row_ptr[n1];
  if (e0 < 0 || e1 < e0 || e1 > E) {
    flag(err, kErrIndex);
    return;
  }
  const bool in_smem = e1 - e0 <= emax;
  const int H4 = H >> 2;
  const int c0 = blockIdx.y * cs4;
  const int w = min(cs4, H4 - c0);
  // each thread keeps one float4 column of the slice and strides over the
  // chunk's nodes (kFusedThreads / w rows at a time; the remainder threads idle)
  const int rows = kFusedThreads / w, row = threadIdx.x / w, cc = threadIdx.x % w, c = (c0 + cc) * 4;
  const int n_end = row < rows ? n1 : n0;
  for (int i = n0 + row; i < n_end; i += rows) {
    const float4 dP = node_backward<STORED ? 1 : 0, false>(i, c, H, N, E, load_row_idx(i, E, row_ptr, col, rev), col,
                                                           rev, PQ, agg, dagg, eps, err,
                                                           Bonds{nullptr, nullptr, 0}, [&](int r, float4 g) {
      if (r < e0 || r >= e1) flag(err, kErrIndex);  // an edge leaving the graph
      else if (in_smem) s_dm[(r - e0) * cs4 + cc] = g;
      else st4(dm + (size_t)r * H + c, g);
    });
    st4(dPQ + (size_t)i * 2 * H + c, dP);
    if (dPQ16) st_bf16x4(dPQ16 + (size_t)i * ld16 + c, dP.x, dP.y, dP.z, dP.w);
  }
  __syncthreads();
  for (int j = n0 + row; j < n_end; j += rows) {
    int r0 = row_ptr[j], r1 = row_ptr[j + 1];
    if (r0 < e0 || r1 > e1 || r1 < r0) {
      flag(err, kErrIndex);
      r1 = r0;
    }
    float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
    if (in_smem)
      for (int e = r0; e < r1; ++e) q = add4(q, s_dm[(e - e0) * cs4 + cc]);
    else
      for (int e = r0; e < r1; ++e) q = add4(q, ld4(dm + (size_t)e * H + c));
    st4(dPQ + (size_t)j * 2 * H + H + c, q);
    if (dPQ16) st_bf16x4(dPQ16 + (size_t)j * ld16 + H + c, q.x, q.y, q.z, q.w);
  }
}

__global__ void __launch_bounds__(kThreads)
aggregate_bwd_gather_kernel(int n_cap, int e_cap, int H, DevDims dims,
                            const int *__restrict__ row_ptr, const float *__restrict__ dm,
                            float *__restrict__ dPQ, unsigned *err, uint16_t *__restrict__ dPQ16, int ld16,
                            int early) {
  const int H4 = H >> 2;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  // sizes and the row's range (collator) before the dependency wait with `early`
  int N = 0, E = 0, r0 = 0, r1 = 0;
  auto load = [&]() {
    N = min(n_cap, dims.nodes(n_cap));
    E = min(e_cap, dims.edges(e_cap));
    if (t < (long long)N * H4) {
      r0 = row_ptr[t / H4];
      r1 = row_ptr[t / H4 + 1];
    }
  };
  if (early) load();
  pdl_entry(GCNN_K_AGG_BWD_GATHER);
  if (!early) load();
  if (t >= (long long)N * H4) return;
  const int j = (int)(t / H4), c = (int)(t % H4) * 4;
  if (r1 < r0 || r0 < 0 || r1 > E) { flag(err, kErrIndex); r1 = r0; }
  float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 4
  for (int e = r0; e < r1; ++e) q = add4(q, ld4(dm + (size_t)e * H + c));
  st4(dPQ + (size_t)j * 2 * H + H + c, q);
  if (dPQ16) st_bf16x4(dPQ16 + (size_t)j * ld16 + H + c, q.x, q.y, q.z, q.w);
}

// Bond rows' gradient dW_E[f][c] = sum over the batch's edge slots r of
// eattr[r][f] dm[r][c] (dm at reverse slots; both directions of a bond carry
// the same features, so slot r pairs with its own features).  Block x sums
// the float4 column 4x over all slots (threads strided over slots, then the
// warps' partials in order): a fixed order, deterministic.
constexpr int kBondThreads = 256, kMaxBondF = 16;

__global__ void __launch_bounds__(kBondThreads)
bond_grad_kernel(int e_cap, int H, int F, int ld, DevDims dims, const float *__restrict__ eattr,
                 const float *__restrict__ dm, float *__restrict__ out) {
  pdl_entry(GCNN_K_BOND_GRAD);
  __shared__ float4 part[kBondThreads / 32][kMaxBondF];
  const int E = min(e_cap, dims.edges(e_cap));
  const int c = blockIdx.x * 4, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float4 acc[kMaxBondF];
#pragma unroll
  for (int f = 0; f < kMaxBondF; ++f) acc[f] = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int r = threadIdx.x; r < E; r += kBondThreads) {
    const float4 g = ld4(dm + (size_t)r * H + c);
#pragma unroll
    for (int f = 0; f < kMaxBondF; ++f)
      if (f < F) {
        const float a = eattr[(size_t)r * ld + f];
        acc[f].x = fmaf(a, g.x, acc[f].x); acc[f].y = fmaf(a, g.y, acc[f].y);
        acc[f].z = fmaf(a, g.z, acc[f].z); acc[f].w = fmaf(a, g.w, acc[f].w);
      }
  }
#pragma unroll
  for (int f = 0; f < kMaxBondF; ++f) {
    if (f < F) {
      float4 v = acc[f];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o); v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
        v.z += __shfl_xor_sync(0xffffffffu, v.z, o); v.w += __shfl_xor_sync(0xffffffffu, v.w, o);
      }
      if (lane == 0) part[w][f] = v;
    }
  }
  __syncthreads();
  if (threadIdx.x < F) {
    float4 t = part[0][threadIdx.x];
    for (int q = 1; q < kBondThreads / 32; ++q) t = add4(t, part[q][threadIdx.x]);
    st4(out + (size_t)threadIdx.x * H + c, t);
  }
}

}  // namespace

int launch_bond_grad(int n_edges, int H, int F, int ld, DevDims dims, const float *eattr, const float *dm, float *out,
                     cudaStream_t s) {
  if (F <= 0) return GCNN_OK;
  if (F > kMaxBondF || H % 4 || ld % 4 || ld < F) return set_error(GCNN_EINVAL, "bond_grad: bad sizes");
  GCNN_TRY(launch(bond_grad_kernel, H / 4, kBondThreads, 0, s, std::max(n_edges, 0), H, F, ld, dims, eattr, dm, out));
  return GCNN_OK;
}

int launch_aggregate_fwd(int n_nodes, int H, DevDims dims, const int *row_ptr, const int *col,
                         const float *PQ, float *agg, float eps, unsigned *err, cudaStream_t s,
                         uint16_t *S16, int ld16, const float *amp, const float *att, const float *eattr,
                         const float *wE, int F, bool idx_early) {
  if (H <= 0 || H % 4) return set_error(GCNN_EINVAL, "aggregate: hidden must be a positive multiple of 4");
  if (F < 0 || (F > 0 && (!eattr || !wE))) return set_error(GCNN_EINVAL, "aggregate: bond features without data");
  if (n_nodes <= 0) return GCNN_OK;
  const long long work = (long long)n_nodes * (H / 4);
  using K = void (*)(int, int, DevDims, const int *, const int *, const float *, float *, float, unsigned *,
                     uint16_t *, int, const float *, const float *, Bonds, int);
  static const K table[8] = {aggregate_fwd_kernel<false, false, false>, aggregate_fwd_kernel<false, true, false>,
                             aggregate_fwd_kernel<true, false, false>,  aggregate_fwd_kernel<true, true, false>,
                             aggregate_fwd_kernel<false, false, true>,  aggregate_fwd_kernel<false, true, true>,
                             aggregate_fwd_kernel<true, false, true>,   aggregate_fwd_kernel<true, true, true>};
  const K kernel = table[(F > 0 ? 4 : 0) + (agg ? 2 : 0) + (S16 ? 1 : 0)];
  GCNN_TRY(launch(kernel, ceil_div(work, kThreads), kThreads, 0, s, n_nodes, H, dims, row_ptr, col, PQ, agg, eps, err,
                  S16, ld16, amp, att, Bonds{eattr, wE, F}, idx_early ? 1 : 0));
  return GCNN_OK;
}

int launch_aggregate_bwd(int n_nodes, int n_edges, int H, DevDims dims, const int *row_ptr,
                         const int *col, const int *rev, const float *PQ, const float *agg,
                         const float *dagg, float *dPQ, float *scratch, float eps, unsigned *err,
                         cudaStream_t s, uint16_t *dPQ16, int ld16, const float *eattr, const float *wE, int F,
                         bool idx_early) {
  if (H <= 0 || H % 4) return set_error(GCNN_EINVAL, "aggregate: hidden must be a positive multiple of 4");
  if (F < 0 || (F > 0 && (!eattr || !wE))) return set_error(GCNN_EINVAL, "aggregate: bond features without data");
  if (n_nodes <= 0) return GCNN_OK;
  const long long work = (long long)n_nodes * (H / 4);
  GCNN_TRY(launch(F > 0 ? aggregate_bwd_edge_kernel<true> : aggregate_bwd_edge_kernel<false>, ceil_div(work, kEdgeThreads),
                  kEdgeThreads, 0, s, n_nodes, n_edges, H, dims, row_ptr, col, rev, PQ, agg, dagg, dPQ, scratch, err,
                  dPQ16, ld16, eps, Bonds{eattr, wE, F}, idx_early ? 1 : 0));
  GCNN_TRY(launch(aggregate_bwd_gather_kernel, ceil_div(work, kThreads), kThreads, 0, s, n_nodes, n_edges, H, dims,
                  row_ptr, (const float *)scratch, dPQ, err, dPQ16, ld16, idx_early ? 1 : 0));
  return GCNN_OK;
}

int aggregate_chunk_capacity(int n_edges) { return ceil_div(std::max(n_edges, 1), kChunkEdges) + 1; }

bool aggregate_bwd_uses_fused(int n_edges) {
  return ceil_div(std::max(n_edges, 0), kChunkEdges) >= 2 * num_sms();
}

int launch_aggregate_bwd_graphs(int n_graphs, int n_nodes, int n_edges, int H, DevDims dims, const int *node_off,
                                const int *row_ptr, const int *col, const int *rev, const float *PQ,
                                const float *agg, const float *dagg, float *dPQ, float *scratch, int *chunks,
                                float eps, unsigned *err, cudaStream_t s, uint16_t *dPQ16, int ld16,
                                const float *eattr, const float *wE, int F, bool make_chunks, bool idx_early) {
  if (H <= 0 || H % 4) return set_error(GCNN_EINVAL, "aggregate: hidden must be a positive multiple of 4");
  if (n_nodes <= 0 || n_graphs <= 0) return GCNN_OK;
  // with bond features the per-edge gradients are kept: their weight gradient reads them
  if (F > 0 || !aggregate_bwd_uses_fused(n_edges))
    return launch_aggregate_bwd(n_nodes, n_edges, H, dims, row_ptr, col, rev, PQ, agg, dagg, dPQ, scratch, eps, err, s,
                                dPQ16, ld16, eattr, wE, F, idx_early);
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [] {
    attr = cudaFuncSetAttribute(aggregate_bwd_fused_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kFusedSmem);
    if (attr == cudaSuccess)
      attr = cudaFuncSetAttribute(aggregate_bwd_fused_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  kFusedSmem);
  });
  if (attr != cudaSuccess) return set_error(GCNN_ECUDA, "aggregate: %s", cudaGetErrorString(attr));
  const int n_chunks = aggregate_chunk_capacity(n_edges) - 1;
  // channel slices so that a chunk's kChunkSlots edges fit the budget
  const int H4 = H / 4;
  const int slices = ceil_div(kChunkSlots * H4 * 16, kFusedSmem);
  const int cs4 = ceil_div(H4, slices);
  if (make_chunks)
    GCNN_TRY(launch(aggregate_chunk_kernel, ceil_div(n_graphs + 1, kThreads), kThreads, 0, s, n_graphs, n_nodes,
                    n_chunks, kChunkEdges, dims, node_off, row_ptr, chunks, err));
  GCNN_TRY(launch(agg ? aggregate_bwd_fused_kernel<true> : aggregate_bwd_fused_kernel<false>,
                  dim3(n_chunks, ceil_div(H4, cs4)), kFusedThreads,
                  (size_t)kChunkSlots * cs4 * 16, s, n_graphs, n_nodes, n_edges, (const int *)chunks, cs4,
                  kChunkSlots, H, dims, node_off, row_ptr, col, rev, PQ, agg, dagg, dPQ, scratch, err, dPQ16, ld16,
                  eps));
  return GCNN_OK;
}

GCNN_TIMELINE_ATTACH(aggregate)

}  // namespace gcnn
