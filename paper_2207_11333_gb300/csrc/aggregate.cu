// Gather + multi-aggregator message passing of the PNA layer (Sec. 3.1, the
// graph-convolution step), and its backward.
//
// By linearity of the one-layer message function, m_ij = W_M [x_i ; x_j] + b_M
// equals P_i + Q_j with P = x A + b_M and Q = x B (A, B the two halves of
// W_M), so the per-edge message never has to be stored: the forward kernel
// gathers Q rows over each destination's CSR row and reduces them on the fly.
//
// Forward:  one thread per (node, 4 channels); FP32; the row's messages stay
//           in registers (first 4 edges) for the two-pass variance.
// Backward: kernel 1, one thread per (node i, 4 channels), recomputes m_ij,
//           routes dagg to every edge (sum: 1, mean: 1/d, min/max: shared
//           equally among exact ties, std: (m - mean) / (d std)), writes
//           dP_i and stores each dm_ij at the slot of the reverse edge;
//           kernel 2, one thread per (node j, 4 channels), sums its own row of
//           that buffer into dQ_j.  No atomics: the result is deterministic.
#include <cfloat>

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

// m_ij = P_i + Q_j for the 4 channels at c (Q taken as 0 for an invalid source)
__device__ __forceinline__ float4 message(const float *__restrict__ PQ, int j, int H, int c, float4 P) {
  return j >= 0 ? add4(P, ld4(PQ + (size_t)j * 2 * H + H + c)) : P;
}

__device__ __forceinline__ void acc_sq(float4 &v, float4 m, float4 mean) {
  const float tx = m.x - mean.x, ty = m.y - mean.y, tz = m.z - mean.z, tw = m.w - mean.w;
  v.x += tx * tx; v.y += ty * ty; v.z += tz * tz; v.w += tw * tw;
}

__global__ void __launch_bounds__(kThreads, 4)
aggregate_fwd_kernel(int n_cap, int H, DevDims dims, const int *__restrict__ row_ptr,
                     const int *__restrict__ col, const float *__restrict__ PQ,
                     float *__restrict__ agg, float eps, unsigned *err, uint16_t *__restrict__ S16, int ld16,
                     const float *__restrict__ amp, const float *__restrict__ att) {
  pdl_entry(GCNN_K_AGG_FWD);
  const int H4 = H >> 2;
  const int N = min(n_cap, dims.nodes(n_cap));
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)N * H4) return;
  const int i = (int)(t / H4), c = (int)(t % H4) * 4;
  const int r0 = row_ptr[i], r1 = row_ptr[i + 1];
  const int d = r1 - r0;
  float *out = agg ? agg + (size_t)i * kAgg * H + c : nullptr;
  const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
  if (d <= 0 || r0 < 0) {
    if (d < 0 || r0 < 0) flag(err, kErrIndex);
    if (out)
#pragma unroll
      for (int a = 0; a < kAgg; ++a) st4(out + a * H, z);
    if (S16)
      for (int a = 0; a < kScalers * kAgg; ++a) st_bf16x4(S16 + (size_t)i * ld16 + a * H + c, 0.f, 0.f, 0.f, 0.f);
    return;
  }
  const float4 P = ld4(PQ + (size_t)i * 2 * H + c);
  float4 s = z;
  float4 mn = make_float4(FLT_MAX, FLT_MAX, FLT_MAX, FLT_MAX);
  float4 mx = make_float4(-FLT_MAX, -FLT_MAX, -FLT_MAX, -FLT_MAX);
  float4 mc[kCache];
  auto take = [&](float4 m) {
    s = add4(s, m);
    mn.x = fminf(mn.x, m.x); mn.y = fminf(mn.y, m.y); mn.z = fminf(mn.z, m.z); mn.w = fminf(mn.w, m.w);
    mx.x = fmaxf(mx.x, m.x); mx.y = fmaxf(mx.y, m.y); mx.z = fmaxf(mx.z, m.z); mx.w = fmaxf(mx.w, m.w);
  };
#pragma unroll
  for (int k = 0; k < kCache; ++k) {
    if (k < d) {
      mc[k] = message(PQ, source(col, r0 + k, N, err), H, c, P);
      take(mc[k]);
    }
  }
  for (int e = r0 + kCache; e < r1; ++e) take(message(PQ, source(col, e, N, err), H, c, P));
  const float df = (float)d;
  const float4 mean = make_float4(s.x / df, s.y / df, s.z / df, s.w / df);
  float4 v = z;  // two-pass variance
#pragma unroll
  for (int k = 0; k < kCache; ++k)
    if (k < d) acc_sq(v, mc[k], mean);
  for (int e = r0 + kCache; e < r1; ++e) acc_sq(v, message(PQ, source(col, e, N, err), H, c, P), mean);
  float4 sd;
  sd.x = sqrtf(fmaxf(v.x / df, 0.f) + eps);
  sd.y = sqrtf(fmaxf(v.y / df, 0.f) + eps);
  sd.z = sqrtf(fmaxf(v.z / df, 0.f) + eps);
  sd.w = sqrtf(fmaxf(v.w / df, 0.f) + eps);
  if (out) {
    st4(out + 0 * H, s);
    st4(out + 1 * H, mean);
    st4(out + 2 * H, mn);
    st4(out + 3 * H, mx);
    st4(out + 4 * H, sd);
  }
  if (S16) {  // scaler-major: identity, amplification, attenuation
    const float4 vv[kAgg] = {s, mean, mn, mx, sd};
    const float sc[kScalers] = {1.f, amp[i], att[i]};
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

__global__ void __launch_bounds__(kEdgeThreads)
aggregate_bwd_edge_kernel(int n_cap, int e_cap, int H, DevDims dims, const int *__restrict__ row_ptr,
                          const int *__restrict__ col, const int *__restrict__ rev,
                          const float *__restrict__ PQ, const float *__restrict__ agg,
                          const float *__restrict__ dagg, float *__restrict__ dPQ,
                          float *__restrict__ dm, unsigned *err, uint16_t *__restrict__ dPQ16, int ld16, float eps) {
  pdl_entry(GCNN_K_AGG_BWD_EDGE);
  const int H4 = H >> 2;
  const int N = min(n_cap, dims.nodes(n_cap));
  const int E = min(e_cap, dims.edges(e_cap));
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)N * H4) return;
  const int i = (int)(t / H4), c = (int)(t % H4) * 4;
  const int r0 = row_ptr[i], r1 = row_ptr[i + 1];
  const int d = r1 - r0;
  float4 dP = make_float4(0.f, 0.f, 0.f, 0.f);
  if (d <= 0 || r0 < 0 || r1 > E) {
    if (d < 0 || r0 < 0 || r1 > E) flag(err, kErrIndex);
    st4(dPQ + (size_t)i * 2 * H + c, dP);
    if (dPQ16) st_bf16x4(dPQ16 + (size_t)i * ld16 + c, 0.f, 0.f, 0.f, 0.f);
    return;
  }
  const float df = (float)d;
  const float4 P = ld4(PQ + (size_t)i * 2 * H + c);
  float4 mc[kCache];
#pragma unroll
  for (int k = 0; k < kCache; ++k)
    if (k < d) mc[k] = message(PQ, source(col, r0 + k, N, err), H, c, P);
  // the forward's statistics: stored, or recomputed in the forward's order
  float4 mean, mn, mx, sd;
  if (agg) {
    const float *a = agg + (size_t)i * kAgg * H + c;
    mean = ld4(a + 1 * H); mn = ld4(a + 2 * H); mx = ld4(a + 3 * H); sd = ld4(a + 4 * H);
  } else {
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
    for (int e = r0 + kCache; e < r1; ++e) take(message(PQ, source(col, e, N, err), H, c, P));
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
  for (int e = r0 + kCache; e < r1; ++e) count(message(PQ, source(col, e, N, err), H, c, P));
  var.x /= df; var.y /= df; var.z /= df; var.w /= df;
  if (!agg) {
    sd.x = sqrtf(fmaxf(var.x, 0.f) + eps);
    sd.y = sqrtf(fmaxf(var.y, 0.f) + eps);
    sd.z = sqrtf(fmaxf(var.z, 0.f) + eps);
    sd.w = sqrtf(fmaxf(var.w, 0.f) + eps);
  }
  // per-node routing coefficients: every edge gets base = dsum + dmean / d,
  // plus dmin / (number of minima) at a minimum, dmax / (number of maxima) at
  // a maximum and dstd (m - mean) / (d std) where the variance is positive
  const float *da = dagg + (size_t)i * kAgg * H + c;
  const float4 dsum = ld4(da + 0 * H), dmean = ld4(da + 1 * H), dmin = ld4(da + 2 * H);
  const float4 dmax = ld4(da + 3 * H), dstd = ld4(da + 4 * H);
  const float4 base = make_float4(dsum.x + dmean.x / df, dsum.y + dmean.y / df, dsum.z + dmean.z / df,
                                  dsum.w + dmean.w / df);
  const float4 cmin = make_float4(dmin.x / nmin.x, dmin.y / nmin.y, dmin.z / nmin.z, dmin.w / nmin.w);
  const float4 cmax = make_float4(dmax.x / nmax.x, dmax.y / nmax.y, dmax.z / nmax.z, dmax.w / nmax.w);
  const float4 cstd = make_float4(var.x > 0.f ? dstd.x / (df * sd.x) : 0.f, var.y > 0.f ? dstd.y / (df * sd.y) : 0.f,
                                  var.z > 0.f ? dstd.z / (df * sd.z) : 0.f, var.w > 0.f ? dstd.w / (df * sd.w) : 0.f);
  auto emit = [&](int e, float4 m) {
    float4 g;
    g.x = route(m.x, base.x, mn.x, cmin.x, mx.x, cmax.x, mean.x, cstd.x);
    g.y = route(m.y, base.y, mn.y, cmin.y, mx.y, cmax.y, mean.y, cstd.y);
    g.z = route(m.z, base.z, mn.z, cmin.z, mx.z, cmax.z, mean.z, cstd.z);
    g.w = route(m.w, base.w, mn.w, cmin.w, mx.w, cmax.w, mean.w, cstd.w);
    dP = add4(dP, g);
    const int re = rev[e];
    if (re >= 0 && re < E) st4(dm + (size_t)re * H + c, g);
    else flag(err, kErrIndex);
  };
#pragma unroll
  for (int k = 0; k < kCache; ++k)
    if (k < d) emit(r0 + k, mc[k]);
  for (int e = r0 + kCache; e < r1; ++e) emit(e, message(PQ, source(col, e, N, err), H, c, P));
  st4(dPQ + (size_t)i * 2 * H + c, dP);
  if (dPQ16) st_bf16x4(dPQ16 + (size_t)i * ld16 + c, dP.x, dP.y, dP.z, dP.w);
}

__global__ void __launch_bounds__(kThreads)
aggregate_bwd_gather_kernel(int n_cap, int e_cap, int H, DevDims dims,
                            const int *__restrict__ row_ptr, const float *__restrict__ dm,
                            float *__restrict__ dPQ, unsigned *err, uint16_t *__restrict__ dPQ16, int ld16) {
  pdl_entry(GCNN_K_AGG_BWD_GATHER);
  const int H4 = H >> 2;
  const int N = min(n_cap, dims.nodes(n_cap));
  const int E = min(e_cap, dims.edges(e_cap));
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)N * H4) return;
  const int j = (int)(t / H4), c = (int)(t % H4) * 4;
  int r0 = row_ptr[j], r1 = row_ptr[j + 1];
  if (r1 < r0 || r0 < 0 || r1 > E) { flag(err, kErrIndex); r1 = r0; }
  float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 4
  for (int e = r0; e < r1; ++e) q = add4(q, ld4(dm + (size_t)e * H + c));
  st4(dPQ + (size_t)j * 2 * H + H + c, q);
  if (dPQ16) st_bf16x4(dPQ16 + (size_t)j * ld16 + H + c, q.x, q.y, q.z, q.w);
}

}  // namespace

int launch_aggregate_fwd(int n_nodes, int H, DevDims dims, const int *row_ptr, const int *col,
                         const float *PQ, float *agg, float eps, unsigned *err, cudaStream_t s,
                         uint16_t *S16, int ld16, const float *amp, const float *att) {
  if (H <= 0 || H % 4) return set_error(GCNN_EINVAL, "aggregate: hidden must be a positive multiple of 4");
  if (n_nodes <= 0) return GCNN_OK;
  const long long work = (long long)n_nodes * (H / 4);
  GCNN_TRY(launch(aggregate_fwd_kernel, ceil_div(work, kThreads), kThreads, 0, s, n_nodes, H, dims, row_ptr, col, PQ,
                  agg, eps, err, S16, ld16, amp, att));
  return GCNN_OK;
}

int launch_aggregate_bwd(int n_nodes, int n_edges, int H, DevDims dims, const int *row_ptr,
                         const int *col, const int *rev, const float *PQ, const float *agg,
                         const float *dagg, float *dPQ, float *scratch, float eps, unsigned *err,
                         cudaStream_t s, uint16_t *dPQ16, int ld16) {
  if (H <= 0 || H % 4) return set_error(GCNN_EINVAL, "aggregate: hidden must be a positive multiple of 4");
  if (n_nodes <= 0) return GCNN_OK;
  const long long work = (long long)n_nodes * (H / 4);
  GCNN_TRY(launch(aggregate_bwd_edge_kernel, ceil_div(work, kEdgeThreads), kEdgeThreads, 0, s, n_nodes, n_edges, H, dims,
                  row_ptr, col, rev, PQ, agg, dagg, dPQ, scratch, err, dPQ16, ld16, eps));
  GCNN_TRY(launch(aggregate_bwd_gather_kernel, ceil_div(work, kThreads), kThreads, 0, s, n_nodes, n_edges, H, dims,
                  row_ptr, (const float *)scratch, dPQ, err, dPQ16, ld16));
  return GCNN_OK;
}

GCNN_TIMELINE_ATTACH(aggregate)

}  // namespace gcnn
