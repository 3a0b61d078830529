// The light steps of the path: atom-type embedding (node features, Sec. 3.1)
// and its gradient, global mean pooling (Sec. 3.1) and its gradient, the
// fully connected head (Sec. 3.1) with the MSE loss (Sec. 3.2) and its
// gradient, and the AdamW update (Sec. 3.2; Sec. 5.1 uses AdamW, lr 1e-3).
// All reductions run in a fixed order (no atomics), so results are
// bit-reproducible run to run.
#include <algorithm>

#include "kernels.cuh"

namespace gcnn {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void st4(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }

// ---------------------------------------------------------------- embedding
__global__ void embed_kernel(int n_cap, int H, DevDims dims, const uint8_t *__restrict__ types,
                             const float *__restrict__ emb, int T, float *__restrict__ x0,
                             uint16_t *__restrict__ x0_16, int ld16) {
  const int H4 = H >> 2;
  const int N = min(n_cap, dims.nodes(n_cap));
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)N * H4) return;
  const int i = (int)(t / H4), c = (int)(t % H4) * 4;
  const int ty = types[i];
  const float4 v = ty < T ? ld4(emb + (size_t)ty * H + c) : make_float4(0.f, 0.f, 0.f, 0.f);
  st4(x0 + (size_t)i * H + c, v);
  if (x0_16) st_bf16x4(x0_16 + (size_t)i * ld16 + c, v.x, v.y, v.z, v.w);
}

constexpr int kEmbChunk = 16;   // nodes per partial sum
constexpr int kMaxTypes = 16;

// partial[ch][t][c] = sum over nodes of chunk ch with type t of dx0[., c]
__global__ void embed_bwd_partial_kernel(int n_cap, int H, DevDims dims,
                                         const uint8_t *__restrict__ types,
                                         const float *__restrict__ dx0, int T,
                                         float *__restrict__ partial) {
  const int N = min(n_cap, dims.nodes(n_cap));
  const int ch = blockIdx.x;
  const int i0 = ch * kEmbChunk;
  const int H4 = H >> 2;
  const int c4 = blockIdx.y * blockDim.x + threadIdx.x;
  if (c4 >= H4) return;
  float4 acc[kMaxTypes];
#pragma unroll
  for (int t = 0; t < kMaxTypes; ++t) acc[t] = make_float4(0.f, 0.f, 0.f, 0.f);
  if (i0 < N) {
    const int i1 = min(N, i0 + kEmbChunk);
    for (int i = i0; i < i1; ++i) {
      const int ty = types[i];
      const float4 v = ld4(dx0 + (size_t)i * H + c4 * 4);
#pragma unroll
      for (int t = 0; t < kMaxTypes; ++t)
        if (t == ty) { acc[t].x += v.x; acc[t].y += v.y; acc[t].z += v.z; acc[t].w += v.w; }
    }
  }
  for (int t = 0; t < T; ++t) st4(partial + ((size_t)ch * T + t) * H + c4 * 4, acc[t]);
}

__global__ void embed_bwd_reduce_kernel(int n_cap, int H, DevDims dims, int T,
                                        const float *__restrict__ partial, float *__restrict__ demb) {
  const int N = min(n_cap, dims.nodes(n_cap));
  const int chunks = (N + kEmbChunk - 1) / kEmbChunk;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;  // over T * H
  if (idx >= T * H) return;
  float s = 0.f;
  for (int ch = 0; ch < chunks; ++ch) s += partial[(size_t)ch * T * H + idx];
  demb[idx] = s;
}

// ---------------------------------------------------------------- pooling
__global__ void pool_fwd_kernel(int g_cap, int H, DevDims dims, const int *__restrict__ node_off,
                                const float *__restrict__ x, float *__restrict__ pooled) {
  const int H4 = H >> 2;
  const int G = min(g_cap, dims.graphs(g_cap));
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)G * H4) return;
  const int g = (int)(t / H4), c = (int)(t % H4) * 4;
  const int a = node_off[g], b = node_off[g + 1];
  float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int i = a; i < b; ++i) {
    const float4 v = ld4(x + (size_t)i * H + c);
    s.x += v.x; s.y += v.y; s.z += v.z; s.w += v.w;
  }
  if (b > a) {
    const float n = (float)(b - a);
    s.x /= n; s.y /= n; s.z /= n; s.w /= n;
  }
  st4(pooled + (size_t)g * H + c, s);
}

__global__ void pool_bwd_kernel(int n_cap, int H, DevDims dims, const int *__restrict__ node_off,
                                const int *__restrict__ graph_id, const float *__restrict__ dpooled,
                                float *__restrict__ dx, uint16_t *__restrict__ D3, int ld3, const float *__restrict__ h,
                                const float *__restrict__ amp, const float *__restrict__ att) {
  const int H4 = H >> 2;
  const int N = min(n_cap, dims.nodes(n_cap));
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)N * H4) return;
  const int i = (int)(t / H4), c = (int)(t % H4) * 4;
  const int g = graph_id[i];
  const float n = (float)(node_off[g + 1] - node_off[g]);
  const float4 v = ld4(dpooled + (size_t)g * H + c);
  const float4 d = make_float4(v.x / n, v.y / n, v.z / n, v.w / n);
  st4(dx + (size_t)i * H + c, d);
  if (D3) {
    const float4 m = ld4(h + (size_t)i * H + c);
    const float gx = m.x > 0.f ? d.x : 0.f, gy = m.y > 0.f ? d.y : 0.f;
    const float gz = m.z > 0.f ? d.z : 0.f, gw = m.w > 0.f ? d.w : 0.f;
    const float a = amp[i], t = att[i];
    uint16_t *o = D3 + (size_t)i * ld3 + c;
    st_bf16x4(o, a * gx, a * gy, a * gz, a * gw);
    st_bf16x4(o + H, t * gx, t * gy, t * gz, t * gw);
    st_bf16x4(o + 2 * H, gx, gy, gz, gw);
  }
}

// ---------------------------------------------------------------- head
// Deterministic block sum of one float per thread (blockDim.x == kThreads).
__device__ float block_sum(float v, float *sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  float s = 0.f;
  if (threadIdx.x == 0)
    for (int q = 0; q < kThreads / 32; ++q) s += sh[q];
  return s;  // valid in thread 0
}

__device__ double block_sum_d(double v, double *sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int q = 0; q < kThreads / 32; ++q) s += sh[q];
  return s;
}

// one block per graph
__global__ void __launch_bounds__(kThreads)
head_fwd_kernel(int g_cap, int H, int Hh, DevDims dims, const float *__restrict__ g,
                const float *__restrict__ w1, const float *__restrict__ b1,
                const float *__restrict__ w2, const float *__restrict__ b2,
                float *__restrict__ z1, float *__restrict__ pred) {
  extern __shared__ float sg[];  // H floats
  __shared__ float red[kThreads / 32];
  const int G = min(g_cap, dims.graphs(g_cap));
  const int gr = blockIdx.x;
  if (gr >= G) return;  // block-uniform
  for (int k = threadIdx.x; k < H; k += blockDim.x) sg[k] = g[(size_t)gr * H + k];
  __syncthreads();
  float part = 0.f;
  for (int c = threadIdx.x; c < Hh; c += blockDim.x) {
    float a[4] = {b1[c], 0.f, 0.f, 0.f};  // four independent chains, summed in a fixed order
    int k = 0;
    for (; k + 4 <= H; k += 4) {
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] += sg[k + u] * w1[(size_t)(k + u) * Hh + c];
    }
    for (; k < H; ++k) a[0] += sg[k] * w1[(size_t)k * Hh + c];
    const float acc = (a[0] + a[1]) + (a[2] + a[3]);
    z1[(size_t)gr * Hh + c] = acc;
    part += fmaxf(acc, 0.f) * w2[c];
  }
  const float s = block_sum(part, red);
  if (threadIdx.x == 0) pred[gr] = s + b2[0];
}

// one block: dL/dpred, the loss sums and the gradient of b2 (G values)
__global__ void __launch_bounds__(kThreads)
head_bwd_loss_kernel(int g_cap, DevDims dims, const float *__restrict__ pred, const float *__restrict__ y,
                     const float *__restrict__ dpred_in, float *__restrict__ dpred, float *__restrict__ grad_b2,
                     double *__restrict__ loss_accum) {
  __shared__ double redd[kThreads / 32];
  __shared__ float redf[kThreads / 32];
  const int G = min(g_cap, dims.graphs(g_cap));
  double se = 0.0, ae = 0.0;
  float db2 = 0.f;
  for (int gr = threadIdx.x; gr < G; gr += blockDim.x) {
    const float r = pred[gr] - y[gr];
    const float dp = dpred_in ? dpred_in[gr] : 2.f * r / (float)G;
    dpred[gr] = dp;
    se += (double)r * (double)r;
    ae += fabs((double)r);
    db2 += dp;
  }
  const double sse = block_sum_d(se, redd);
  const double sae = block_sum_d(ae, redd);
  const float sdb2 = block_sum(db2, redf);
  if (threadIdx.x == 0) {
    grad_b2[0] = sdb2;
    if (loss_accum) {
      loss_accum[0] += sse;
      loss_accum[1] += sae;
      loss_accum[2] += (double)G;
    }
  }
}

// grads of w1 (H x Hh), b1, w2 and dg (G x H): one thread per output, sums
// over graphs / head units in a fixed order; dz1 = [z1 > 0] dpred w2 inline
__global__ void __launch_bounds__(kThreads)
head_bwd_grad_kernel(int g_cap, int H, int Hh, DevDims dims, const float *__restrict__ g,
                     const float *__restrict__ w1, const float *__restrict__ w2, const float *__restrict__ z1,
                     const float *__restrict__ dpred, float *__restrict__ grad_head, float *__restrict__ dg) {
  const int G = min(g_cap, dims.graphs(g_cap));
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long n_w1 = (long long)H * Hh;
  if (idx < n_w1) {
    const int k = (int)(idx / Hh), c = (int)(idx % Hh);
    const float wc = w2[c];
    float a[4] = {0.f, 0.f, 0.f, 0.f};
    int gr = 0;
    for (; gr + 4 <= G; gr += 4) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float z = z1[(size_t)(gr + u) * Hh + c];
        a[u] += z > 0.f ? g[(size_t)(gr + u) * H + k] * (dpred[gr + u] * wc) : 0.f;
      }
    }
    for (; gr < G; ++gr) {
      const float z = z1[(size_t)gr * Hh + c];
      a[0] += z > 0.f ? g[(size_t)gr * H + k] * (dpred[gr] * wc) : 0.f;
    }
    grad_head[idx] = (a[0] + a[1]) + (a[2] + a[3]);
  } else if (idx < n_w1 + Hh) {
    const int c = (int)(idx - n_w1);
    const float wc = w2[c];
    float s = 0.f;
    for (int gr = 0; gr < G; ++gr) s += z1[(size_t)gr * Hh + c] > 0.f ? dpred[gr] * wc : 0.f;
    grad_head[idx] = s;
  } else if (idx < n_w1 + 2 * Hh) {
    const int c = (int)(idx - n_w1 - Hh);
    float s = 0.f;
    for (int gr = 0; gr < G; ++gr) s += fmaxf(z1[(size_t)gr * Hh + c], 0.f) * dpred[gr];
    grad_head[idx] = s;
  } else if (idx < n_w1 + 2 * Hh + (long long)g_cap * H) {
    const long long r = idx - n_w1 - 2 * Hh;
    const int gr = (int)(r / H), k = (int)(r % H);
    if (gr >= G) return;
    const float dp = dpred[gr];
    float a[4] = {0.f, 0.f, 0.f, 0.f};
    int c = 0;
    for (; c + 4 <= Hh; c += 4) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float z = z1[(size_t)gr * Hh + c + u];
        a[u] += z > 0.f ? w1[(size_t)k * Hh + c + u] * (dp * w2[c + u]) : 0.f;
      }
    }
    for (; c < Hh; ++c) {
      const float z = z1[(size_t)gr * Hh + c];
      a[0] += z > 0.f ? w1[(size_t)k * Hh + c] * (dp * w2[c]) : 0.f;
    }
    dg[(size_t)gr * H + k] = (a[0] + a[1]) + (a[2] + a[3]);
  }
}

// ---------------------------------------------------------------- AdamW
// step[0]: step counter; coef[0] = 1/(1-beta1^t), coef[1] = 1/(1-beta2^t)
__global__ void adam_tick_kernel(int *step, float *coef, float beta1, float beta2) {
  const int t = step[0] + 1;
  step[0] = t;
  coef[0] = (float)(1.0 / (1.0 - pow((double)beta1, (double)t)));
  coef[1] = (float)(1.0 / (1.0 - pow((double)beta2, (double)t)));
}

__device__ __forceinline__ void adam_one(float &p, float g, float &m, float &v, float lr, float c1,
                                         float c2, float b1, float b2, float eps, float wd) {
  if (wd > 0.f) p -= lr * wd * p;
  m = b1 * m + (1.f - b1) * g;
  v = b2 * v + (1.f - b2) * g * g;
  p -= lr * (m * c1) / (sqrtf(v * c2) + eps);
}

__global__ void __launch_bounds__(kThreads)
adam_kernel(int64_t n, float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
            float *__restrict__ v, const float *__restrict__ coef, const float *__restrict__ lrp,
            float b1, float b2, float eps, float wd) {
  const float c1 = coef[0], c2 = coef[1], lr = lrp[0];
  const int64_t n4 = n / 4;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n4; q += stride) {
    float4 P = ld4(p + 4 * q), Gv = ld4(g + 4 * q), Mv = ld4(m + 4 * q), V = ld4(v + 4 * q);
    adam_one(P.x, Gv.x, Mv.x, V.x, lr, c1, c2, b1, b2, eps, wd);
    adam_one(P.y, Gv.y, Mv.y, V.y, lr, c1, c2, b1, b2, eps, wd);
    adam_one(P.z, Gv.z, Mv.z, V.z, lr, c1, c2, b1, b2, eps, wd);
    adam_one(P.w, Gv.w, Mv.w, V.w, lr, c1, c2, b1, b2, eps, wd);
    st4(p + 4 * q, P);
    st4(m + 4 * q, Mv);
    st4(v + 4 * q, V);
  }
  if (blockIdx.x == 0 && threadIdx.x < (int)(n - 4 * n4)) {
    const int64_t k = 4 * n4 + threadIdx.x;
    float P = p[k], M = m[k], V = v[k];
    adam_one(P, g[k], M, V, lr, c1, c2, b1, b2, eps, wd);
    p[k] = P; m[k] = M; v[k] = V;
  }
}

constexpr int kColChunk = 32;  // nodes per partial column sum

// Column c < cols of the virtual matrix [a0 * [mask > 0] | a1] (a1 nullable):
// partial[ch][c] = sum over the nodes of chunk ch.
__global__ void colsum_partial_kernel(int n_cap, int cols0, int cols1, DevDims dims, const float *__restrict__ a0,
                                      int ld0, const float *__restrict__ mask, int ldm, const float *__restrict__ a1,
                                      int ld1, float *__restrict__ partial) {
  const int N = min(n_cap, dims.nodes(n_cap));
  const int cols = cols0 + cols1;
  const int ch = blockIdx.y;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  const int i0 = ch * kColChunk;
  float v[kColChunk];
#pragma unroll
  for (int q = 0; q < kColChunk; ++q) {
    const int i = i0 + q;
    float x = 0.f;
    if (i < N) {
      if (c < cols0) {
        x = a0[(size_t)i * ld0 + c];
        if (mask && !(mask[(size_t)i * ldm + c] > 0.f)) x = 0.f;
      } else {
        x = a1[(size_t)i * ld1 + (c - cols0)];
      }
    }
    v[q] = x;
  }
  float sum = 0.f;
#pragma unroll
  for (int q = 0; q < kColChunk; ++q) sum += v[q];
  partial[(size_t)ch * cols + c] = sum;
}

__global__ void colsum_reduce_kernel(int n_cap, int cols0, int cols1, DevDims dims, const float *__restrict__ partial,
                                     float *__restrict__ out0, float *__restrict__ out1) {
  const int N = min(n_cap, dims.nodes(n_cap));
  const int cols = cols0 + cols1;
  const int chunks = (N + kColChunk - 1) / kColChunk;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  float a[4] = {0.f, 0.f, 0.f, 0.f};
  int ch = 0;
  for (; ch + 4 <= chunks; ch += 4) {
#pragma unroll
    for (int u = 0; u < 4; ++u) a[u] += partial[(size_t)(ch + u) * cols + c];
  }
  for (; ch < chunks; ++ch) a[0] += partial[(size_t)ch * cols + c];
  const float s = (a[0] + a[1]) + (a[2] + a[3]);
  if (c < cols0) out0[c] = s;
  else out1[c - cols0] = s;
}

}  // namespace

int launch_colsum2(int n_cap, int cols0, int cols1, DevDims dims, const float *a0, int ld0, const float *mask,
                   int ldm, const float *a1, int ld1, float *partial, float *out0, float *out1, cudaStream_t s) {
  const int cols = cols0 + cols1;
  if (cols <= 0) return GCNN_OK;
  const int chunks = (int)ceil_div(std::max(n_cap, 1), kColChunk);
  dim3 grid(ceil_div(cols, 128), chunks);
  colsum_partial_kernel<<<grid, 128, 0, s>>>(n_cap, cols0, cols1, dims, a0, ld0, mask, ldm, a1, ld1, partial);
  GCNN_LAUNCH_CHECK();
  colsum_reduce_kernel<<<ceil_div(cols, 128), 128, 0, s>>>(n_cap, cols0, cols1, dims, partial, out0, out1);
  GCNN_LAUNCH_CHECK();
  return GCNN_OK;
}

int launch_embed(int n_nodes, int H, DevDims dims, const uint8_t *types, const float *emb,
                 int n_types, float *x0, cudaStream_t s, uint16_t *x0_16, int ld16) {
  if (n_nodes <= 0) return GCNN_OK;
  const long long work = (long long)n_nodes * (H / 4);
  embed_kernel<<<ceil_div(work, kThreads), kThreads, 0, s>>>(n_nodes, H, dims, types, emb, n_types, x0, x0_16, ld16);
  GCNN_LAUNCH_CHECK();
  return GCNN_OK;
}

int launch_embed_bwd(int n_nodes, int H, DevDims dims, const uint8_t *types, const float *dx0,
                     int n_types, float *partial, int max_chunks, float *demb, cudaStream_t s) {
  if (n_types > kMaxTypes) return set_error(GCNN_EINVAL, "at most %d atom types", kMaxTypes);
  const int chunks = (int)ceil_div(n_nodes, kEmbChunk);
  if (chunks > max_chunks) return set_error(GCNN_EINVAL, "embedding workspace too small");
  const int H4 = H / 4;
  if (chunks > 0) {
    dim3 grid(chunks, ceil_div(H4, 64));
    embed_bwd_partial_kernel<<<grid, 64, 0, s>>>(n_nodes, H, dims, types, dx0, n_types, partial);
    GCNN_LAUNCH_CHECK();
  }
  embed_bwd_reduce_kernel<<<ceil_div((long long)n_types * H, kThreads), kThreads, 0, s>>>(
      n_nodes, H, dims, n_types, partial, demb);
  GCNN_LAUNCH_CHECK();
  return GCNN_OK;
}

int launch_pool_fwd(int G, int H, DevDims dims, const int *node_off, const float *x, float *pooled,
                    cudaStream_t s) {
  if (G <= 0) return GCNN_OK;
  const long long work = (long long)G * (H / 4);
  pool_fwd_kernel<<<ceil_div(work, kThreads), kThreads, 0, s>>>(G, H, dims, node_off, x, pooled);
  GCNN_LAUNCH_CHECK();
  return GCNN_OK;
}

int launch_pool_bwd(int G, int n_nodes, int H, DevDims dims, const int *node_off,
                    const int *graph_id, const float *dpooled, float *dx, cudaStream_t s, uint16_t *D3,
                    int ld3, const float *h, const float *amp, const float *att) {
  (void)G;
  if (n_nodes <= 0) return GCNN_OK;
  const long long work = (long long)n_nodes * (H / 4);
  pool_bwd_kernel<<<ceil_div(work, kThreads), kThreads, 0, s>>>(n_nodes, H, dims, node_off, graph_id,
                                                                 dpooled, dx, D3, ld3, h, amp, att);
  GCNN_LAUNCH_CHECK();
  return GCNN_OK;
}

int launch_head_fwd(int G, int H, int Hh, DevDims dims, const float *g, const float *w1,
                    const float *b1, const float *w2, const float *b2, float *z1, float *pred,
                    cudaStream_t s) {
  if (G <= 0) return GCNN_OK;
  head_fwd_kernel<<<G, kThreads, H * sizeof(float), s>>>(G, H, Hh, dims, g, w1, b1, w2, b2, z1, pred);
  GCNN_LAUNCH_CHECK();
  return GCNN_OK;
}

int launch_head_bwd(int G, int H, int Hh, DevDims dims, const float *g, const float *w1,
                    const float *w2, const float *z1, const float *pred, const float *y,
                    const float *dpred_in, float *dpred, float *dz1, float *grad_head, float *dg,
                    double *loss_accum, cudaStream_t s) {
  (void)dz1;
  float *grad_b2 = grad_head + (size_t)H * Hh + 2 * Hh;
  head_bwd_loss_kernel<<<1, kThreads, 0, s>>>(G, dims, pred, y, dpred_in, dpred, grad_b2, loss_accum);
  GCNN_LAUNCH_CHECK();
  const long long work = (long long)H * Hh + 2 * Hh + (long long)G * H;
  head_bwd_grad_kernel<<<ceil_div(work, kThreads), kThreads, 0, s>>>(G, H, Hh, dims, g, w1, w2, z1, dpred,
                                                                      grad_head, dg);
  GCNN_LAUNCH_CHECK();
  return GCNN_OK;
}

int launch_adam(int64_t n, float *param, const float *grad, float *m, float *v, int *step,
                const float *lr, float beta1, float beta2, float eps, float wd, cudaStream_t s) {
  // coef lives right after the step counter (two floats)
  float *coef = reinterpret_cast<float *>(step + 1);
  adam_tick_kernel<<<1, 1, 0, s>>>(step, coef, beta1, beta2);
  GCNN_LAUNCH_CHECK();
  int blocks = (int)std::min<int64_t>((n / 4 + kThreads - 1) / kThreads + 1, 152 * 8);
  adam_kernel<<<blocks, kThreads, 0, s>>>(n, param, grad, m, v, coef, lr, beta1, beta2, eps, wd);
  GCNN_LAUNCH_CHECK();
  return GCNN_OK;
}

}  // namespace gcnn
