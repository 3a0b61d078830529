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
  pdl_entry(GCNN_K_EMBED);
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

constexpr int kMaxTypes = 16;
constexpr int kRedThreads = 256;
constexpr int kEmbBwdThreads = 512;   // one block per 4-column slice: nodes strided over the block
constexpr int kColsumThreads = 1024;
constexpr int kColsumWidth = 32;    // columns per CTA of the bias sums
constexpr int kColsumMaxRanks = 8;  // CTAs of a cluster (row ranges), portable size

__device__ __forceinline__ float4 add4(float4 a, float4 b) {
  return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}

// barrier over every thread of the cluster's CTAs (release / acquire)
__device__ __forceinline__ void colsum_cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// 16 bytes at shared-memory address a of the cluster's CTA `rank`
__device__ __forceinline__ float4 colsum_ld_cluster4(uint32_t a, int rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  float4 v;
  asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(r)
               : "memory");
  return v;
}

// Butterfly sum over the warp (fixed order; every lane gets the total).
__device__ __forceinline__ float4 warp_sum4(float4 a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a.x += __shfl_xor_sync(0xffffffffu, a.x, o);
    a.y += __shfl_xor_sync(0xffffffffu, a.y, o);
    a.z += __shfl_xor_sync(0xffffffffu, a.z, o);
    a.w += __shfl_xor_sync(0xffffffffu, a.w, o);
  }
  return a;
}

// dEmb[t][c..c+3] = sum of dx0[i][c..c+3] over the nodes i of type t.  One
// block per 4-column slice; nodes strided over the block's threads, then a
// fixed-order reduction (warp butterflies, warps in index order).
__global__ void __launch_bounds__(kEmbBwdThreads)
embed_bwd_kernel(int n_cap, int H, DevDims dims, const uint8_t *__restrict__ types, const float *__restrict__ dx0,
                 int T, float *__restrict__ demb) {
  pdl_entry(GCNN_K_EMBED_BWD);
  __shared__ float4 sh[kEmbBwdThreads / 32][kMaxTypes];
  const int N = min(n_cap, dims.nodes(n_cap));
  const int c = blockIdx.x * 4;
  float4 acc[kMaxTypes];
#pragma unroll
  for (int t = 0; t < kMaxTypes; ++t) acc[t] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 4
  for (int i = threadIdx.x; i < N; i += kEmbBwdThreads) {
    const int ty = types[i];
    const float4 v = ld4(dx0 + (size_t)i * H + c);
#pragma unroll
    for (int t = 0; t < kMaxTypes; ++t)
      if (t == ty) acc[t] = add4(acc[t], v);
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int t = 0; t < kMaxTypes; ++t) {
    if (t >= T) break;
    const float4 a = warp_sum4(acc[t]);
    if (lane == 0) sh[w][t] = a;
  }
  __syncthreads();
  if (threadIdx.x < T) {
    float4 sum = sh[0][threadIdx.x];
    for (int q = 1; q < kEmbBwdThreads / 32; ++q) sum = add4(sum, sh[q][threadIdx.x]);
    st4(demb + (size_t)threadIdx.x * H + c, sum);
  }
}

// ---------------------------------------------------------------- pooling
__global__ void pool_fwd_kernel(int g_cap, int H, DevDims dims, const int *__restrict__ node_off,
                                const float *__restrict__ x, float *__restrict__ pooled) {
  pdl_entry(GCNN_K_POOL_FWD);
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
  pdl_entry(GCNN_K_POOL_BWD);
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
// Deterministic block sum of one value per thread (blockDim.x == NT): warp
// butterflies, then the warps' sums in index order.  Valid in thread 0.
template <int NT, typename F>
__device__ F block_sum(F v, F *sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  F s = F(0);
  if (threadIdx.x == 0)
    for (int q = 0; q < NT / 32; ++q) s += sh[q];
  return s;
}

constexpr int kHeadThreads = 512;

// Per-graph part of the head (one block per graph).  Forward: mean pooling of
// the last layer's features, z1 = g W1 + b1, pred = ReLU(z1) w2 + b2.
// Backward: dpred (given, or 2 (pred - y) / G), dz1 = [z1 > 0] dpred w2,
// dg = W1 dz1 and the pooling gradient dx_i = dg / n_g on the graph's nodes,
// optionally also as the BF16 blocks [amp g | att g | g], g = dx [h > 0].
// W1 is staged in shared memory, rk rows at a time.

__device__ __forceinline__ void cp_async16(float *dst_smem, const float *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst_smem)),
               "l"(src)
               : "memory");
}

// partials of the one-chunk path: at most kHeadThreads float4
constexpr int kHeadRed = kHeadThreads;

template <bool kFwd, bool kBwd>
__global__ void __launch_bounds__(kHeadThreads) head_graph_kernel(HeadArgs a) {
  extern __shared__ float sm[];
  __shared__ float red[kHeadThreads / 32];
  __shared__ float s_pred, s_dp;
  const int H = a.H, Hh = a.Hh, rk = a.rk;
  float *Ws = sm;                     // rk x Hh
  float *sv = Ws + (size_t)rk * Hh;   // H: pooled features, later dg
  float *sz = sv + H;                 // Hh: z1
  float *sd = sz + Hh;                // Hh: dz1
  const int gr = blockIdx.x;
  const int tid = threadIdx.x;
  const int nchunks = (H + rk - 1) / rk;
  // one chunk of W1 and whole float4 columns: W1 arrives by asynchronous copies
  // while the graph is pooled
  const bool one = nchunks == 1 && (Hh & 3) == 0;
  // Before the dependency wait: W1 is a parameter (written by the optimizer
  // or by a host copy, never by the kernel just before this one, which is a
  // GEMM of the last layer) and the graph offsets come from the collator, so
  // the copy of W1 and the offsets' loads overlap the previous kernel's tail.
  if (kFwd && one) {
    for (int q = tid; q < H * (Hh >> 2); q += kHeadThreads) cp_async16(Ws + 4 * q, a.w1 + 4 * (size_t)q);
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  const int G = min(a.g_cap, a.dims.graphs(a.g_cap));
  const int n0 = gr < G ? a.node_off[gr] : 0, n1 = gr < G ? a.node_off[gr + 1] : 0, nn = n1 - n0;
  pdl_entry(GCNN_K_HEAD_GRAPH);
  if (gr >= G) {  // block-uniform
    asm volatile("cp.async.wait_all;" ::: "memory");
    return;
  }
  int staged = -1;
  auto stage = [&](int ch) {  // rows [ch * rk, ...) of W1 into Ws
    __syncthreads();
    const int k0 = ch * rk, cnt = min(rk, H - k0) * Hh;
    const float4 *src = reinterpret_cast<const float4 *>(a.w1 + (size_t)k0 * Hh);
    float4 *dst = reinterpret_cast<float4 *>(Ws);
#pragma unroll 4
    for (int q = tid; q < cnt / 4; q += kHeadThreads) dst[q] = src[q];
    for (int q = cnt / 4 * 4 + tid; q < cnt; q += kHeadThreads) Ws[q] = a.w1[(size_t)k0 * Hh + q];
    __syncthreads();
    staged = ch;
  };
  // one chunk: pooling and z1 use every thread (float4 column x row segment,
  // partials summed in segment order) while W1 arrives
  if (kFwd && one) {
    float4 *part4 = reinterpret_cast<float4 *>(sd + Hh);  // kHeadRed float4
    const int H4 = H >> 2, Hh4 = Hh >> 2;
    staged = 0;
    const int R = max(1, kHeadThreads / H4);
    if (tid < R * H4) {
      const int c4 = tid % H4;
      float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int i = n0 + tid / H4; i < n1; i += R) acc = add4(acc, ld4(a.x + (size_t)i * H + 4 * c4));
      part4[tid] = acc;
    }
    __syncthreads();
    for (int c4 = tid; c4 < H4; c4 += kHeadThreads) {
      float4 v = part4[c4];
      for (int r = 1; r < R; ++r) v = add4(v, part4[r * H4 + c4]);
      if (nn > 0) {
        const float inv = (float)nn;
        v = make_float4(v.x / inv, v.y / inv, v.z / inv, v.w / inv);
      }
      st4(sv + 4 * c4, v);
      st4(a.pooled + (size_t)gr * H + 4 * c4, v);
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    const int S = max(1, kHeadThreads / Hh4), kper = (H + S - 1) / S;
    if (tid < S * Hh4) {
      const int c4 = tid % Hh4, seg = tid / Hh4, k1 = min(H, (seg + 1) * kper);
      float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int k = seg * kper; k < k1; ++k) {
        const float gk = sv[k];
        const float4 w = ld4(Ws + (size_t)k * Hh + 4 * c4);
        acc.x = fmaf(gk, w.x, acc.x); acc.y = fmaf(gk, w.y, acc.y);
        acc.z = fmaf(gk, w.z, acc.z); acc.w = fmaf(gk, w.w, acc.w);
      }
      part4[tid] = acc;
    }
    __syncthreads();
    for (int c4 = tid; c4 < Hh4; c4 += kHeadThreads) {
      float4 v = make_float4(a.b1[4 * c4], a.b1[4 * c4 + 1], a.b1[4 * c4 + 2], a.b1[4 * c4 + 3]);
      for (int sg = 0; sg < S; ++sg) v = add4(v, part4[sg * Hh4 + c4]);
      st4(sz + 4 * c4, v);
    }
    __syncthreads();
    float part = 0.f;
    for (int c = tid; c < Hh; c += kHeadThreads) {
      a.z1[(size_t)gr * Hh + c] = sz[c];
      part += fmaxf(sz[c], 0.f) * a.w2[c];
    }
    const float s = block_sum<kHeadThreads>(part, red);
    if (tid == 0) {
      s_pred = s + a.b2[0];
      a.pred[gr] = s_pred;
    }
  } else if (kFwd) {
    for (int k = tid; k < H; k += kHeadThreads) {
      float s4[4] = {0.f, 0.f, 0.f, 0.f};
      int i = n0;
      for (; i + 4 <= n1; i += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u) s4[u] += a.x[(size_t)(i + u) * H + k];
      }
      for (; i < n1; ++i) s4[0] += a.x[(size_t)i * H + k];
      float v = (s4[0] + s4[1]) + (s4[2] + s4[3]);
      if (nn > 0) v /= (float)nn;
      sv[k] = v;
      a.pooled[(size_t)gr * H + k] = v;
    }
    for (int c = tid; c < Hh; c += kHeadThreads) sz[c] = a.b1[c];
    for (int ch = 0; ch < nchunks; ++ch) {
      stage(ch);
      const int k0 = ch * rk, rows = min(rk, H - k0);
      for (int c = tid; c < Hh; c += kHeadThreads) {
        float acc = sz[c];
#pragma unroll 8
        for (int k = 0; k < rows; ++k) acc += sv[k0 + k] * Ws[(size_t)k * Hh + c];
        sz[c] = acc;
      }
    }
    __syncthreads();
    float part = 0.f;
    for (int c = tid; c < Hh; c += kHeadThreads) {
      a.z1[(size_t)gr * Hh + c] = sz[c];
      part += fmaxf(sz[c], 0.f) * a.w2[c];
    }
    const float s = block_sum<kHeadThreads>(part, red);
    if (tid == 0) {
      s_pred = s + a.b2[0];
      a.pred[gr] = s_pred;
    }
  }
  if (kBwd) {
    if (!kFwd) {
      for (int c = tid; c < Hh; c += kHeadThreads) sz[c] = a.z1[(size_t)gr * Hh + c];
      if (tid == 0) s_pred = a.pred[gr];
    }
    __syncthreads();
    if (tid == 0) {
      const float r = s_pred - a.y[gr];
      // the MSE gradient times the loss scale (data-parallel weighting, 1 alone)
      const float dp = a.dpred_in ? a.dpred_in[gr] : (2.f * r / (float)G) * (a.loss_scale ? a.loss_scale[0] : 1.f);
      a.dpred[gr] = dp;
      s_dp = dp;
    }
    __syncthreads();
    const float dp = s_dp;
    for (int c = tid; c < Hh; c += kHeadThreads) {
      const float d = sz[c] > 0.f ? dp * a.w2[c] : 0.f;
      sd[c] = d;
      a.dz1[(size_t)gr * Hh + c] = d;
    }
    // dg = W1 dz1, chunks in reverse order (the forward's last chunk is still
    // staged): one thread per row of W1, four running sums over float4
    // columns (16-byte aligned when Hh is a multiple of 4)
    for (int ch = nchunks - 1; ch >= 0; --ch) {
      if (staged != ch) stage(ch);
      else __syncthreads();
      const int k0 = ch * rk, rows = min(rk, H - k0);
      for (int k = tid; k < rows; k += kHeadThreads) {
        const float *w = Ws + (size_t)k * Hh;
        float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
        int c = 0;
        if ((Hh & 3) == 0) {
#pragma unroll 4
          for (; c < Hh; c += 4) {
            const float4 wv = ld4(w + c), dv = ld4(sd + c);
            s0 = fmaf(wv.x, dv.x, s0); s1 = fmaf(wv.y, dv.y, s1);
            s2 = fmaf(wv.z, dv.z, s2); s3 = fmaf(wv.w, dv.w, s3);
          }
        }
        for (; c < Hh; ++c) s0 = fmaf(w[c], sd[c], s0);
        const float acc = (s0 + s1) + (s2 + s3);
        sv[k0 + k] = acc;
        a.dg[(size_t)gr * H + k0 + k] = acc;
      }
    }
    __syncthreads();
    // mean pooling backward on the graph's nodes, four items per thread at a
    // time: every load of the four before any store
    const float n = (float)nn;
    const int H4 = H >> 2, items = nn * H4;
    constexpr int U = 4;
    for (int q0 = tid; q0 < items; q0 += U * kHeadThreads) {
      float4 e[U], m[U];
      float am[U], at[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int q = min(q0 + u * kHeadThreads, items - 1);  // a valid item; only real ones are stored
        const int i = n0 + q / H4, c = (q % H4) * 4;
        e[u] = a.dx_add ? ld4(a.dx_add + (size_t)i * H + c) : make_float4(0.f, 0.f, 0.f, 0.f);
        if (a.D3) {
          m[u] = ld4(a.h + (size_t)i * H + c);
          am[u] = a.amp[i];
          at[u] = a.att[i];
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int q = q0 + u * kHeadThreads;
        if (q >= items) break;
        const int i = n0 + q / H4, c = (q % H4) * 4;
        // plus the node-level head's gradient on the same atoms, if any
        float4 d = make_float4(sv[c] / n, sv[c + 1] / n, sv[c + 2] / n, sv[c + 3] / n);
        if (a.dx_add) d = make_float4(d.x + e[u].x, d.y + e[u].y, d.z + e[u].z, d.w + e[u].w);
        st4(a.dx + (size_t)i * H + c, d);
        if (a.D3) {
          const float gx = m[u].x > 0.f ? d.x : 0.f, gy = m[u].y > 0.f ? d.y : 0.f;
          const float gz = m[u].z > 0.f ? d.z : 0.f, gw = m[u].w > 0.f ? d.w : 0.f;
          uint16_t *o = a.D3 + (size_t)i * a.ld3 + c;
          st_bf16x4(o, am[u] * gx, am[u] * gy, am[u] * gz, am[u] * gw);
          st_bf16x4(o + H, at[u] * gx, at[u] * gy, at[u] * gz, at[u] * gw);
          st_bf16x4(o + 2 * H, gx, gy, gz, gw);
        }
      }
    }
  }
}

// Head parameter gradients, summed over the batch's graphs in a fixed order:
// W1 (H x Hh) = pooled^T dz1 in 32 x 32 tiles (grid.y < ceil(H / 32)); the last
// row of blocks: b1 = sum dz1, w2 = sum ReLU(z1) dpred, and in block (0, .)
// b2 = sum dpred and the FP64 loss sums (squared and absolute error, count).
constexpr int kHT = 32, kHG = 64;


__global__ void __launch_bounds__(kRedThreads) head_grad_kernel(HeadGradArgs a) {
  pdl_entry(GCNN_K_HEAD_GRAD);
  __shared__ float sp[kHG][kHT + 1], sd[kHG][kHT + 1];
  __shared__ double redd[kRedThreads / 32];
  __shared__ float redf[kRedThreads / 32];
  const int G = min(a.g_cap, a.dims.graphs(a.g_cap));
  const int H = a.H, Hh = a.Hh, tid = threadIdx.x;
  const int c0 = blockIdx.x * kHT;
  const int tc = tid & 31, q8 = tid >> 5;
  if ((int)blockIdx.y < (H + kHT - 1) / kHT) {
    const int k0 = blockIdx.y * kHT;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int g0 = 0; g0 < G; g0 += kHG) {
      const int gn = min(kHG, G - g0);
      __syncthreads();
      for (int q = tid; q < kHG * kHT; q += kRedThreads) {
        const int gg = q / kHT, cc = q % kHT;
        const bool in = gg < gn;
        sp[gg][cc] = in && k0 + cc < H ? a.pooled[(size_t)(g0 + gg) * H + k0 + cc] : 0.f;
        sd[gg][cc] = in && c0 + cc < Hh ? a.dz1[(size_t)(g0 + gg) * Hh + c0 + cc] : 0.f;
      }
      __syncthreads();
      for (int gg = 0; gg < gn; ++gg) {
        const float d = sd[gg][tc];
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[r] += sp[gg][q8 + 8 * r] * d;
      }
    }
    const int c = c0 + tc;
    if (c < Hh)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int k = k0 + q8 + 8 * r;
        if (k < H) a.grad[(size_t)k * Hh + c] = acc[r];
      }
    return;
  }
  // b1 and w2 for columns c0 .. c0 + 31: graphs strided over the 8 warps
  {
    const int c = c0 + tc;
    float sb = 0.f, sw = 0.f;
    if (c < Hh)
      for (int g = q8; g < G; g += kRedThreads / 32) {
        sb += a.dz1[(size_t)g * Hh + c];
        sw += fmaxf(a.z1[(size_t)g * Hh + c], 0.f) * a.dpred[g];
      }
    sp[q8][tc] = sb;
    sd[q8][tc] = sw;
    __syncthreads();
    if (q8 == 0 && c < Hh) {
      float tb = sp[0][tc], tw = sd[0][tc];
      for (int q = 1; q < kRedThreads / 32; ++q) {
        tb += sp[q][tc];
        tw += sd[q][tc];
      }
      a.grad[(size_t)H * Hh + c] = tb;
      a.grad[(size_t)H * Hh + Hh + c] = tw;
    }
  }
  if (blockIdx.x == 0) {
    double se = 0.0, ae = 0.0;
    float db2 = 0.f;
    for (int g = tid; g < G; g += kRedThreads) {
      const float r = a.pred[g] - a.y[g];
      se += (double)r * (double)r;
      ae += fabs((double)r);
      db2 += a.dpred[g];
    }
    const double sse = block_sum<kRedThreads>(se, redd);
    const double sae = block_sum<kRedThreads>(ae, redd);
    const float sdb2 = block_sum<kRedThreads>(db2, redf);
    if (tid == 0) {
      a.grad[(size_t)H * Hh + 2 * Hh] = sdb2;
      if (a.loss_accum) {
        a.loss_accum[0] += sse;
        a.loss_accum[1] += sae;
        a.loss_accum[2] += (double)G;
      }
    }
  }
}

// ---------------------------------------------------------------- node head
// One warp per atom: pred = ReLU(zn) . w2n + b2n (lanes over the Hh columns,
// fixed-order butterfly), then the loss gradient and dzn.
constexpr int kNodeWarps = 8;

__global__ void __launch_bounds__(kNodeWarps * 32) node_pred_kernel(NodeHeadArgs a, bool train) {
  pdl_entry(GCNN_K_NODE_PRED);
  const int N = min(a.n_cap, a.dims.nodes(a.n_cap));
  const int i = blockIdx.x * kNodeWarps + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (i >= N) return;  // warp-uniform
  const float *z = a.zn + (size_t)i * a.Hh;
  float acc = 0.f;
  for (int c = lane; c < a.Hh; c += 32) acc += fmaxf(z[c], 0.f) * a.w2n[c];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  const float p = acc + a.b2n[0];
  if (lane == 0) a.pred[i] = p;
  if (!train) return;
  const float dp = (a.weight * 2.f * (p - a.y[i]) / (float)N) * (a.loss_scale ? a.loss_scale[0] : 1.f);
  if (lane == 0) a.dpred[i] = dp;
  float *dz = a.dzn + (size_t)i * a.Hh;
  for (int c = lane; c < a.Hh; c += 32) dz[c] = z[c] > 0.f ? dp * a.w2n[c] : 0.f;
}

// w2n for columns blockIdx.x * 32 + lane (atoms strided over the 8 warps, then
// the warps' partials in order); the last block: b2n and the loss sums.
__global__ void __launch_bounds__(kRedThreads) node_grad_kernel(NodeHeadArgs a, float *grad, double *accum) {
  pdl_entry(GCNN_K_NODE_GRAD);
  __shared__ float part[kRedThreads / 32][33];
  __shared__ double redd[kRedThreads / 32];
  __shared__ float redf[kRedThreads / 32];
  const int N = min(a.n_cap, a.dims.nodes(a.n_cap));
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if ((int)blockIdx.x < gridDim.x - 1) {
    const int c = blockIdx.x * 32 + lane;
    float s = 0.f;
    if (c < a.Hh)
      for (int i = w; i < N; i += kRedThreads / 32) s += fmaxf(a.zn[(size_t)i * a.Hh + c], 0.f) * a.dpred[i];
    part[w][lane] = s;
    __syncthreads();
    if (w == 0 && c < a.Hh) {
      float t = part[0][lane];
      for (int q = 1; q < kRedThreads / 32; ++q) t += part[q][lane];
      grad[c] = t;
    }
    return;
  }
  double se = 0.0;
  float db = 0.f;
  for (int i = tid; i < N; i += kRedThreads) {
    const float r = a.pred[i] - a.y[i];
    se += (double)r * (double)r;
    db += a.dpred[i];
  }
  const double sse = block_sum<kRedThreads>(se, redd);
  const float sdb = block_sum<kRedThreads>(db, redf);
  if (tid == 0) {
    grad[a.Hh] = sdb;
    if (accum) {
      accum[3] += sse;
      accum[4] += (double)N;
    }
  }
}

// ---------------------------------------------------------------- AdamW
// Moment decays beta and their complements 1 - beta, each rounded once to
// FP32 from double: 1 - (float)0.999 would carry a 1.3e-5 relative error.
struct AdamBetas {
  float b1, omb1, b2, omb2;
};

__device__ __forceinline__ void adam_one(float &p, float g, float &m, float &v, float lr, float c1,
                                         float c2, const AdamBetas &bt, float eps, float wd) {
  if (wd > 0.f) p -= lr * wd * p;
  m = bt.b1 * m + bt.omb1 * g;
  v = bt.b2 * v + bt.omb2 * (g * g);
  p -= lr * (m * c1) / (sqrtf(v * c2) + eps);
}

// Destination of parameter i (a multiple of 4) in the packed BF16 operands of
// the backward GEMMs, or -1: per layer Wd[n][s*H + c] = W_U[H + blk(s)*5H + n][c]
// (s = 0, 1, 2 for the amplification, attenuation and identity blocks) and
// Wx[n] = [W_U[n][0..H) | W_M[n][0..2H)].
__device__ __forceinline__ long long packed_index(long long i, const AdamPack &k) {
  // 32-bit offsets: a layer's parameters and its packed operands hold < 2^31 elements
  const long long o0l = i - k.layers_begin;
  if (o0l < 0 || o0l >= (long long)k.L * k.layer_size) return -1;
  const unsigned H = (unsigned)k.H, o0 = (unsigned)o0l, ls = (unsigned)k.layer_size;
  const unsigned l = o0 / ls, o = o0 - l * ls;
  const unsigned base = l * 18u * H * H, wx = base + 15u * H * H;
  if (o < 2u * H * H) {  // W_M
    const unsigned r = o / (2u * H);
    return wx + r * 3u * H + H + (o - r * 2u * H);
  }
  if (o < 2u * H * H + H || o >= 18u * H * H + H) return -1;  // biases
  const unsigned u = o - (2u * H * H + H);
  const unsigned r = u / H, c = u - r * H;
  if (r < H) return wx + r * 3u * H + c;
  const unsigned rr = r - H, blk = rr / (5u * H), n = rr - blk * 5u * H;
  return base + n * 3u * H + ((blk + 2u) % 3u) * H + c;
}

// AdamW over two spans of the flat FP32 parameters.  The step counter
// state[0] is read by every block, so the update of step t uses the bias
// corrections of t = state[0] + 1; with `advance` the last block to finish
// (ticket) moves it on.  Optionally writes the BF16 copies of the updated
// parameters (flat and packed).
__global__ void __launch_bounds__(kThreads)
adam_kernel(AdamSpan sp, int advance, float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
            float *__restrict__ v, int *__restrict__ state, unsigned *__restrict__ ticket,
            const float *__restrict__ lrp, AdamBetas bt, float eps, float wd, uint16_t *__restrict__ wb,
            uint16_t *__restrict__ wpack, AdamPack pk) {
  pdl_entry(GCNN_K_ADAM);
  // bias corrections 1 / (1 - beta^t) in FP32 in every thread (an FP64 pow
  // per block costs microseconds on this part's narrow FP64 pipe).  1 - beta^t
  // is formed as -expm1(t log1p(-(1 - beta))) from the complement: the
  // difference of two rounded numbers near 1 is never taken, which with
  // beta2 = 0.999 would cost ~1e-7 / (1 - beta2^t) relative error
  const float t = (float)(state[0] + 1);
  const float c1 = -1.f / expm1f(t * log1pf(-bt.omb1)), c2 = -1.f / expm1f(t * log1pf(-bt.omb2)), lr = lrp[0];
  const int64_t q0 = sp.n0 / 4, n4 = q0 + sp.n1 / 4;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n4; r += stride) {
    const int64_t q = (r < q0 ? sp.b0 + 4 * r : sp.b1 + 4 * (r - q0)) / 4;  // float4 index
    float4 P = ld4(p + 4 * q), Gv = ld4(g + 4 * q), Mv = ld4(m + 4 * q), V = ld4(v + 4 * q);
    adam_one(P.x, Gv.x, Mv.x, V.x, lr, c1, c2, bt, eps, wd);
    adam_one(P.y, Gv.y, Mv.y, V.y, lr, c1, c2, bt, eps, wd);
    adam_one(P.z, Gv.z, Mv.z, V.z, lr, c1, c2, bt, eps, wd);
    adam_one(P.w, Gv.w, Mv.w, V.w, lr, c1, c2, bt, eps, wd);
    st4(p + 4 * q, P);
    st4(m + 4 * q, Mv);
    st4(v + 4 * q, V);
    if (wb) {
      st_bf16x4(wb + 4 * q, P.x, P.y, P.z, P.w);
      const long long d = wpack ? packed_index(4 * q, pk) : -1;
      if (d >= 0) st_bf16x4(wpack + d, P.x, P.y, P.z, P.w);
    }
  }
  if (blockIdx.x == 0 && threadIdx.x < (int)(sp.n1 % 4)) {
    const int64_t k = sp.b1 + sp.n1 / 4 * 4 + threadIdx.x;
    float P = p[k], M = m[k], V = v[k];
    adam_one(P, g[k], M, V, lr, c1, c2, bt, eps, wd);
    p[k] = P; m[k] = M; v[k] = V;
    if (wb) wb[k] = (uint16_t)(bf16x2(P, 0.f) & 0xFFFFu);
  }
  // the last block to finish advances the step counter
  if (!advance) return;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(ticket, 1u) == gridDim.x - 1) {
      state[0] = t;
      *ticket = 0u;
    }
  }
}

// out0[c] = sum_i a0[i][c] [mask[i][c] > 0] for c < cols0 and out1[c] =
// sum_i a1[i][c] for c < cols1 (the bias gradients).  The columns of
// [a0 | a1] go in groups of 32 (blockIdx.x): eight lanes of a warp read one
// row's 128 bytes, so a warp covers four rows per load.  The rows are cut into
// gridDim.y contiguous ranges, one per CTA of a cluster.  Fixed order
// throughout: each thread adds its rows in increasing order, the four rows of
// a warp by butterfly, the warps in index order, and the cluster's CTAs in
// rank order (distributed shared memory), so the sums are bit-reproducible.
// The launch makes the cluster (1, gridDim.y, 1), so a CTA's rank in its
// cluster is blockIdx.y and rank 0 writes the group's sums.
__global__ void __launch_bounds__(kColsumThreads)
colsum_kernel(int n_cap, int cols0, int cols, DevDims dims, const float *__restrict__ a0, int ld0,
              const float *__restrict__ mask, int ldm, const float *__restrict__ a1, int ld1,
              float *__restrict__ out0, float *__restrict__ out1) {
  pdl_entry(GCNN_K_COLSUM);
  constexpr int kWarps = kColsumThreads / 32, kRowsPerPass = kColsumThreads / 8;
  __shared__ float4 sh[kWarps][8];
  __shared__ float4 part[8];
  const int N = min(n_cap, dims.nodes(n_cap));
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, q = lane & 7;
  const int c = blockIdx.x * kColsumWidth + 4 * q;
  const bool first = c < cols0;
  const int seg = (N + (int)gridDim.y - 1) / (int)gridDim.y;
  const int i0 = (int)blockIdx.y * seg, i1 = min(N, i0 + seg);
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  if (c < cols) {
    const float *src = first ? a0 + c : a1 + (c - cols0);
    const int ld = first ? ld0 : ld1;
    const float *mk = first ? mask : nullptr;
    for (int i = i0 + (threadIdx.x >> 3); i < i1; i += 4 * kRowsPerPass) {
      float4 x[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int r = i + u * kRowsPerPass;
        if (r < i1) {
          x[u] = ld4(src + (size_t)r * ld);
          if (mk) {
            const float4 m = ld4(mk + (size_t)r * ldm + c);
            x[u].x = m.x > 0.f ? x[u].x : 0.f;
            x[u].y = m.y > 0.f ? x[u].y : 0.f;
            x[u].z = m.z > 0.f ? x[u].z : 0.f;
            x[u].w = m.w > 0.f ? x[u].w : 0.f;
          }
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (i + u * kRowsPerPass < i1) acc = add4(acc, x[u]);
    }
  }
#pragma unroll
  for (int o = 8; o < 32; o <<= 1) {
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    acc.z += __shfl_xor_sync(0xffffffffu, acc.z, o);
    acc.w += __shfl_xor_sync(0xffffffffu, acc.w, o);
  }
  if (lane < 8) sh[w][lane] = acc;
  __syncthreads();
  if (threadIdx.x < 8) {
    float4 sum = sh[0][threadIdx.x];
#pragma unroll
    for (int k = 1; k < kWarps; ++k) sum = add4(sum, sh[k][threadIdx.x]);
    part[threadIdx.x] = sum;
  }
  colsum_cluster_sync();
  if (blockIdx.y == 0 && threadIdx.x < 8 && c < cols) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(&part[threadIdx.x]);
    float4 sum = colsum_ld_cluster4(a, 0);
    for (int k = 1; k < (int)gridDim.y; ++k) sum = add4(sum, colsum_ld_cluster4(a, k));
    st4(first ? out0 + c : out1 + (c - cols0), sum);
  }
  // no CTA leaves while rank 0 may still read its partial sums
  colsum_cluster_sync();
}

}  // namespace

int launch_colsum2(int n_cap, int cols0, int cols1, DevDims dims, const float *a0, int ld0, const float *mask,
                   int ldm, const float *a1, int ld1, float *out0, float *out1, cudaStream_t s) {
  const int cols = cols0 + cols1;
  if (cols <= 0 || n_cap <= 0) return GCNN_OK;
  if (cols0 % 4 || cols1 % 4 || ld0 % 4 || ld1 % 4 || (mask && ldm % 4))
    return set_error(GCNN_EINVAL, "colsum: widths and strides must be multiples of 4");
  // about one CTA per SM: the column groups times the row ranges of a cluster
  const int groups = (int)ceil_div(cols, kColsumWidth);
  const int ranks = std::max(1, std::min(kColsumMaxRanks, num_sms() / groups));
  cudaLaunchAttribute attr[2];
  int n = 0;
  attr[n].id = cudaLaunchAttributeClusterDimension;
  attr[n].val.clusterDim.x = 1;
  attr[n].val.clusterDim.y = (unsigned)ranks;
  attr[n].val.clusterDim.z = 1;
  ++n;
  if (pdl_enabled(s)) {
    attr[n].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[n].val.programmaticStreamSerializationAllowed = 1;
    ++n;
  }
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)groups, (unsigned)ranks);
  cfg.blockDim = dim3(kColsumThreads);
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = n;
  GCNN_CUDA_TRY(cudaLaunchKernelEx(&cfg, colsum_kernel, n_cap, cols0, cols, dims, a0, ld0, mask, ldm, a1, ld1, out0,
                                   out1));
  return GCNN_OK;
}

int launch_embed(int n_nodes, int H, DevDims dims, const uint8_t *types, const float *emb,
                 int n_types, float *x0, cudaStream_t s, uint16_t *x0_16, int ld16) {
  if (n_nodes <= 0) return GCNN_OK;
  const long long work = (long long)n_nodes * (H / 4);
  GCNN_TRY(launch(embed_kernel, ceil_div(work, kThreads), kThreads, 0, s, n_nodes, H, dims, types, emb, n_types, x0,
                  x0_16, ld16));
  return GCNN_OK;
}

int launch_embed_bwd(int n_nodes, int H, DevDims dims, const uint8_t *types, const float *dx0, int n_types,
                     float *demb, cudaStream_t s) {
  if (n_types > kMaxTypes) return set_error(GCNN_EINVAL, "at most %d atom types", kMaxTypes);
  if (H % 4) return set_error(GCNN_EINVAL, "embedding: hidden must be a multiple of 4");
  GCNN_TRY(launch(embed_bwd_kernel, H / 4, kEmbBwdThreads, 0, s, std::max(n_nodes, 0), H, dims, types, dx0, n_types,
                  demb));
  return GCNN_OK;
}

int launch_pool_fwd(int G, int H, DevDims dims, const int *node_off, const float *x, float *pooled,
                    cudaStream_t s) {
  if (G <= 0) return GCNN_OK;
  const long long work = (long long)G * (H / 4);
  GCNN_TRY(launch(pool_fwd_kernel, ceil_div(work, kThreads), kThreads, 0, s, G, H, dims, node_off, x, pooled));
  return GCNN_OK;
}

int launch_pool_bwd(int G, int n_nodes, int H, DevDims dims, const int *node_off,
                    const int *graph_id, const float *dpooled, float *dx, cudaStream_t s, uint16_t *D3,
                    int ld3, const float *h, const float *amp, const float *att) {
  (void)G;
  if (n_nodes <= 0) return GCNN_OK;
  const long long work = (long long)n_nodes * (H / 4);
  GCNN_TRY(launch(pool_bwd_kernel, ceil_div(work, kThreads), kThreads, 0, s, n_nodes, H, dims, node_off, graph_id,
                  dpooled, dx, D3, ld3, h, amp, att));
  return GCNN_OK;
}

namespace {
constexpr int kHeadSmemFloats = 40 * 1024;  // 160 KB: W1 rows plus pooled / z1 / dz1 vectors

template <bool F, bool B>
int head_graph(HeadArgs a, cudaStream_t s) {
  static bool configured = false;
  // the one-chunk forward also keeps kHeadRed float4 partials
  const bool one = a.rk >= a.H && a.Hh % 4 == 0;
  const size_t bytes =
      sizeof(float) * ((size_t)a.rk * a.Hh + a.H + 2 * (size_t)a.Hh) + (one ? sizeof(float4) * kHeadRed : 0);
  if (!configured) {
    GCNN_CUDA_TRY(cudaFuncSetAttribute(head_graph_kernel<F, B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(sizeof(float) * kHeadSmemFloats + sizeof(float4) * kHeadRed)));
    configured = true;
  }
  GCNN_TRY(launch(head_graph_kernel<F, B>, a.g_cap, kHeadThreads, bytes, s, a));
  return GCNN_OK;
}
}  // namespace

int launch_head_graph(HeadArgs a, bool fwd, bool bwd, cudaStream_t s) {
  if (a.g_cap <= 0 || (!fwd && !bwd)) return GCNN_OK;
  if (a.H % 4 || a.H <= 0 || a.Hh <= 0) return set_error(GCNN_EINVAL, "head: hidden must be a positive multiple of 4");
  const long long room = kHeadSmemFloats - a.H - 2LL * a.Hh;
  long long rk = std::min<long long>(a.H, room / a.Hh) / 4 * 4;
  if (rk < 4) return set_error(GCNN_EINVAL, "head: layer too wide for shared memory");
  a.rk = (int)rk;
  if (fwd && bwd) return head_graph<true, true>(a, s);
  if (fwd) return head_graph<true, false>(a, s);
  return head_graph<false, true>(a, s);
}

int launch_head_grad(const HeadGradArgs &a, cudaStream_t s) {
  if (a.g_cap <= 0) return GCNN_OK;
  dim3 grid(ceil_div(a.Hh, kHT), ceil_div(a.H, kHT) + 1);
  GCNN_TRY(launch(head_grad_kernel, grid, kRedThreads, 0, s, a));
  return GCNN_OK;
}

int launch_node_pred(const NodeHeadArgs &a, bool train, cudaStream_t s) {
  if (a.n_cap <= 0) return GCNN_OK;
  GCNN_TRY(launch(node_pred_kernel, ceil_div(a.n_cap, kNodeWarps), kNodeWarps * 32, 0, s, a, train));
  return GCNN_OK;
}

int launch_node_grad(const NodeHeadArgs &a, float *grad_w2n, double *loss_accum, cudaStream_t s) {
  if (a.n_cap <= 0) return GCNN_OK;
  GCNN_TRY(launch(node_grad_kernel, ceil_div(a.Hh, 32) + 1, kRedThreads, 0, s, a, grad_w2n, loss_accum));
  return GCNN_OK;
}

int launch_adam(AdamSpan span, bool advance, int max_blocks, float *param, const float *grad, float *m, float *v,
                int *state, unsigned *ticket, const float *lr, double beta1, double beta2, float eps, float wd,
                uint16_t *wb, uint16_t *wpack, AdamPack pk, cudaStream_t s) {
  if (span.b0 % 4 || span.n0 % 4 || span.b1 % 4 || span.n0 < 0 || span.n1 < 0)
    return set_error(GCNN_EINVAL, "adam: spans must start and the first must end on multiples of 4");
  if (span.n0 + span.n1 <= 0) return GCNN_OK;
  const int64_t cap = max_blocks > 0 ? max_blocks : (int64_t)num_sms() * 8;
  const int blocks = (int)std::min<int64_t>(((span.n0 + span.n1) / 4 + kThreads - 1) / kThreads + 1, cap);
  const AdamBetas bt{(float)beta1, (float)(1.0 - beta1), (float)beta2, (float)(1.0 - beta2)};
  GCNN_TRY(launch(adam_kernel, blocks, kThreads, 0, s, span, advance ? 1 : 0, param, grad, m, v, state, ticket, lr,
                  bt, eps, wd, wb, wpack, pk));
  return GCNN_OK;
}

namespace {
// FP32 FFMA throughput probe: 8 independent fused multiply-add chains per
// thread (x = x * b + c), unrolled 16 deep; the sum is stored only under a
// never-true condition so that the chains stay live.
__global__ void __launch_bounds__(256) ffma_peak_kernel(int iters, float b, float c, float *out) {
  float x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = 1e-3f * (float)threadIdx.x + (float)k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int k = 0; k < 8; ++k) x[k] = fmaf(x[k], b, c);
  }
  float sum = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) sum += x[k];
  if (sum == -1.f) out[blockIdx.x] = sum;
}
}  // namespace

namespace {
__global__ void step_end_kernel() { pdl_entry(GCNN_K_STEP_END); }
}  // namespace

int launch_step_end(cudaStream_t s) {
  GCNN_TRY(launch(step_end_kernel, 1, 32, 0, s));
  return GCNN_OK;
}

int launch_ffma_peak(int iters, float *out, cudaStream_t s, double *flop) {
  const int blocks = num_sms() * 8;
  ffma_peak_kernel<<<blocks, 256, 0, s>>>(iters, 1.0000001f, 1e-7f, out);
  GCNN_LAUNCH_CHECK();
  *flop = 2.0 * 8 * 16 * (double)iters * blocks * 256;
  return GCNN_OK;
}

GCNN_TIMELINE_ATTACH(small)

}  // namespace gcnn
