// FP32 GEMM on the CUDA cores (FFMA): the dense node-wise linear layers of
// the PNA convolution (message layer W_M, update layer W_U) and their weight
// and input gradients, for the full-FP32 path.
//
// Operands are "virtual": each is assembled while it is staged into shared
// memory from up to kMaxSeg segments along the feature dimension, each with an
// optional per-node scale (the degree scalers) and an optional ReLU mask (the
// backward of the update's ReLU).  So [x ; agg ; amp*agg ; att*agg] (16H
// wide) is never materialised, and a "ones" segment appends a row that
// yields bias gradients as column sums inside the weight-gradient GEMM.
//
// Tiling: 128 x 128 x 8 block tile, 256 threads, 8 x 8 outputs per thread,
// register-staged double buffering of the shared-memory tiles.  Split-K
// writes per-split partial tiles that a second kernel sums in split order
// (deterministic) and finishes with bias / ReLU.
#include <algorithm>

#include "kernels.cuh"

namespace gcnn {
namespace {

constexpr int BM = 128, BN = 128, BK = 8, kThreads = 256;

__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }

struct Sizes {
  int M, K;
};

__device__ __forceinline__ Sizes actual_sizes(const GemmDesc &d, DevDims dims) {
  Sizes s{d.M, d.K};
  if (d.node_dim == kNodeM) s.M = min(d.M, dims.nodes(d.M));
  if (d.node_dim == kNodeK) s.K = min(d.K, dims.nodes(d.K));
  return s;
}

__device__ __forceinline__ int find_seg(const Operand &op, int f) {
  int s = 0;
#pragma unroll
  for (int q = 1; q < kMaxSeg; ++q)
    if (q < op.nseg && op.seg[q].begin <= f) s = q;
  return s;
}

__device__ __forceinline__ float4 apply_mask(float4 v, const float *mask) {
  const float4 mk = ld4(mask);
  v.x = mk.x > 0.f ? v.x : 0.f;
  v.y = mk.y > 0.f ? v.y : 0.f;
  v.z = mk.z > 0.f ? v.z : 0.f;
  v.w = mk.w > 0.f ? v.w : 0.f;
  return v;
}

// Four consecutive features f..f+3 of node `node` (row-major node x feature source).
__device__ __forceinline__ float4 load_feat4(const Seg &sg, int node, int f) {
  float4 v;
  if (sg.ptr) {
    const size_t off = (size_t)node * sg.ld + (f - sg.begin);
    v = ld4(sg.ptr + off);
    if (sg.mask) v = apply_mask(v, sg.mask + off);
  } else {
    v = make_float4(1.f, 1.f, 1.f, 1.f);
  }
  if (sg.rowscale) {
    const float r = sg.rowscale[node];
    v.x *= r; v.y *= r; v.z *= r; v.w *= r;
  }
  return v;
}

__device__ __forceinline__ float load_feat1(const Seg &sg, int node, int f) {
  float v = 1.f;
  if (sg.ptr) {
    const size_t off = (size_t)node * sg.ld + (f - sg.begin);
    v = sg.ptr[off];
    if (sg.mask && !(sg.mask[off] > 0.f)) v = 0.f;
  }
  if (sg.rowscale) v *= sg.rowscale[node];
  return v;
}

template <bool AK, bool BNC>
__global__ void __launch_bounds__(kThreads, 2)
sgemm_kernel(GemmDesc d, DevDims dims, float *__restrict__ partial, int splits, int kps) {
  pdl_entry(GCNN_K_GEMM_SIMT);
  __shared__ __align__(16) float As[2][BK][BM];
  __shared__ __align__(16) float Bs[2][BK][BN];
  const Sizes sz = actual_sizes(d, dims);
  const int M = sz.M, K = sz.K, N = d.N;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int z = blockIdx.z;
  if (m0 >= M) return;  // block-uniform
  const int kbeg = z * kps;
  const int kend = min(K, kbeg + kps);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;

  float4 ra, rb;
  // ---- global -> registers
  auto load_a = [&](int k0) {
    if (AK) {  // A(m,k) = ptr[m*ld + k - begin]; thread: row tid>>1, 4 k's at (tid&1)*4
      const int r = tid >> 1, kq = (tid & 1) * 4;
      const int m = m0 + r, k = k0 + kq;
      ra = make_float4(0.f, 0.f, 0.f, 0.f);
      if (m < M && k < kend) ra = load_feat4(d.A.seg[find_seg(d.A, k)], m, k);
    } else {   // A(m,k) = ptr[k*ld + m - begin]; thread: k tid>>5, 4 m's at (tid&31)*4
      const int kk = tid >> 5, mq = (tid & 31) * 4;
      const int m = m0 + mq, k = k0 + kk;
      ra = make_float4(0.f, 0.f, 0.f, 0.f);
      if (k < kend && m < M) {
        const int s0 = find_seg(d.A, m);
        if (m + 3 < M && find_seg(d.A, m + 3) == s0) {
          ra = load_feat4(d.A.seg[s0], k, m);
        } else {
          float t[4];
#pragma unroll
          for (int q = 0; q < 4; ++q)
            t[q] = (m + q < M) ? load_feat1(d.A.seg[find_seg(d.A, m + q)], k, m + q) : 0.f;
          ra = make_float4(t[0], t[1], t[2], t[3]);
        }
      }
    }
  };
  auto load_b = [&](int k0) {
    if (BNC) {  // B(k,n) = ptr[(k-begin)*ld + n]; thread: k tid>>5, 4 n's at (tid&31)*4
      const int kk = tid >> 5, nq = (tid & 31) * 4;
      const int k = k0 + kk, n = n0 + nq;
      rb = make_float4(0.f, 0.f, 0.f, 0.f);
      if (k < kend && n < N) {
        const Seg &sg = d.B.seg[find_seg(d.B, k)];
        const size_t off = (size_t)(k - sg.begin) * sg.ld + n;
        rb = ld4(sg.ptr + off);
        if (sg.mask) rb = apply_mask(rb, sg.mask + off);
        if (sg.rowscale) {
          const float r = sg.rowscale[k - sg.begin];
          rb.x *= r; rb.y *= r; rb.z *= r; rb.w *= r;
        }
      }
    } else {    // B(k,n) = ptr[n*ld + k - begin]; thread: n tid>>1, 4 k's at (tid&1)*4
      const int r = tid >> 1, kq = (tid & 1) * 4;
      const int n = n0 + r, k = k0 + kq;
      rb = make_float4(0.f, 0.f, 0.f, 0.f);
      if (n < N && k < kend) {
        const Seg &sg = d.B.seg[find_seg(d.B, k)];
        rb = ld4(sg.ptr + (size_t)n * sg.ld + (k - sg.begin));
      }
    }
  };
  // ---- registers -> shared
  auto store_ab = [&](int buf) {
    if (AK) {
      const int r = tid >> 1, kq = (tid & 1) * 4;
      As[buf][kq + 0][r] = ra.x; As[buf][kq + 1][r] = ra.y;
      As[buf][kq + 2][r] = ra.z; As[buf][kq + 3][r] = ra.w;
    } else {
      *reinterpret_cast<float4 *>(&As[buf][tid >> 5][(tid & 31) * 4]) = ra;
    }
    if (BNC) {
      *reinterpret_cast<float4 *>(&Bs[buf][tid >> 5][(tid & 31) * 4]) = rb;
    } else {
      const int r = tid >> 1, kq = (tid & 1) * 4;
      Bs[buf][kq + 0][r] = rb.x; Bs[buf][kq + 1][r] = rb.y;
      Bs[buf][kq + 2][r] = rb.z; Bs[buf][kq + 3][r] = rb.w;
    }
  };

  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

  if (kbeg < kend) {
    load_a(kbeg);
    load_b(kbeg);
    store_ab(0);
    __syncthreads();
    int buf = 0;
    for (int k0 = kbeg; k0 < kend; k0 += BK) {
      const bool more = k0 + BK < kend;
      if (more) { load_a(k0 + BK); load_b(k0 + BK); }
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        const float4 a0 = *reinterpret_cast<const float4 *>(&As[buf][kk][ty * 4]);
        const float4 a1 = *reinterpret_cast<const float4 *>(&As[buf][kk][64 + ty * 4]);
        const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[buf][kk][tx * 4]);
        const float4 b1 = *reinterpret_cast<const float4 *>(&Bs[buf][kk][64 + tx * 4]);
        const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
      }
      if (more) store_ab(buf ^ 1);
      __syncthreads();
      buf ^= 1;
    }
  }

  // ---- epilogue
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int m = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
    if (m >= M) continue;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int n = n0 + h * 64 + tx * 4;
      if (n >= N) continue;
      float4 v = make_float4(acc[i][h * 4 + 0], acc[i][h * 4 + 1], acc[i][h * 4 + 2], acc[i][h * 4 + 3]);
      if (splits > 1) {
        *reinterpret_cast<float4 *>(partial + ((size_t)z * d.M + m) * N + n) = v;
        continue;
      }
      if (d.bias) {
        v.x += (n + 0 < d.bias_n) ? d.bias[n + 0] : 0.f;
        v.y += (n + 1 < d.bias_n) ? d.bias[n + 1] : 0.f;
        v.z += (n + 2 < d.bias_n) ? d.bias[n + 2] : 0.f;
        v.w += (n + 3 < d.bias_n) ? d.bias[n + 3] : 0.f;
      }
      if (d.relu) {
        v.x = fmaxf(v.x, 0.f); v.y = fmaxf(v.y, 0.f); v.z = fmaxf(v.z, 0.f); v.w = fmaxf(v.w, 0.f);
      }
      float *c = d.C + (size_t)m * d.ldc + n;
      if (d.last_row_cols > 0 && m == M - 1) {
        const float t[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (n + q < d.last_row_cols) c[q] = t[q];
      } else {
        *reinterpret_cast<float4 *>(c) = v;
      }
    }
  }
}

// C = epilogue(sum_z partial[z]); one thread per 4 outputs
__global__ void __launch_bounds__(kThreads)
splitk_reduce_kernel(GemmDesc d, DevDims dims, const float *__restrict__ partial, int splits) {
  pdl_entry(GCNN_K_GEMM_SIMT_REDUCE);
  const Sizes sz = actual_sizes(d, dims);
  const int M = sz.M, N = d.N, N4 = N / 4;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)M * N4) return;
  const int m = (int)(t / N4), n = (int)(t % N4) * 4;
  float4 v = ld4(partial + (size_t)m * N + n);
  for (int z = 1; z < splits; ++z) {
    const float4 p = ld4(partial + ((size_t)z * d.M + m) * N + n);
    v.x += p.x; v.y += p.y; v.z += p.z; v.w += p.w;
  }
  if (d.bias) {
    v.x += (n + 0 < d.bias_n) ? d.bias[n + 0] : 0.f;
    v.y += (n + 1 < d.bias_n) ? d.bias[n + 1] : 0.f;
    v.z += (n + 2 < d.bias_n) ? d.bias[n + 2] : 0.f;
    v.w += (n + 3 < d.bias_n) ? d.bias[n + 3] : 0.f;
  }
  if (d.relu) {
    v.x = fmaxf(v.x, 0.f); v.y = fmaxf(v.y, 0.f); v.z = fmaxf(v.z, 0.f); v.w = fmaxf(v.w, 0.f);
  }
  float *c = d.C + (size_t)m * d.ldc + n;
  if (d.last_row_cols > 0 && m == M - 1) {
    const float tt[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (n + q < d.last_row_cols) c[q] = tt[q];
  } else {
    *reinterpret_cast<float4 *>(c) = v;
  }
}

int g_num_sms = 0;

}  // namespace

int num_sms() {
  if (g_num_sms == 0) {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && n > 0)
      g_num_sms = n;
    else
      g_num_sms = 148;
  }
  return g_num_sms;
}

namespace {

int choose_splits(int M, int N, int K) {
  const long long tiles = (long long)ceil_div(M, BM) * ceil_div(N, BN);
  const int ktiles = (int)ceil_div(K, BK);
  const long long target = 2LL * num_sms();
  int s = (int)std::max<long long>(1, (target + tiles - 1) / tiles);
  s = std::min(s, std::max(1, ktiles / 8));  // at least 8 k-tiles per split
  return std::min(s, 32);
}

bool operand_ok(const Operand &op, bool vec_along_feature) {
  if (op.nseg < 1 || op.nseg > kMaxSeg || op.seg[0].begin != 0) return false;
  for (int q = 0; q < op.nseg; ++q) {
    const Seg &s = op.seg[q];
    if (s.begin % 4) return false;
    if (q > 0 && s.begin <= op.seg[q - 1].begin) return false;
    if (s.ptr && (s.ld % 4 || reinterpret_cast<uintptr_t>(s.ptr) % 16)) return false;
    if (s.mask && (!s.ptr || reinterpret_cast<uintptr_t>(s.mask) % 16)) return false;
  }
  (void)vec_along_feature;
  return true;
}

}  // namespace

size_t gemm_simt_workspace_floats(int M, int N, int K) {
  const int s = choose_splits(M, N, K);
  return s > 1 ? (size_t)s * M * N : 0;
}

int run_gemm_simt(const GemmDesc &d, DevDims dims, const GemmWorkspace &ws, cudaStream_t s) {
  if (d.M <= 0 || d.N <= 0 || d.K < 0) return GCNN_OK;
  if (d.N % 4 || d.ldc % 4 || reinterpret_cast<uintptr_t>(d.C) % 16)
    return set_error(GCNN_EINVAL, "gemm: N, ldc must be multiples of 4 and C 16-byte aligned");
  if (d.a_kcontig && d.K % 4) return set_error(GCNN_EINVAL, "gemm: K must be a multiple of 4");
  if (!d.b_ncontig && d.K % 4) return set_error(GCNN_EINVAL, "gemm: K must be a multiple of 4");
  if (!operand_ok(d.A, true) || !operand_ok(d.B, true))
    return set_error(GCNN_EINVAL, "gemm: bad operand segments (alignment / order)");
  for (int q = 0; q < d.B.nseg; ++q)
    if (!d.B.seg[q].ptr) return set_error(GCNN_EINVAL, "gemm: B segments need data");
  int splits = std::min(choose_splits(d.M, d.N, d.K), ws.max_splits);
  if (splits > 1 && (size_t)splits * d.M * d.N > ws.floats) splits = 1;
  int kps = (int)(ceil_div(d.K, (long long)splits * BK) * BK);
  if (kps == 0) kps = BK;
  dim3 grid(ceil_div(d.N, BN), ceil_div(d.M, BM), splits);
  float *part = splits > 1 ? ws.partial : nullptr;
  if (d.a_kcontig && d.b_ncontig)
    GCNN_TRY(launch(sgemm_kernel<true, true>, grid, kThreads, 0, s, d, dims, part, splits, kps));
  else if (d.a_kcontig && !d.b_ncontig)
    GCNN_TRY(launch(sgemm_kernel<true, false>, grid, kThreads, 0, s, d, dims, part, splits, kps));
  else if (!d.a_kcontig && d.b_ncontig)
    GCNN_TRY(launch(sgemm_kernel<false, true>, grid, kThreads, 0, s, d, dims, part, splits, kps));
  else
    GCNN_TRY(launch(sgemm_kernel<false, false>, grid, kThreads, 0, s, d, dims, part, splits, kps));
  if (splits > 1) GCNN_TRY(run_splitk_reduce(d, dims, part, splits, s));
  return GCNN_OK;
}

int run_splitk_reduce(const GemmDesc &d, DevDims dims, const float *partial, int splits, cudaStream_t s) {
  const long long work = (long long)d.M * (d.N / 4);
  GCNN_TRY(launch(splitk_reduce_kernel, ceil_div(work, kThreads), kThreads, 0, s, d, dims, partial, splits));
  return GCNN_OK;
}

GCNN_TIMELINE_ATTACH(gemm_simt)

}  // namespace gcnn
