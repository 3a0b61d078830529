// BF16 GEMM on the Blackwell tensor cores (tcgen05, FP32 accumulator in TMEM)
// for the dense node-wise layers of the PNA convolution and their gradients.
//
// Operands are BF16 arrays written by the kernels that produce them (the
// embedding, the update GEMM's epilogue, the aggregation kernels, the weight
// cast after each optimizer step), possibly several along K ("segments", e.g.
// [x | scaled aggregates]) or along M (the weight-gradient GEMMs append a row
// of ones whose product is the bias gradient).  Staging is a pure copy:
// 16-byte cp.async chunks into a 4-stage ring of 128-byte-swizzled shared-
// memory tiles, K-major when the source is contiguous along K and MN-major
// when it is contiguous along M / N (the weight-gradient GEMMs reduce over
// nodes, and activations are stored node-major).
//
// Per CTA: one 128 x BN output tile (BN <= 256, a multiple of 16), K in steps
// of 64.  One thread issues four tcgen05.mma (M = 128, N = BN, K = 16) per
// stage and commits them to the stage's mbarrier; the stage is refilled only
// after that barrier fires.  The epilogue reads TMEM (tcgen05.ld) and applies
// bias / ReLU, writing FP32 and optional BF16 side outputs, or split-K partials
// that a second kernel sums in split order.  Every wait is bounded: on expiry
// the kernel sets kErrTimeout in the device error word and skips its epilogue.
#include <algorithm>

#include "kernels.cuh"

namespace gcnn {
namespace {

constexpr int BM = 128, BK = 64, STAGES = 4, kThreads = 256;
constexpr int kMaxBN = 256;
constexpr int kATileBytes = BM * BK * 2;        // 16 KB
constexpr int kBTileBytes = kMaxBN * BK * 2;    // 32 KB
constexpr int kStageBytes = kATileBytes + kBTileBytes;
constexpr int kSmemBytes = STAGES * kStageBytes + 1024 /* alignment slack */ + 256 /* barriers */;
constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz
constexpr uint32_t kMnAtomBytes = 64 * 128;      // one 64-wide MN atom over 64 K rows

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}

// ---------------------------------------------------------------- cp.async
__device__ __forceinline__ void cp16(uint32_t dst, const void *src, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// ---------------------------------------------------------------- mbarrier
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase with the given parity; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > kWaitCycles) return false;
  }
  return true;
}

// ---------------------------------------------------------------- tcgen05
__device__ __forceinline__ void tmem_alloc(uint32_t *dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_free(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor, 128-byte swizzle.  K-major tiles: 8-row
// groups 1024 bytes apart (stride byte offset), leading offset unused.
// MN-major tiles: 64-element MN atoms kMnAtomBytes apart (leading byte
// offset), 8-row K groups 1024 bytes apart (stride byte offset).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, bool mn_major) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(mn_major ? (kMnAtomBytes >> 4) : 1u) << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version (sm_100 family)
  d |= (uint64_t)2 << 61;  // 128-byte swizzle
  return d;
}

// Instruction descriptor, kind::f16: BF16 A and B, FP32 D.
__device__ __forceinline__ uint32_t instr_desc(int M, int N, bool a_mn, bool b_mn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((a_mn ? 1u : 0u) << 15) | ((b_mn ? 1u : 0u) << 16) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

// 32 lanes x 8 consecutive 32-bit columns; thread t receives lane (base + t).
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float v[8]) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int q = 0; q < 8; ++q) v[q] = __uint_as_float(r[q]);
}

// ---------------------------------------------------------------- staging
struct Sizes {
  int M, K;
};

__device__ __forceinline__ Sizes actual_sizes(const TcDesc &d, DevDims dims) {
  Sizes s{d.M, d.K};
  if (d.node_dim == kNodeM) s.M = min(d.M, dims.nodes(d.M));
  if (d.node_dim == kNodeK) s.K = min(d.K, dims.nodes(d.K));
  return s;
}

__device__ __forceinline__ int find_seg(const TcOperand &op, int f) {
  int s = 0;
#pragma unroll
  for (int q = 1; q < kMaxSeg; ++q)
    if (q < op.nseg && op.seg[q].begin <= f) s = q;
  return s;
}

// byte offset of 16-byte chunk (row r, chunk c) in a K-major swizzled tile
__device__ __forceinline__ uint32_t kmaj_off(int r, int c) { return (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4)); }
// byte offset of the chunk holding MN elements mn..mn+7 of K row kk in an MN-major tile
__device__ __forceinline__ uint32_t mnmaj_off(int mn, int kk) {
  return (uint32_t)((mn >> 6) * kMnAtomBytes + kk * 128 + ((((mn & 63) >> 3) ^ (kk & 7)) << 4));
}

// One 16-byte chunk of a "ones" segment: element i is 1 where mn + i == mn_one and valid.
__device__ __forceinline__ void st_ones(uint8_t *dst, int mn, int M, bool kvalid) {
  uint32_t w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
  for (int i = 0; i < 8; ++i)
    if (kvalid && mn + i < M) w[i >> 1] |= (i & 1) ? 0x3F800000u : 0x3F80u;
  *reinterpret_cast<uint4 *>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
}

// A tile (128 x 64) of k-tile k0 -> smem
__device__ __forceinline__ void stage_a(const TcDesc &d, int M, int K, int m0, int k0, uint8_t *tile) {
  const int tid = threadIdx.x;
  const uint32_t base = smem_u32(tile);
  if (!d.A.mn_major) {  // A(m,k) = ptr[m*ld + k - begin]
#pragma unroll
    for (int i = 0; i < (BM * 8) / kThreads; ++i) {
      const int q = tid + i * kThreads;
      const int r = q >> 3, c = q & 7;
      const int m = m0 + r, k = k0 + c * 8;
      const bool ok = m < M && k < K;
      const TcSeg &sg = d.A.seg[find_seg(d.A, ok ? k : 0)];
      if (sg.ptr) cp16(base + kmaj_off(r, c), ok ? sg.ptr + (size_t)m * sg.ld + (k - sg.begin) : sg.ptr, ok);
      else st_ones(tile + kmaj_off(r, c), 0, 8, ok);
    }
  } else {  // A(m,k) = ptr[k*ld + m - begin]; consecutive threads walk m
#pragma unroll
    for (int i = 0; i < (BM * 8) / kThreads; ++i) {
      const int q = tid + i * kThreads;
      const int kk = q >> 4, c = q & 15;
      const int ml = c * 8, m = m0 + ml, k = k0 + kk;
      const bool ok = m < M && k < K;
      const TcSeg &sg = d.A.seg[find_seg(d.A, ok ? m : 0)];
      const uint32_t off = mnmaj_off(ml, kk);
      if (sg.ptr) cp16(base + off, ok ? sg.ptr + (size_t)k * sg.ld + (m - sg.begin) : sg.ptr, ok);
      else st_ones(tile + off, m, M, k < K);
    }
  }
}

// B tile (BN x 64; row n = output column) of k-tile k0 -> smem
__device__ __forceinline__ void stage_b(const TcDesc &d, int N, int K, int BN, int n0, int k0, uint8_t *tile) {
  const int tid = threadIdx.x;
  const uint32_t base = smem_u32(tile);
  const int chunks = BN * 8;
  if (!d.B.mn_major) {  // B(k,n) = ptr[n*ld + k - begin]
    for (int q = tid; q < chunks; q += kThreads) {
      const int r = q >> 3, c = q & 7;
      const int n = n0 + r, k = k0 + c * 8;
      const bool ok = n < N && k < K;
      const TcSeg &sg = d.B.seg[find_seg(d.B, ok ? k : 0)];
      cp16(base + kmaj_off(r, c), ok ? sg.ptr + (size_t)n * sg.ld + (k - sg.begin) : sg.ptr, ok);
    }
  } else {  // B(k,n) = ptr[(k-begin)*ld + n]; consecutive threads walk n
    const int cpr = BN >> 3;  // chunks per K row
    for (int q = tid; q < chunks; q += kThreads) {
      const int kk = q / cpr, c = q - kk * cpr;
      const int nl = c * 8, n = n0 + nl, k = k0 + kk;
      const bool ok = n < N && k < K;
      const TcSeg &sg = d.B.seg[find_seg(d.B, ok ? k : 0)];
      cp16(base + mnmaj_off(nl, kk), ok ? sg.ptr + (size_t)(k - sg.begin) * sg.ld + n : sg.ptr, ok);
    }
  }
}

// ---------------------------------------------------------------- epilogue
// Final value v (bias and ReLU applied) of C(row, n..n+7) to every output.
__device__ __forceinline__ void emit8(const TcEpilogue &e, int M, int N, int row, int n, const float v[8]) {
  const int lim = (e.last_row_cols > 0 && row == M - 1) ? min(N, e.last_row_cols) : N;
  if (e.C) {
    float *c = e.C + (size_t)row * e.ldc + n;
    if (n + 8 <= lim) {
      *reinterpret_cast<float4 *>(c) = make_float4(v[0], v[1], v[2], v[3]);
      *reinterpret_cast<float4 *>(c + 4) = make_float4(v[4], v[5], v[6], v[7]);
    } else {
      for (int q = 0; q < 8 && n + q < lim; ++q) c[q] = v[q];
    }
  }
  if (e.C16 && n + 8 <= N) {
    *reinterpret_cast<uint4 *>(e.C16 + (size_t)row * e.ld16 + n) =
        make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]), pack_bf16(v[6], v[7]));
  }
  if (e.D3 && n + 8 <= N) {  // [v * [mask > 0], amp * (...), att * (...)]
    float g[8];
    const float *mk = e.mask + (size_t)row * e.ldm + n;
#pragma unroll
    for (int q = 0; q < 8; ++q) g[q] = mk[q] > 0.f ? v[q] : 0.f;
    const float a = e.amp[row], t = e.att[row];
    uint16_t *o = e.D3 + (size_t)row * e.ld3 + n;
    *reinterpret_cast<uint4 *>(o) =
        make_uint4(pack_bf16(g[0], g[1]), pack_bf16(g[2], g[3]), pack_bf16(g[4], g[5]), pack_bf16(g[6], g[7]));
    *reinterpret_cast<uint4 *>(o + N) = make_uint4(pack_bf16(a * g[0], a * g[1]), pack_bf16(a * g[2], a * g[3]),
                                                   pack_bf16(a * g[4], a * g[5]), pack_bf16(a * g[6], a * g[7]));
    *reinterpret_cast<uint4 *>(o + 2 * N) = make_uint4(pack_bf16(t * g[0], t * g[1]), pack_bf16(t * g[2], t * g[3]),
                                                       pack_bf16(t * g[4], t * g[5]), pack_bf16(t * g[6], t * g[7]));
  }
}

__device__ __forceinline__ void finish8(const TcEpilogue &e, int n, float v[8]) {
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    if (e.bias && n + q < e.bias_n) v[q] += e.bias[n + q];
    if (e.relu) v[q] = fmaxf(v[q], 0.f);
  }
}

__global__ void __launch_bounds__(kThreads, 1)
tc_gemm_kernel(TcDesc d, DevDims dims, float *__restrict__ partial, int splits, int kps, int BN, unsigned *err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + STAGES * kStageBytes);
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + STAGES);

  const Sizes sz = actual_sizes(d, dims);
  const int M = sz.M, K = sz.K, N = d.N;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int z = blockIdx.z;
  if (m0 >= M) return;  // block-uniform, before any barrier or TMEM use
  const int kbeg = z * kps;
  const int kend = min(K, kbeg + kps);
  const int nk = kend > kbeg ? (kend - kbeg + BK - 1) / BK : 0;
  const int tid = threadIdx.x, warp = tid >> 5;
  const uint32_t ncols = BN <= 32 ? 32 : (BN <= 64 ? 64 : (BN <= 128 ? 128 : 256));

  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) mbar_init(&bars[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(tmem_slot, ncols);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  const uint32_t idesc = instr_desc(BM, BN, d.A.mn_major, d.B.mn_major);
  const uint32_t a_step = d.A.mn_major ? 2048u : 32u;  // bytes per K = 16 slice
  const uint32_t b_step = d.B.mn_major ? 2048u : 32u;

  auto load_stage = [&](int kt) {
    uint8_t *a_tile = smem + (kt % STAGES) * kStageBytes;
    const int k0 = kbeg + kt * BK;
    stage_a(d, M, kend, m0, k0, a_tile);
    stage_b(d, N, kend, BN, n0, k0, a_tile + kATileBytes);
  };

  // prologue: stages 0 .. STAGES-2 in flight
#pragma unroll
  for (int p = 0; p < STAGES - 1; ++p) {
    if (p < nk) load_stage(p);
    cp_commit();
  }
  bool ok = true;
  for (int kt = 0; kt < nk; ++kt) {
    cp_wait<STAGES - 2>();  // this thread's copies of stage kt have landed
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      fence_after_sync();
      const uint32_t a_base = smem_u32(smem + (kt % STAGES) * kStageBytes);
      const uint32_t b_base = a_base + kATileBytes;
#pragma unroll
      for (int j = 0; j < BK / 16; ++j)
        mma_bf16(tmem, smem_desc(a_base + j * a_step, d.A.mn_major), smem_desc(b_base + j * b_step, d.B.mn_major),
                 idesc, (kt > 0 || j > 0) ? 1u : 0u);
      mma_commit(&bars[kt % STAGES]);
    }
    // refill the slot of k-tile kt-1 with k-tile kt+STAGES-1 once its MMAs are done
    const int nxt = kt + STAGES - 1;
    bool expired = false;
    if (nxt < nk && kt >= 1) expired = !mbar_wait(&bars[(kt - 1) % STAGES], ((kt - 1) / STAGES) & 1);
    if (__syncthreads_or(expired)) {  // block-uniform exit
      ok = false;
      break;
    }
    if (nxt < nk) load_stage(nxt);
    cp_commit();
  }
  cp_wait<0>();
  bool expired = false;
  if (nk > 0 && ok) {
    const int last = nk - 1;
    expired = !mbar_wait(&bars[last % STAGES], (last / STAGES) & 1);
  }
  if (__syncthreads_or(expired)) ok = false;
  fence_after_sync();

  if (ok) {
    const int lane_base = 32 * (warp & 3);
    const int row = m0 + lane_base + (tid & 31);
    const int ch = (BN / 8 + 1) / 2;
    const int g0 = warp < 4 ? 0 : ch, g1 = warp < 4 ? ch : BN / 8;
    for (int gq = g0; gq < g1; ++gq) {
      float v[8];
      if (nk > 0) {
        tmem_ld8(tmem + ((uint32_t)lane_base << 16) + (uint32_t)(gq * 8), v);
      } else {
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = 0.f;
      }
      const int n = n0 + gq * 8;
      if (row >= M || n >= N) continue;
      if (splits > 1) {
        float *p = partial + ((size_t)z * d.M + row) * N + n;
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
        *reinterpret_cast<float4 *>(p + 4) = make_float4(v[4], v[5], v[6], v[7]);
        continue;
      }
      finish8(d.ep, n, v);
      emit8(d.ep, M, N, row, n, v);
    }
  } else if (tid == 0 && err) {
    atomicOr(err, kErrTimeout);
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_free(tmem, ncols);
}

// C = epilogue(sum over splits); one thread per 8 outputs
__global__ void __launch_bounds__(256) tc_reduce_kernel(TcDesc d, DevDims dims, const float *__restrict__ partial,
                                                       int splits) {
  const Sizes sz = actual_sizes(d, dims);
  const int M = sz.M, N = d.N, N8 = N / 8;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)M * N8) return;
  const int row = (int)(t / N8), n = (int)(t % N8) * 8;
  float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int z = 0; z < splits; ++z) {
    const float *p = partial + ((size_t)z * d.M + row) * N + n;
    const float4 a = *reinterpret_cast<const float4 *>(p), b = *reinterpret_cast<const float4 *>(p + 4);
    v[0] += a.x; v[1] += a.y; v[2] += a.z; v[3] += a.w; v[4] += b.x; v[5] += b.y; v[6] += b.z; v[7] += b.w;
  }
  finish8(d.ep, n, v);
  emit8(d.ep, M, N, row, n, v);
}

int g_configured = 0;

int choose(int M, int N, int K, int *BN, int *ntiles, int *splits) {
  *ntiles = (N + kMaxBN - 1) / kMaxBN;
  *BN = ((N + *ntiles - 1) / *ntiles + 15) / 16 * 16;
  const long long tiles = (long long)*ntiles * ((M + BM - 1) / BM);
  const int ktiles = (K + BK - 1) / BK;
  // one wave (one 197 KB CTA per SM), at least 4 k-tiles per split
  int s = (int)std::max<long long>(1, num_sms() / tiles);
  s = std::min(s, std::max(1, ktiles / 4));
  *splits = std::min(s, 32);
  return ktiles;
}

bool seg_ok(const TcOperand &op) {
  if (op.nseg < 1 || op.nseg > kMaxSeg || op.seg[0].begin != 0) return false;
  for (int q = 0; q < op.nseg; ++q) {
    const TcSeg &sg = op.seg[q];
    if (sg.begin % 8 || (q > 0 && sg.begin <= op.seg[q - 1].begin)) return false;
    if (sg.ptr && (sg.ld % 8 || reinterpret_cast<uintptr_t>(sg.ptr) % 16)) return false;
  }
  return true;
}

}  // namespace

int run_gemm_tc(const TcDesc &d, DevDims dims, const GemmWorkspace &ws, unsigned *err, cudaStream_t s) {
  if (d.M <= 0 || d.N <= 0 || d.K < 0) return GCNN_OK;
  const TcEpilogue &e = d.ep;
  if (d.N % 8 || (e.C && (e.ldc % 4 || reinterpret_cast<uintptr_t>(e.C) % 16)) ||
      (e.C16 && (e.ld16 % 8 || reinterpret_cast<uintptr_t>(e.C16) % 16)) ||
      (e.D3 && (e.ld3 % 8 || reinterpret_cast<uintptr_t>(e.D3) % 16 || !e.mask || !e.amp || !e.att)))
    return set_error(GCNN_EINVAL, "tc gemm: N must be a multiple of 8 and outputs 16-byte aligned");
  if ((!d.A.mn_major || !d.B.mn_major) && d.K % 8) return set_error(GCNN_EINVAL, "tc gemm: K must be a multiple of 8");
  if (!seg_ok(d.A) || !seg_ok(d.B)) return set_error(GCNN_EINVAL, "tc gemm: bad operand segments");
  for (int q = 0; q < d.B.nseg; ++q)
    if (!d.B.seg[q].ptr) return set_error(GCNN_EINVAL, "tc gemm: B segments need data");
  if (!g_configured) {
    GCNN_CUDA_TRY(cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes));
    g_configured = 1;
  }
  int BN, ntiles, splits;
  const int ktiles = choose(d.M, d.N, d.K, &BN, &ntiles, &splits);
  splits = std::min(splits, ws.max_splits);
  if (splits > 1 && (size_t)splits * d.M * d.N > ws.floats) splits = 1;
  const int kps = (ktiles + splits - 1) / splits * BK;
  dim3 grid(ntiles, (d.M + BM - 1) / BM, splits);
  tc_gemm_kernel<<<grid, kThreads, kSmemBytes, s>>>(d, dims, splits > 1 ? ws.partial : nullptr, splits, kps, BN, err);
  GCNN_LAUNCH_CHECK();
  if (splits > 1) {
    const long long work = (long long)d.M * (d.N / 8);
    tc_reduce_kernel<<<ceil_div(work, 256), 256, 0, s>>>(d, dims, ws.partial, splits);
    GCNN_LAUNCH_CHECK();
  }
  return GCNN_OK;
}

size_t gemm_tc_workspace_floats(int M, int N, int K) {
  int BN, ntiles, splits;
  choose(M, N, K, &BN, &ntiles, &splits);
  return splits > 1 ? (size_t)splits * M * N : 0;
}

// ---------------------------------------------------------------- casts
namespace {
__global__ void cast_bf16_kernel(int64_t n, const float *__restrict__ src, uint16_t *__restrict__ dst) {
  const int64_t n8 = n / 8;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n8; q += stride) {
    const float4 a = reinterpret_cast<const float4 *>(src)[2 * q], b = reinterpret_cast<const float4 *>(src)[2 * q + 1];
    reinterpret_cast<uint4 *>(dst)[q] =
        make_uint4(pack_bf16(a.x, a.y), pack_bf16(a.z, a.w), pack_bf16(b.x, b.y), pack_bf16(b.z, b.w));
  }
  if (blockIdx.x == 0 && threadIdx.x < (int)(n - 8 * n8)) {
    const int64_t k = 8 * n8 + threadIdx.x;
    dst[k] = (uint16_t)(pack_bf16(src[k], 0.f) & 0xFFFFu);
  }
}
}  // namespace

int launch_cast_bf16(int64_t n, const float *src, uint16_t *dst, cudaStream_t s) {
  if (n <= 0) return GCNN_OK;
  if (reinterpret_cast<uintptr_t>(src) % 16 || reinterpret_cast<uintptr_t>(dst) % 16)
    return set_error(GCNN_EINVAL, "cast: buffers must be 16-byte aligned");
  const int blocks = (int)std::min<int64_t>((n / 8 + 255) / 256 + 1, (int64_t)num_sms() * 8);
  cast_bf16_kernel<<<blocks, 256, 0, s>>>(n, src, dst);
  GCNN_LAUNCH_CHECK();
  return GCNN_OK;
}

}  // namespace gcnn
