// BF16 GEMM on the Blackwell tensor cores for the dense node-wise layers of
// the PNA convolution and their gradients: TMA loads, tcgen05.mma with the
// FP32 accumulator in TMEM, warp-specialised mbarrier pipeline.
//
// Each operand is one BF16 row-major array described by a TMA tensor map
// (128-byte swizzle, 64-element boxes along the contiguous dimension):
//   K-major  (contiguous along K): A tiles 128 rows x 64 k, B tiles BN x 64 k
//   MN-major (contiguous along M/N, e.g. node-major activations in the
//            weight-gradient GEMMs that reduce over nodes): boxes of
//            64 M/N elements x 64 k rows
// Zero fill past the array's extent pads K to a multiple of 64.  Rows past
// the batch's true node count inside the array are cleared in shared memory
// before the MMA when K runs over nodes.
//
// Roles (256 threads, one 128 x BN output tile per CTA, BN <= 128; two CTAs
// fit one SM, whose tensor core then runs both CTAs' MMAs side by side):
//   warp 0   one lane issues the TMA loads of a stage after the stage's
//            "empty" barrier fired, with the byte count on its "full" barrier
//   warp 1   waits "full", issues four tcgen05.mma (K = 16 each) and commits
//            them to the stage's "empty" barrier; after the last stage it
//            commits to the "accumulator ready" barrier
//   all 8    wait for the accumulator, drain TMEM (tcgen05.ld) into an FP32
//            tile staged in the idle pipeline buffers, then write it
//            row-contiguously: bias / ReLU, FP32 and BF16 outputs, the masked
//            and scaled BF16 gradient blocks, or split-K partials
// Every wait is bounded (~2 s): on expiry the kernel sets kErrTimeout in the
// device error word, skips its epilogue and releases TMEM.
#include <cuda.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "kernels.cuh"

namespace gcnn {
namespace {

constexpr int BM = 128, BK = 64, STAGES = 3, kThreads = 256;
constexpr int kMaxBN = 128;
// Co-resident CTAs per SM: about 100 KB of shared memory and at most 128
// registers per thread each.  One CTA issues its MMAs at a latency-bound rate
// well below the SM's tensor throughput for tiles up to 128 wide; a second
// CTA on the same SM, from another stream's GEMM or from the next wave of a
// large grid, nearly doubles the SM's rate.  A launch is planned for at most
// one CTA per SM: within one short launch a second CTA per SM only adds its
// fixed costs (measured).
constexpr int kCtasPerSm = 2;
constexpr int kDrain = 4;  // 8-column TMEM loads in flight per thread in the epilogue (register budget)
constexpr int kATileBytes = BM * BK * 2;        // 16 KB
constexpr int kBTileBytes = kMaxBN * BK * 2;    // 16 KB
constexpr int kStageBytes = kATileBytes + kBTileBytes;
// masked-gradient epilogue: ReLU-mask bits (8 words per tile row) and the
// tile rows' degree scalers, prefetched during the main loop
constexpr int kMaskWords = kMaxBN / 32;
constexpr int kSideBytes = BM * kMaskWords * 4 + 2 * BM * 4;
constexpr int kSmemBytes = STAGES * kStageBytes + 1024 /* alignment slack */ + 256 /* barriers */ + kSideBytes;
constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz
constexpr uint32_t kMnAtomBytes = 64 * 128;      // 64 M/N elements x 64 k rows

struct TcMaps {
  CUtensorMap a, b;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

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

__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > kWaitCycles) return false;
  }
  return true;
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// ---------------------------------------------------------------- TMA
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int c0, int c1, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_u32(bar))
      : "memory");
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

// Shared-memory matrix descriptor, 128-byte swizzle.  K-major: 8-row groups
// 1024 bytes apart, leading offset unused.  MN-major: 64-element atoms
// kMnAtomBytes apart (leading), 8-row k groups 1024 bytes apart (stride).
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

// 32 lanes x 8 consecutive 32-bit columns (thread t: lane base + t); the
// registers are valid after tmem_wait_ld().
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t r[8]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// ---------------------------------------------------------------- epilogue
__device__ __forceinline__ void finish8(const TcEpilogue &e, int n, float v[8]) {
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    if (e.bias && n + q < e.bias_n) v[q] += e.bias[n + q];
    if (e.relu) v[q] = fmaxf(v[q], 0.f);
  }
}

__device__ __forceinline__ void st_bf16x8(uint16_t *p, const float v[8], float s) {
  *reinterpret_cast<uint4 *>(p) = make_uint4(bf16x2(s * v[0], s * v[1]), bf16x2(s * v[2], s * v[3]),
                                             bf16x2(s * v[4], s * v[5]), bf16x2(s * v[6], s * v[7]));
}

// Final value v of C(row, n..n+7) to every requested output.
__device__ __forceinline__ void emit8(const TcEpilogue &e, int N, int row, int n, const float v[8]) {
  if (e.C) {
    float *c = e.C + (size_t)row * e.ldc + n;
    *reinterpret_cast<float4 *>(c) = make_float4(v[0], v[1], v[2], v[3]);
    *reinterpret_cast<float4 *>(c + 4) = make_float4(v[4], v[5], v[6], v[7]);
  }
  if (e.C16) st_bf16x8(e.C16 + (size_t)row * e.ld16 + n, v, 1.f);
  if (e.D3) {  // [amp g | att g | g], g = v * [mask > 0]
    const float4 m0 = *reinterpret_cast<const float4 *>(e.mask + (size_t)row * e.ldm + n);
    const float4 m1 = *reinterpret_cast<const float4 *>(e.mask + (size_t)row * e.ldm + n + 4);
    const float mk[8] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z, m1.w};
    float g[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) g[q] = mk[q] > 0.f ? v[q] : 0.f;
    uint16_t *o = e.D3 + (size_t)row * e.ld3 + n;
    st_bf16x8(o, g, e.amp[row]);
    st_bf16x8(o + N, g, e.att[row]);
    st_bf16x8(o + 2 * N, g, 1.f);
  }
}

// ---------------------------------------------------------------- cluster
// barrier over every thread of every CTA of the cluster (release / acquire)
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// 16 bytes at shared-memory address a of cluster CTA `rank`
__device__ __forceinline__ float4 ld_cluster4(uint32_t a, int rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  float4 v;
  asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(r)
               : "memory");
  return v;
}

// Rows r0, r0 + rs, r0 + 2 rs, r0 + 3 rs (those below re) of the staged tile
// at column cn, each summed over the cluster's `ranks` CTAs in rank order (the
// K-splits of one output tile), or the CTA's own rows.  The four rows' loads
// from rank z + 1 are issued before the sums of rank z, so a warp waits for
// one remote-load latency per rank, not one per row and rank; the order of
// the additions, and so every result bit, does not depend on this.
// LEAN (register-capped kernels): one rank's loads at a time.
template <bool LEAN>
__device__ __forceinline__ void rows_sum4(const float *S, int RS, int r0, int rs, int re, int cn, int ranks,
                                          float4 v[4]) {
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  if (ranks == 1) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
      v[u] = r0 + rs * u < re ? *reinterpret_cast<const float4 *>(S + (size_t)(r0 + rs * u) * RS + cn) : zero;
    return;
  }
  uint32_t a[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) a[u] = smem_u32(S + (size_t)(r0 + rs * u) * RS + cn);
  if constexpr (LEAN) {
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = r0 + rs * u < re ? ld_cluster4(a[u], 0) : zero;
    for (int z = 1; z < ranks; ++z) {
      float4 t[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) t[u] = r0 + rs * u < re ? ld_cluster4(a[u], z) : zero;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        v[u].x += t[u].x; v[u].y += t[u].y; v[u].z += t[u].z; v[u].w += t[u].w;
      }
    }
  } else {
    float4 t[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      v[u] = r0 + rs * u < re ? ld_cluster4(a[u], 0) : zero;
      t[u] = r0 + rs * u < re ? ld_cluster4(a[u], 1) : zero;
    }
    for (int z = 1; z < ranks; ++z) {
      float4 n[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) n[u] = (z + 1 < ranks && r0 + rs * u < re) ? ld_cluster4(a[u], z + 1) : zero;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        v[u].x += t[u].x; v[u].y += t[u].y; v[u].z += t[u].z; v[u].w += t[u].w;
        t[u] = n[u];
      }
    }
  }
}

// ---------------------------------------------------------------- tile stores
// The FP32 tile staged in shared memory (row pitch RS floats) goes to global
// memory row by row.  A row's BN columns take lpr lanes of a warp, 4 columns
// each (lpr the smallest power of two covering BN / 4), so one warp
// instruction covers rpi = 32 / lpr rows: narrow tiles keep every lane busy.
// Slot q = rpi w + (lane / lpr) of warp w takes rows q, q + 8 rpi, q + 16 rpi,
// q + 24 rpi as one batch (every load of a batch issued before its stores),
// then the next 32 rpi rows.  One routine per epilogue kind keeps each kernel
// instantiation's store loop small.
enum EpiKind { kEpiPartial = 0, kEpiC = 1, kEpiD3 = 2 };

struct StoreLanes {
  int cn;     // first column of this lane's 4-column slice
  int slot;   // first row, relative to the range's start
  int rs;     // rows between the batch's four rows (8 rpi)
};

// WIDE: one row per warp instruction whatever BN (the register-capped
// kernels, which the narrower layout would make spill)
template <bool WIDE = false>
__device__ __forceinline__ StoreLanes store_lanes(int BN, int warp, int lane) {
  int lpr = 32;
  if (!WIDE)
    while (lpr > 1 && 4 * (lpr / 2) >= BN) lpr /= 2;
  const int rpi = 32 / lpr;
  return StoreLanes{4 * (lane % lpr), rpi * warp + lane / lpr, 8 * rpi};
}

// split-K partial tile: P[row][n] (pitch N), no epilogue
__device__ __forceinline__ void store_partial(const float *S, int RS, int rows, int BN, int N, int m0, int n0,
                                              float *__restrict__ P, int warp, int lane) {
  const StoreLanes sl = store_lanes(BN, warp, lane);
  const int rs = sl.rs;
#pragma unroll 1
  for (int h = 0; h < 2; ++h) {
    const int cn = 128 * h + sl.cn;
    if (cn >= BN || n0 + cn >= N) continue;
    float *dst = P + (size_t)m0 * N + n0 + cn;
    for (int r0 = sl.slot; r0 < rows; r0 += 4 * rs) {
      float4 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        v[u] = r0 + rs * u < rows ? *reinterpret_cast<const float4 *>(S + (size_t)(r0 + rs * u) * RS + cn)
                                  : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (r0 + rs * u < rows) *reinterpret_cast<float4 *>(dst + (size_t)(r0 + rs * u) * N) = v[u];
    }
  }
}

// C (FP32) and / or C16 (BF16) with optional bias and ReLU, tile rows [rb, re)
// summed over `ranks` cluster CTAs
template <bool LEAN>
__device__ __forceinline__ void store_c(const float *S, int RS, int rb, int re, int ranks, int BN, int N, int m0,
                                        int n0, const TcEpilogue e, int warp, int lane) {
  const StoreLanes sl = store_lanes<LEAN>(BN, warp, lane);
  const int rs = sl.rs;
#pragma unroll 1
  for (int h = 0; h < 2; ++h) {
    const int cn = 128 * h + sl.cn;
    const int n = n0 + cn;
    if (cn >= BN || n >= N) continue;
    float b[4] = {0.f, 0.f, 0.f, 0.f};
    if (e.bias)
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (n + q < e.bias_n) b[q] = e.bias[n + q];
    for (int r0 = rb + sl.slot; r0 < re; r0 += 4 * rs) {
      float4 v[4];
      rows_sum4<LEAN>(S, RS, r0, rs, re, cn, ranks, v);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (r0 + rs * u >= re) break;
        const size_t row = (size_t)(m0 + r0 + rs * u);
        float4 x = make_float4(v[u].x + b[0], v[u].y + b[1], v[u].z + b[2], v[u].w + b[3]);
        if (e.relu) {
          x.x = fmaxf(x.x, 0.f); x.y = fmaxf(x.y, 0.f); x.z = fmaxf(x.z, 0.f); x.w = fmaxf(x.w, 0.f);
        }
        if (e.C) *reinterpret_cast<float4 *>(e.C + row * e.ldc + n) = x;
        if (e.C16) st_bf16x4(e.C16 + row * e.ld16 + n, x.x, x.y, x.z, x.w);
      }
    }
  }
}

// C (FP32, nullable) and the BF16 blocks [amp g | att g | g] of D3, g = v [mask > 0],
// tile rows [rb, re) summed over `ranks` cluster CTAs; mask bits and degree
// scalers come from shared memory (prefetched)
__device__ __forceinline__ void store_d3(const float *S, int RS, int rb, int re, int ranks, int BN, int N, int m0,
                                         int n0, const TcEpilogue e, const uint32_t *mbits, const float *s_amp,
                                         const float *s_att, int warp, int lane) {
  const StoreLanes sl = store_lanes(BN, warp, lane);
  const int rs = sl.rs;
#pragma unroll 1
  for (int h = 0; h < 2; ++h) {
    const int cn = 128 * h + sl.cn;
    const int n = n0 + cn;
    if (cn >= BN || n >= N) continue;
    const int word = cn / 32, shift = cn % 32;
    for (int r0 = rb + sl.slot; r0 < re; r0 += 4 * rs) {
      float4 v[4];
      uint32_t mk[4];
      float am[4], at[4];
      rows_sum4<false>(S, RS, r0, rs, re, cn, ranks, v);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int r = r0 + rs * u;
        mk[u] = 0u;
        am[u] = at[u] = 0.f;
        if (r < re) {
          mk[u] = mbits[r * kMaskWords + word] >> shift;
          am[u] = s_amp[r];
          at[u] = s_att[r];
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (r0 + rs * u >= re) break;
        const size_t row = (size_t)(m0 + r0 + rs * u);
        const float4 x = v[u];
        if (e.C) *reinterpret_cast<float4 *>(e.C + row * e.ldc + n) = x;
        const float gx = (mk[u] & 1u) ? x.x : 0.f, gy = (mk[u] & 2u) ? x.y : 0.f;
        const float gz = (mk[u] & 4u) ? x.z : 0.f, gw = (mk[u] & 8u) ? x.w : 0.f;
        uint16_t *o = e.D3 + row * e.ld3 + n;
        st_bf16x4(o, am[u] * gx, am[u] * gy, am[u] * gz, am[u] * gw);
        st_bf16x4(o + N, at[u] * gx, at[u] * gy, at[u] * gz, at[u] * gw);
        st_bf16x4(o + 2 * N, gx, gy, gz, gw);
      }
    }
  }
}

struct Sizes {
  int M, K;
};

// Row stride (floats) of the staged FP32 output tile: consecutive rows shift
// by 16 bytes modulo 128, so the row-per-thread TMEM drain stores 16-byte
// vectors without shared-memory bank conflicts.
__host__ __device__ constexpr int stage_stride(int BN) { return BN + (36 - BN % 32) % 32; }
static_assert(BM * stage_stride(kMaxBN) * 4 <= STAGES * kStageBytes, "staged tile must fit the pipeline buffers");

__device__ __forceinline__ Sizes actual_sizes(const TcDesc &d, DevDims dims) {
  Sizes s{d.M, d.K};
  if (d.node_dim == kNodeM) s.M = min(d.M, dims.nodes(d.M));
  if (d.node_dim == kNodeK) s.K = min(d.K, dims.nodes(d.K));
  return s;
}

// Clear k rows [from, 64) of an MN-major tile of `atoms` 64-wide atoms (lane-parallel).
__device__ __forceinline__ void clear_k_rows(uint8_t *tile, int atoms, int from, int lane) {
  const int rows = 64 - from;
  for (int q = lane; q < atoms * rows * 8; q += 32) {
    const int a = q / (rows * 8), r = from + (q / 8) % rows, c = q % 8;
    *reinterpret_cast<uint4 *>(tile + a * kMnAtomBytes + r * 128 + c * 16) = make_uint4(0u, 0u, 0u, 0u);
  }
}

// CL: the grid's z dimension (K-splits of one output tile) is a thread-block
// cluster; the split-K partial tiles are summed through distributed shared
// memory instead of a partial buffer and a reduction kernel.
// LEAN: at most 80 registers per thread (3 CTAs' worth of the register
// file): the weight-gradient GEMMs, which run on the backward's second stream
// beside the memory-bound aggregation backward, leave that kernel more of the
// SM's registers for its loads in flight.  Same arithmetic and order.
template <int EPI, bool CL, bool LEAN>
__global__ void __launch_bounds__(kThreads, LEAN ? 3 : kCtasPerSm)
tma_gemm_kernel(const __grid_constant__ TcMaps maps, TcDesc d, DevDims dims, float *__restrict__ partial, int splits,
                int kps, int BN, unsigned *err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + STAGES * kStageBytes);
  uint64_t *empty = full + STAGES;
  uint64_t *acc_ready = empty + STAGES;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(acc_ready + 1);
  uint32_t *flag = tmem_slot + 1;
  uint32_t *mbits = reinterpret_cast<uint32_t *>(smem + STAGES * kStageBytes + 256);  // BM x kMaskWords
  float *s_amp = reinterpret_cast<float *>(mbits + BM * kMaskWords), *s_att = s_amp + BM;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // shared-memory set-up and descriptor prefetch overlap the previous kernel
  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(acc_ready, 1);
    *flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&maps.a)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&maps.b)) : "memory");
  }
  // the batch sizes come from the collator, many launches before this one
  const Sizes sz = actual_sizes(d, dims);
  const int M = sz.M, K = sz.K, N = d.N;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int z = blockIdx.z;
  const int kid = EPI == kEpiPartial ? GCNN_K_GEMM_TC_PARTIAL : (EPI == kEpiC ? GCNN_K_GEMM_TC_C : GCNN_K_GEMM_TC_D3);
  if (m0 >= M) {  // block-uniform, before any barrier wait or TMEM use
    pdl_entry(kid);
    return;
  }
  const int kbeg = z * kps;
  const int kend = min(K, kbeg + kps);
  const int nk = kend > kbeg ? (kend - kbeg + BK - 1) / BK : 0;
  const uint32_t ncols = BN <= 32 ? 32 : (BN <= 64 ? 64 : (BN <= 128 ? 128 : 256));
  const int b_atoms = (BN + 63) / 64;
  const uint32_t a_bytes = kATileBytes;
  const uint32_t b_bytes = d.B.mn_major ? (uint32_t)b_atoms * kMnAtomBytes : (uint32_t)BN * BK * 2;
  auto load_a = [&](int s, int k0) {
    uint8_t *a_tile = smem + s * kStageBytes;
    if (!d.A.mn_major) {
      tma_load_2d(smem_u32(a_tile), &maps.a, k0, m0, &full[s]);
    } else {
      tma_load_2d(smem_u32(a_tile), &maps.a, m0, k0, &full[s]);
      tma_load_2d(smem_u32(a_tile + kMnAtomBytes), &maps.a, m0 + 64, k0, &full[s]);
    }
  };
  auto load_b = [&](int s, int k0) {
    uint8_t *b_tile = smem + s * kStageBytes + kATileBytes;
    if (!d.B.mn_major) {
      tma_load_2d(smem_u32(b_tile), &maps.b, k0, n0, &full[s]);
    } else {
      for (int j = 0; j < b_atoms; ++j)
        tma_load_2d(smem_u32(b_tile + j * kMnAtomBytes), &maps.b, n0 + 64 * j, k0, &full[s]);
    }
  };
  // the stable operand's first stages go out before the dependency wait
  const int pre = d.stable != kStableNone ? min(nk, STAGES) : 0;
  if (tid == 0)
    for (int kt = 0; kt < pre; ++kt) {
      mbar_expect_tx(&full[kt], a_bytes + b_bytes);
      if (d.stable == kStableA) load_a(kt, kbeg + kt * BK);
      else load_b(kt, kbeg + kt * BK);
    }
  pdl_entry(kid);

  if (warp == 0) tmem_alloc(tmem_slot, ncols);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------ TMA producer
    if (lane == 0) {
      for (int kt = 0; kt < nk; ++kt) {
        const int s = kt % STAGES;
        if (kt >= STAGES && !mbar_wait(&empty[s], ((kt / STAGES) - 1) & 1)) {
          atomicOr(flag, 1u);
          break;
        }
        const int k0 = kbeg + kt * BK;
        if (kt < pre) {  // the other operand of a stage started before the wait
          if (d.stable == kStableA) load_b(s, k0);
          else load_a(s, k0);
          continue;
        }
        mbar_expect_tx(&full[s], a_bytes + b_bytes);
        load_a(s, k0);
        load_b(s, k0);
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------ MMA issuer
    const uint32_t idesc = instr_desc(BM, BN, d.A.mn_major, d.B.mn_major);
    const uint32_t a_step = d.A.mn_major ? 2048u : 32u;
    const uint32_t b_step = d.B.mn_major ? 2048u : 32u;
    bool ok = true;
    for (int kt = 0; kt < nk; ++kt) {
      const int s = kt % STAGES;
      if (!mbar_wait(&full[s], (kt / STAGES) & 1)) ok = false;
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) {
        if (lane == 0) atomicOr(flag, 1u);
        break;
      }
      uint8_t *a_tile = smem + s * kStageBytes;
      uint8_t *b_tile = a_tile + kATileBytes;
      const int k0 = kbeg + kt * BK;
      if (d.node_dim == kNodeK && k0 + BK > K) {  // rows past the batch's nodes must not contribute
        const int from = K - k0;
        if (d.A.mn_major) clear_k_rows(a_tile, 2, from, lane);
        if (d.B.mn_major) clear_k_rows(b_tile, b_atoms, from, lane);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
      }
      if (lane == 0) {
        fence_after_sync();
        const uint32_t a_base = smem_u32(a_tile), b_base = smem_u32(b_tile);
#pragma unroll
        for (int j = 0; j < BK / 16; ++j)
          mma_bf16(tmem, smem_desc(a_base + j * a_step, d.A.mn_major), smem_desc(b_base + j * b_step, d.B.mn_major),
                   idesc, (kt > 0 || j > 0) ? 1u : 0u);
        mma_commit(&empty[s]);
      }
      __syncwarp();
    }
    if (ok && nk > 0 && lane == 0) mma_commit(acc_ready);
  } else if (EPI == kEpiD3) {
    // ------------------------------------------------ epilogue inputs (warps 2-7)
    // mask bit (row r, column 32 w + lane) = [mask > 0]; eight rows per batch
    // with their loads issued together
    const TcEpilogue e = d.ep;
    const int rows = min(BM, M - m0), words = (BN + 31) / 32;
    const int pw = warp - 2, npw = kThreads / 32 - 2;
    for (int q0 = pw; q0 < BM * words; q0 += 8 * npw) {
      bool bit[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int q = q0 + u * npw, r = q / words, c = 32 * (q % words) + lane;
        bit[u] = false;
        if (q < BM * words && r < rows && c < BN && n0 + c < N)
          bit[u] = e.mask[(size_t)(m0 + r) * e.ldm + n0 + c] > 0.f;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int q = q0 + u * npw;
        const uint32_t b = __ballot_sync(0xffffffffu, bit[u]);
        if (lane == 0 && q < BM * words) mbits[(q / words) * kMaskWords + q % words] = b;
      }
    }
    for (int r = tid - 64; r < BM; r += kThreads - 64) {
      s_amp[r] = r < rows ? e.amp[m0 + r] : 0.f;
      s_att[r] = r < rows ? e.att[m0 + r] : 0.f;
    }
  }
  // ------------------------------------------------ epilogue (all 8 warps)
  // (1) warp w drains TMEM lanes 32*(w%4).. (tile rows) and half w/4 of the
  //     columns into an FP32 tile staged in the idle pipeline buffers;
  // (2) the warps write the tile row by row, each row's 4-column slices
  //     spread over the lanes (coalesced stores).
  {
    bool ok = true;
    if (nk > 0) {
      ok = mbar_wait(acc_ready, 0);
      if (!ok && lane == 0) atomicOr(flag, 1u);
      fence_after_sync();
    }
    ok = __all_sync(0xffffffffu, ok);
    float *S = reinterpret_cast<float *>(smem);
    const int RS = stage_stride(BN);
    if (ok) {
      const int r = 32 * (warp & 3) + lane;
      const int groups = BN / 8, half = (groups + 1) / 2;
      const int g0 = warp < 4 ? 0 : half, g1 = warp < 4 ? half : groups;
      for (int gb = g0; gb < g1; gb += kDrain) {
        uint32_t v[kDrain][8];
        const int cnt = min(kDrain, g1 - gb);
        if (nk > 0) {
#pragma unroll
          for (int u = 0; u < kDrain; ++u)
            if (u < cnt) tmem_ld8(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)((gb + u) * 8), v[u]);
          tmem_wait_ld();
        } else {
#pragma unroll
          for (int u = 0; u < kDrain; ++u)
#pragma unroll
            for (int q = 0; q < 8; ++q) v[u][q] = 0u;
        }
#pragma unroll
        for (int u = 0; u < kDrain; ++u) {
          if (u >= cnt) break;
          float *p = S + (size_t)r * RS + (gb + u) * 8;
          *reinterpret_cast<uint4 *>(p) = make_uint4(v[u][0], v[u][1], v[u][2], v[u][3]);
          *reinterpret_cast<uint4 *>(p + 4) = make_uint4(v[u][4], v[u][5], v[u][6], v[u][7]);
        }
      }
    }
    const bool failed = __syncthreads_or(!ok);
    if (CL) cluster_sync();  // every CTA's tile is staged (reached after a failure too)
    if (!failed) {
      const int rows = min(BM, M - m0);
      int rb = 0, re = rows, ranks = 1;
      if (CL) {  // this CTA's share of the tile's rows, summed over the cluster
        const int share = (rows + splits - 1) / splits;
        rb = min(rows, z * share);
        re = min(rows, rb + share);
        ranks = splits;
      }
      if constexpr (EPI == kEpiPartial)
        store_partial(S, RS, rows, BN, N, m0, n0, partial + (size_t)z * d.M * N, warp, lane);
      else if constexpr (EPI == kEpiC)
        store_c<LEAN>(S, RS, rb, re, ranks, BN, N, m0, n0, d.ep, warp, lane);
      else
        store_d3(S, RS, rb, re, ranks, BN, N, m0, n0, d.ep, mbits, s_amp, s_att, warp, lane);
    }
    if (CL) cluster_sync();  // no CTA leaves while its tile may still be read
  }
  fence_before_sync();
  __syncthreads();
  if (tid == 0 && *flag && err) atomicOr(err, kErrTimeout);
  if (warp == 0) tmem_free(tmem, ncols);
}

// C = epilogue(sum over splits); one thread per 8 outputs
__global__ void __launch_bounds__(256) tc_reduce_kernel(TcDesc d, DevDims dims, const float *__restrict__ partial,
                                                       int splits) {
  pdl_entry(GCNN_K_GEMM_TC_REDUCE);
  const Sizes sz = actual_sizes(d, dims);
  const int M = sz.M, N = d.N, N8 = N / 8;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)M * N8) return;
  const int row = (int)(t / N8), n = (int)(t % N8) * 8;
  float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
  for (int z = 0; z < splits; ++z) {
    const float *p = partial + ((size_t)z * d.M + row) * N + n;
    const float4 a = *reinterpret_cast<const float4 *>(p), b = *reinterpret_cast<const float4 *>(p + 4);
    v[0] += a.x; v[1] += a.y; v[2] += a.z; v[3] += a.w; v[4] += b.x; v[5] += b.y; v[6] += b.z; v[7] += b.w;
  }
  const TcEpilogue e = d.ep;
  finish8(e, n, v);
  emit8(e, N, row, n, v);
}

// ---------------------------------------------------------------- host
using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder() {
  static EncodeTiled fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
  });
  return fn;
}

// Map of a row-major BF16 array [rows][cols] (row pitch ld elements), boxes of
// 64 contiguous elements x box_rows rows, 128-byte swizzle, zero fill.
int make_map(CUtensorMap *m, const TcMat &a, int box_rows) {
  EncodeTiled enc = encoder();
  if (!enc) return set_error(GCNN_ECUDA, "cuTensorMapEncodeTiled is not available");
  if (!a.ptr || a.rows < 1 || a.cols < 1 || a.ld % 8 || a.cols > a.ld || reinterpret_cast<uintptr_t>(a.ptr) % 16)
    return set_error(GCNN_EINVAL, "tc gemm: operand must be 16-byte aligned with ld a multiple of 8");
  const cuuint64_t dim[2] = {(cuuint64_t)a.cols, (cuuint64_t)a.rows};
  const cuuint64_t stride[1] = {(cuuint64_t)a.ld * 2};
  const cuuint32_t box[2] = {64u, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1u, 1u};
  const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<uint16_t *>(a.ptr), dim, stride, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error(GCNN_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return GCNN_OK;
}

constexpr int kMaxCluster = 6;  // largest split-K cluster (co-resident capacity falls beyond)

template <int EPI, bool CL, bool LEAN = false>
void set_smem_attr(int *rc) {
  if (*rc == GCNN_OK &&
      cudaFuncSetAttribute(tma_gemm_kernel<EPI, CL, LEAN>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes) !=
          cudaSuccess)
    *rc = set_error(GCNN_ECUDA, "tc gemm: cannot set the shared-memory size");
}

// co-resident clusters of `size` CTAs of the cluster kernel of one epilogue kind
template <int EPI>
int cluster_capacity_of(int size) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 1;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = size;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(1, 1, size);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = kSmemBytes;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, (void *)tma_gemm_kernel<EPI, true, false>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

int g_rc = GCNN_OK;
int g_capacity[2][kMaxCluster + 1];  // [masked-gradient kind][cluster size]

// shared-memory attributes and cluster capacities, once per process
int configure() {
  static std::once_flag once;
  std::call_once(once, [] {
    int rc = GCNN_OK;
    set_smem_attr<kEpiPartial, false>(&rc);
    set_smem_attr<kEpiC, false>(&rc);
    set_smem_attr<kEpiD3, false>(&rc);
    set_smem_attr<kEpiC, true>(&rc);
    set_smem_attr<kEpiD3, true>(&rc);
    set_smem_attr<kEpiPartial, false, true>(&rc);
    set_smem_attr<kEpiC, false, true>(&rc);
    set_smem_attr<kEpiC, true, true>(&rc);
    for (int sz = 2; sz <= kMaxCluster && rc == GCNN_OK; ++sz) {
      g_capacity[0][sz] = cluster_capacity_of<kEpiC>(sz);
      g_capacity[1][sz] = cluster_capacity_of<kEpiD3>(sz);
    }
    g_rc = rc;
  });
  return g_rc;
}

struct Plan {
  int BN, ntiles, splits;
  bool cluster;  // split-K summed in a cluster through distributed shared memory
};

// Tile width and split count of one launch.  A CTA's time is dominated by
// the bytes it moves: operand tiles from L2 (~100 GB/s per SM), the FP32
// accumulator tile and the epilogue outputs to memory (~40 GB/s per SM
// sustained by one CTA), and for split-K either a reduction pass over partial
// tiles in global memory (a separate kernel) or, with the splits of a tile
// in one cluster, reads of the other CTAs' staged tiles (~50 GB/s per SM) and
// two cluster barriers, each CTA then storing its share of the rows.  Among
// widths BN (multiple of 16, <= 128) and splits whose grid fits one CTA per
// SM (clusters within their co-resident capacity), take the smallest
// estimate; grids larger than that use the widest tiles and no split.
// out_bytes: epilogue bytes per output element; b_mn: B tiles are MN-major
// (loaded in 64-column atoms); d3: masked-gradient epilogue.
Plan choose(int M, int N, int K, int max_splits, int max_ctas, double out_bytes, bool b_mn, bool d3) {
  const int sms = max_ctas > 0 ? std::min(max_ctas, num_sms()) : num_sms();
  const long long mtiles = (M + BM - 1) / BM;
  const int ktiles = std::max(1, (K + BK - 1) / BK);
  Plan best{0, 0, 1, false};
  double best_t = 1e30;
  for (int bn = 16; bn <= kMaxBN; bn += 16) {
    const int nt = (N + bn - 1) / bn;
    if (nt > 1 && (long long)bn * (nt - 1) >= N) continue;
    const double b_tile = b_mn ? ((bn + 63) / 64) * 8192.0 : bn * 128.0;
    for (int sp = 1; sp <= std::min(max_splits, ktiles); ++sp) {
      if (mtiles * nt * sp > sms) break;
      const int kps = (ktiles + sp - 1) / sp;
      const double t_load = kps * (kATileBytes + b_tile) / 1.0e5;          // us at 100 GB/s
      const double t_out = BM * (double)bn * (sp > 1 ? 4.0 : out_bytes) / 4.0e4;  // us at 40 GB/s
      const double t_red = sp > 1 ? 2.0 + (double)M * N * (4.0 * sp + out_bytes) / 5.0e6 : 0.0;
      const double t = t_load + t_out + t_red;
      if (t < best_t) {
        best_t = t;
        best = Plan{bn, nt, sp, false};
      }
      if (sp >= 2 && sp <= kMaxCluster && mtiles * nt <= g_capacity[d3 ? 1 : 0][sp] && mtiles * nt * sp <= sms) {
        const double t_cl = t_load + BM * (double)bn * 4.0 / 5.0e4 + 0.5 + BM * (double)bn * out_bytes / sp / 4.0e4;
        if (t_cl < best_t) {
          best_t = t_cl;
          best = Plan{bn, nt, sp, true};
        }
      }
    }
  }
  if (best.BN == 0) {  // more than one wave: widest tiles, no split
    best.ntiles = (N + kMaxBN - 1) / kMaxBN;
    best.BN = ((N + best.ntiles - 1) / best.ntiles + 15) / 16 * 16;
    best.splits = 1;
  }
  return best;
}

// Upper bound of the split count choose() can return for these sizes.
int max_splits_of(int M, int K) {
  const long long mtiles = (M + BM - 1) / BM;
  const int ktiles = std::max(1, (K + BK - 1) / BK);
  return (int)std::max<long long>(1, std::min<long long>({32LL, (long long)ktiles, num_sms() / std::max(1LL, mtiles)}));
}

// kernel<<<grid, kThreads, kSmemBytes, s>>> as a cluster of (1, 1, cz) CTAs
// (cz > 1), with programmatic serialisation like every launch of the library
template <typename... P, typename... A>
int launch_gemm(void (*kernel)(P...), dim3 grid, int cz, cudaStream_t s, A &&...args) {
  cudaLaunchAttribute attr[2];
  int n = 0;
  if (cz > 1) {
    attr[n].id = cudaLaunchAttributeClusterDimension;
    attr[n].val.clusterDim.x = 1;
    attr[n].val.clusterDim.y = 1;
    attr[n].val.clusterDim.z = cz;
    ++n;
  }
  if (pdl_enabled(s)) {
    attr[n].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[n].val.programmaticStreamSerializationAllowed = 1;
    ++n;
  }
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = kSmemBytes;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = n;
  GCNN_CUDA_TRY(cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...));
  return GCNN_OK;
}

}  // namespace

namespace {
// One GEMM with the planner's plan, or with `force` (measurement: gcnn_gemm_study).
int run_planned(const TcDesc &d, DevDims dims, const GemmWorkspace &ws, unsigned *err, cudaStream_t s,
                const Plan *force, Plan *used) {
  if (d.M <= 0 || d.N <= 0 || d.K < 0) return GCNN_OK;
  const TcEpilogue &e = d.ep;
  if (d.N % 8 || (e.C && (e.ldc % 4 || reinterpret_cast<uintptr_t>(e.C) % 16)) ||
      (e.C16 && (e.ld16 % 8 || reinterpret_cast<uintptr_t>(e.C16) % 16)) ||
      (e.D3 && (e.ld3 % 8 || reinterpret_cast<uintptr_t>(e.D3) % 16 || !e.mask || !e.amp || !e.att ||
                e.ldm % 4 || reinterpret_cast<uintptr_t>(e.mask) % 16 || e.bias || e.relu)))
    return set_error(GCNN_EINVAL, "tc gemm: N must be a multiple of 8 and outputs 16-byte aligned");
  GCNN_TRY(configure());
  const double out_bytes = (e.C ? 4.0 : 0.0) + (e.C16 ? 2.0 : 0.0) + (e.D3 ? 10.0 : 0.0);
  Plan plan = choose(d.M, d.N, d.K, ws.max_splits, ws.max_ctas, out_bytes, d.B.mn_major, e.D3 != nullptr);
  if (force) plan = *force;
  if (plan.BN < 16 || plan.BN > kMaxBN || plan.BN % 16 || plan.ntiles < 1 || plan.splits < 1)
    return set_error(GCNN_EINVAL, "tc gemm: tile width must be a multiple of 16 in [16, %d]", kMaxBN);
  if (plan.splits > 1 && !plan.cluster && (size_t)plan.splits * d.M * d.N > ws.floats) plan.splits = 1;
  if (used) *used = plan;
  const int BN = plan.BN, ntiles = plan.ntiles, splits = plan.splits;
  const int ktiles = (d.K + BK - 1) / BK;
  TcMaps maps;
  GCNN_TRY(make_map(&maps.a, d.A, d.A.mn_major ? 64 : BM));
  GCNN_TRY(make_map(&maps.b, d.B, d.B.mn_major ? 64 : BN));
  const int kps = (ktiles + splits - 1) / splits * BK;
  dim3 grid(ntiles, (d.M + BM - 1) / BM, splits);
  // the masked-gradient epilogue has no register-capped form
  const bool lean = d.lean && !e.D3;
  if (splits > 1 && plan.cluster) {
    auto kernel = e.D3 ? tma_gemm_kernel<kEpiD3, true, false>
                       : (lean ? tma_gemm_kernel<kEpiC, true, true> : tma_gemm_kernel<kEpiC, true, false>);
    return launch_gemm(kernel, grid, splits, s, maps, d, dims, (float *)nullptr, splits, kps, BN, err);
  }
  auto kernel = splits > 1 ? (lean ? tma_gemm_kernel<kEpiPartial, false, true> : tma_gemm_kernel<kEpiPartial, false, false>)
                           : (e.D3 ? tma_gemm_kernel<kEpiD3, false, false>
                                   : (lean ? tma_gemm_kernel<kEpiC, false, true> : tma_gemm_kernel<kEpiC, false, false>));
  GCNN_TRY(launch_gemm(kernel, grid, 1, s, maps, d, dims, splits > 1 ? ws.partial : nullptr, splits, kps, BN, err));
  if (splits > 1) {
    const long long work = (long long)d.M * (d.N / 8);
    GCNN_TRY(launch(tc_reduce_kernel, ceil_div(work, 256), 256, 0, s, d, dims, (const float *)ws.partial, splits));
  }
  return GCNN_OK;
}

}  // namespace

int run_gemm_tc(const TcDesc &d, DevDims dims, const GemmWorkspace &ws, unsigned *err, cudaStream_t s) {
  return run_planned(d, dims, ws, err, s, nullptr, nullptr);
}

// One CTA per SM: with two CTA slots per SM the second stream's GEMM and the
// main stream's run side by side on every SM instead of splitting the SMs.
int side_gemm_ctas() { return num_sms(); }

size_t gemm_tc_workspace_floats(int M, int N, int K) {
  const int sp = max_splits_of(M, K);
  return sp > 1 ? (size_t)sp * M * N : 0;
}

// ---------------------------------------------------------------- study
// Timing of the training step's six BF16 GEMM shapes for n_atoms rows and
// hidden H (measurement support; gcnn_gemm_study documents the modes and the
// rows).  Operands are arbitrary BF16 values in device buffers of the step's
// layouts; each time is the best of five replays of a graph of 20 launches.
namespace {
struct StudyShape {
  int id;
  TcDesc d;
  int max_ctas;
};

int study_time(const StudyShape &sh, DevDims dims, const GemmWorkspace &ws, unsigned *err, cudaStream_t s,
               const Plan *force, Plan *used, double *us) {
  for (int i = 0; i < 3; ++i) GCNN_TRY(run_planned(sh.d, dims, ws, err, s, force, used));
  GCNN_CUDA_TRY(cudaStreamSynchronize(s));
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  GCNN_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  int rc = GCNN_OK;
  for (int i = 0; i < 20 && rc == GCNN_OK; ++i) rc = run_planned(sh.d, dims, ws, err, s, force, nullptr);
  const cudaError_t e = cudaStreamEndCapture(s, &g);
  if (rc != GCNN_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return rc != GCNN_OK ? rc : set_error(GCNN_ECUDA, "gemm study: capture failed");
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  double best = 1e30;
  if (cudaGraphInstantiate(&ge, g, 0) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess || cudaGraphLaunch(ge, s) != cudaSuccess)
    rc = set_error(GCNN_ECUDA, "gemm study: graph set-up failed");
  for (int k = 0; k < 5 && rc == GCNN_OK; ++k) {
    float ms = 0.f;
    if (cudaEventRecord(e0, s) != cudaSuccess || cudaGraphLaunch(ge, s) != cudaSuccess ||
        cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
      rc = set_error(GCNN_ECUDA, "gemm study: timing failed");
    best = std::min(best, 1e3 * ms / 20.0);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (ge) cudaGraphExecDestroy(ge);
  cudaGraphDestroy(g);
  *us = best;
  return rc;
}
}  // namespace

int gemm_tc_study(int n_atoms, int H, int mode, double *rows, int max_rows, int *n_rows) {
  *n_rows = 0;
  if (n_atoms < 1 || H < 8 || H % 8 || H > 256 || (mode != 0 && mode != 1) || !rows || max_rows < 1)
    return set_error(GCNN_EINVAL, "gemm study: bad arguments (hidden a multiple of 8, at most 256)");
  GCNN_TRY(configure());
  const int Ng = (n_atoms + 255) / 256 * 256, K3 = (3 * H + 63) / 64 * 64, KH = (H + 63) / 64 * 64;
  const size_t wsf = (size_t)32 * 16 * H * H + (size_t)32 * Ng * 5 * H;
  uint16_t *U = nullptr, *G5 = nullptr, *W = nullptr, *D3 = nullptr;
  float *C = nullptr, *F = nullptr, *ws_p = nullptr;
  int *dd = nullptr;
  unsigned *err = nullptr;
  cudaStream_t s = nullptr;
  int rc = GCNN_OK;
  const size_t nU = (size_t)Ng * 16 * H, nG = (size_t)Ng * 5 * H, nW = (size_t)36 * H * H;
  if (cudaMalloc(&U, 2 * nU) != cudaSuccess || cudaMalloc(&G5, 2 * nG) != cudaSuccess ||
      cudaMalloc(&W, 2 * nW) != cudaSuccess || cudaMalloc(&D3, 2 * nG) != cudaSuccess ||
      cudaMalloc(&C, 4 * nG) != cudaSuccess || cudaMalloc(&F, 4 * ((size_t)Ng * H + 2 * Ng + 5 * H)) != cudaSuccess ||
      cudaMalloc(&ws_p, 4 * wsf) != cudaSuccess || cudaMalloc(&dd, 16) != cudaSuccess ||
      cudaMalloc(&err, 4) != cudaSuccess || cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
    rc = set_error(GCNN_ENOMEM, "gemm study: allocation failed");
  if (rc == GCNN_OK) {
    const int hd[4] = {1, n_atoms, 0, 0};
    // BF16 0x3c00..0x3c3f (about 0.008-0.016) and FP32 0.5 everywhere: finite outputs
    if (cudaMemset(U, 0x3c, 2 * nU) != cudaSuccess || cudaMemset(G5, 0x3c, 2 * nG) != cudaSuccess ||
        cudaMemset(W, 0x3c, 2 * nW) != cudaSuccess || cudaMemset(F, 0, 4 * ((size_t)Ng * H + 2 * Ng + 5 * H)) != cudaSuccess ||
        cudaMemset(err, 0, 4) != cudaSuccess || cudaMemcpy(dd, hd, 16, cudaMemcpyHostToDevice) != cudaSuccess)
      rc = set_error(GCNN_ECUDA, "gemm study: initialisation failed");
  }
  // weights: message [H][2H], update [16H][H], dagg's [5H][3H], dx's [H][3H]
  const uint16_t *Wm = W, *Wu = W + 2 * H * H, *Wd = W + 18 * H * H, *Wx = W + 33 * H * H;
  float *mask = F, *amp = F + (size_t)Ng * H, *att = amp + Ng, *bias = att + Ng;
  std::vector<StudyShape> shapes;
  auto M = [](const uint16_t *p, int ld, int r, int c, bool mn) { return TcMat{p, ld, r, c, mn}; };
  {  // 0: message, x [A | B] + b
    TcDesc d{}; d.M = Ng; d.N = 2 * H; d.K = KH; d.node_dim = kNodeM;
    d.A = M(U, 16 * H, Ng, H, false); d.B = M(Wm, 2 * H, H, 2 * H, true); d.stable = kStableB;
    d.ep.C = C; d.ep.ldc = 2 * H; d.ep.bias = bias; d.ep.bias_n = H;
    shapes.push_back({0, d, 0});
  }
  {  // 1: update, ReLU(U W_U + b) in FP32 and BF16
    TcDesc d{}; d.M = Ng; d.N = H; d.K = 16 * H; d.node_dim = kNodeM;
    d.A = M(U, 16 * H, Ng, 16 * H, false); d.B = M(Wu, H, 16 * H, H, true); d.stable = kStableB;
    d.ep.C = C; d.ep.ldc = H; d.ep.bias = bias; d.ep.bias_n = H; d.ep.relu = true; d.ep.C16 = D3; d.ep.ld16 = H;
    shapes.push_back({1, d, 0});
  }
  {  // 2: dW_U = U^T g (side stream)
    TcDesc d{}; d.M = 16 * H; d.N = H; d.K = Ng; d.node_dim = kNodeK;
    d.A = M(U, 16 * H, Ng, 16 * H, true); d.B = M(G5 + 2 * H, 5 * H, Ng, H, true); d.stable = kStableA;
    d.ep.C = C; d.ep.ldc = H; d.lean = true;
    shapes.push_back({2, d, side_gemm_ctas()});
  }
  {  // 3: dagg = [amp g | att g | g] Wd^T
    TcDesc d{}; d.M = Ng; d.N = 5 * H; d.K = K3; d.node_dim = kNodeM;
    d.A = M(G5, 5 * H, Ng, 3 * H, false); d.B = M(Wd, 3 * H, 5 * H, 3 * H, false); d.stable = kStableB;
    d.ep.C = C; d.ep.ldc = 5 * H;
    shapes.push_back({3, d, 0});
  }
  {  // 4: dW_M = x^T [dP | dQ] (side stream)
    TcDesc d{}; d.M = H; d.N = 2 * H; d.K = Ng; d.node_dim = kNodeK;
    d.A = M(U, 16 * H, Ng, H, true); d.B = M(G5 + 3 * H, 5 * H, Ng, 2 * H, true); d.stable = kStableA;
    d.ep.C = C; d.ep.ldc = 2 * H; d.lean = true;
    shapes.push_back({4, d, side_gemm_ctas()});
  }
  {  // 5: dx = [g | dP | dQ] Wx^T with the masked, scaled BF16 blocks
    TcDesc d{}; d.M = Ng; d.N = H; d.K = K3; d.node_dim = kNodeM;
    d.A = M(G5 + 2 * H, 5 * H, Ng, 3 * H, false); d.B = M(Wx, 3 * H, H, 3 * H, false); d.stable = kStableB;
    d.ep.C = C; d.ep.ldc = H; d.ep.D3 = D3; d.ep.ld3 = 5 * H; d.ep.mask = mask; d.ep.ldm = H; d.ep.amp = amp;
    d.ep.att = att;
    shapes.push_back({5, d, 0});
  }
  const DevDims dims{dd};
  auto emit = [&](int shape, const Plan &p, int K, double us, int is_default) {
    if (*n_rows >= max_rows) return;
    double *r = rows + 8 * (size_t)(*n_rows)++;
    r[0] = shape; r[1] = p.BN; r[2] = p.ntiles; r[3] = p.splits; r[4] = p.cluster ? 1 : 0; r[5] = K; r[6] = us;
    r[7] = is_default;
  };
  for (const StudyShape &sh : shapes) {
    if (rc != GCNN_OK) break;
    const GemmWorkspace w{ws_p, wsf, 32, sh.max_ctas};
    const int sms = sh.max_ctas > 0 ? sh.max_ctas : num_sms();
    if (mode == 0) {  // the planner's plan, then every plan of the planner's search space
      Plan used{};
      double us = 0.0;
      rc = study_time(sh, dims, w, err, s, nullptr, &used, &us);
      if (rc == GCNN_OK) emit(sh.id, used, sh.d.K, us, 1);
      const int mt = (sh.d.M + BM - 1) / BM, kt = (sh.d.K + BK - 1) / BK;
      for (int bn = 16; bn <= kMaxBN && rc == GCNN_OK; bn += 16) {
        const int nt = (sh.d.N + bn - 1) / bn;
        if (nt > 1 && bn * (nt - 1) >= sh.d.N) continue;
        for (int sp = 1; sp <= std::min(kt, 8) && rc == GCNN_OK; ++sp) {
          if (mt * nt * sp > sms) break;
          for (int cl = 0; cl <= 1 && rc == GCNN_OK; ++cl) {
            if (cl && (sp < 2 || sp > kMaxCluster || mt * nt > g_capacity[sh.d.ep.D3 ? 1 : 0][sp])) continue;
            if (!cl && sp > 1 && (size_t)sp * sh.d.M * sh.d.N > wsf) continue;
            const Plan f{bn, nt, sp, cl == 1};
            rc = study_time(sh, dims, w, err, s, &f, &used, &us);
            if (rc == GCNN_OK) emit(sh.id, used, sh.d.K, us, 0);
          }
        }
      }
    } else if (sh.id == 1) {  // the update shape: time against K at tile widths without split
      for (int bn : {32, 64, 112, 128}) {
        const int nt = (sh.d.N + bn - 1) / bn;
        for (int k = 64; k <= sh.d.K && rc == GCNN_OK; k = k < 512 ? 2 * k : k + 512) {
          StudyShape t = sh;
          t.d.K = k;
          t.d.A.cols = std::min(sh.d.A.cols, k);
          t.d.B.rows = std::min(sh.d.B.rows, k);
          const Plan f{bn, nt, 1, false};
          Plan used{};
          double us = 0.0;
          rc = study_time(t, dims, w, err, s, &f, &used, &us);
          if (rc == GCNN_OK) emit(sh.id, used, k, us, 0);
        }
      }
    }
  }
  unsigned herr = 0;
  if (rc == GCNN_OK && (cudaMemcpy(&herr, err, 4, cudaMemcpyDeviceToHost) != cudaSuccess || herr))
    rc = set_error(GCNN_EDEVICE, "gemm study: device error word 0x%x", herr);
  if (s) cudaStreamSynchronize(s);
  for (void *p : {(void *)U, (void *)G5, (void *)W, (void *)D3, (void *)C, (void *)F, (void *)ws_p, (void *)dd,
                  (void *)err})
    if (p) cudaFree(p);
  if (s) cudaStreamDestroy(s);
  return rc;
}

// ---------------------------------------------------------------- casts
namespace {
__global__ void cast_bf16_kernel(int64_t n, const float *__restrict__ src, uint16_t *__restrict__ dst) {
  pdl_entry(GCNN_K_CAST_BF16);
  const int64_t n8 = n / 8;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n8; q += stride) {
    const float4 a = reinterpret_cast<const float4 *>(src)[2 * q], b = reinterpret_cast<const float4 *>(src)[2 * q + 1];
    reinterpret_cast<uint4 *>(dst)[q] =
        make_uint4(bf16x2(a.x, a.y), bf16x2(a.z, a.w), bf16x2(b.x, b.y), bf16x2(b.z, b.w));
  }
  if (blockIdx.x == 0 && threadIdx.x < (int)(n - 8 * n8)) {
    const int64_t k = 8 * n8 + threadIdx.x;
    dst[k] = (uint16_t)(bf16x2(src[k], 0.f) & 0xFFFFu);
  }
}

// Per layer: Wd[n][s*H + c] = W_U[H + blk(s)*5H + n][c] with the scaler order
// (amplification, attenuation, identity) of the backward operand;
// Wx[n] = [W_U[n][0..H) | W_M[n][0..2H)].
__global__ void pack_layer_kernel(int H, const float *__restrict__ msg_w, const float *__restrict__ upd_w,
                                  uint16_t *__restrict__ Wd, uint16_t *__restrict__ Wx) {
  pdl_entry(GCNN_K_PACK_LAYER);
  const long long nd = 15LL * H * H, nx = 3LL * H * H;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < nd) {
    const int n = (int)(t / (3 * H)), k = (int)(t % (3 * H));
    const int s = k / H, c = k % H;
    const int blk = s == 0 ? 1 : (s == 1 ? 2 : 0);
    Wd[t] = (uint16_t)(bf16x2(upd_w[(size_t)(H + blk * 5 * H + n) * H + c], 0.f) & 0xFFFFu);
  } else if (t < nd + nx) {
    const long long u = t - nd;
    const int n = (int)(u / (3 * H)), k = (int)(u % (3 * H));
    const float v = k < H ? upd_w[(size_t)n * H + k] : msg_w[(size_t)n * 2 * H + (k - H)];
    Wx[u] = (uint16_t)(bf16x2(v, 0.f) & 0xFFFFu);
  }
}
}  // namespace

int launch_cast_bf16(int64_t n, const float *src, uint16_t *dst, cudaStream_t s) {
  if (n <= 0) return GCNN_OK;
  if (reinterpret_cast<uintptr_t>(src) % 16 || reinterpret_cast<uintptr_t>(dst) % 16)
    return set_error(GCNN_EINVAL, "cast: buffers must be 16-byte aligned");
  const int blocks = (int)std::min<int64_t>((n / 8 + 255) / 256 + 1, (int64_t)num_sms() * 8);
  GCNN_TRY(launch(cast_bf16_kernel, blocks, 256, 0, s, n, src, dst));
  return GCNN_OK;
}

int launch_pack_layer(int H, const float *msg_w, const float *upd_w, uint16_t *Wd, uint16_t *Wx, cudaStream_t s) {
  const long long work = 18LL * H * H;
  GCNN_TRY(launch(pack_layer_kernel, ceil_div(work, 256), 256, 0, s, H, msg_w, upd_w, Wd, Wx));
  return GCNN_OK;
}

GCNN_TIMELINE_ATTACH(gemm_tc)

}  // namespace gcnn
