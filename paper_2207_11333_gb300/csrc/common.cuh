// Internal definitions shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <utility>

#include "gcnn.h"

namespace gcnn {

// Thread-local error message; returns `code` so callers can `return set_error(...)`.
int set_error(int code, const char *fmt, ...);

#define GCNN_CUDA_TRY(expr)                                                                       \
  do {                                                                                            \
    cudaError_t e_ = (expr);                                                                      \
    if (e_ != cudaSuccess)                                                                        \
      return ::gcnn::set_error(GCNN_ECUDA, "%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_), \
                               __FILE__, __LINE__);                                               \
  } while (0)

#define GCNN_TRY(expr)              \
  do {                              \
    int r_ = (expr);                \
    if (r_ != GCNN_OK) return r_;   \
  } while (0)

#define GCNN_LAUNCH_CHECK() GCNN_CUDA_TRY(cudaGetLastError())

// Bits of the device error word (set with atomicOr by bounds checks; the
// offending access is skipped).
enum : unsigned {
  kErrCollateRange = 1u,   // a graph violates the store limits or capacity
  kErrCapacity = 2u,       // batch totals exceed the context's capacity
  kErrIndex = 4u,          // an index read from memory is out of range
  kErrTimeout = 8u,        // a bounded wait inside a kernel expired
};

// Per-graph limits of the collator (a warp sorts one graph in shared memory).
constexpr int kMaxGraphNodes = 255;
constexpr int kMaxGraphEdges = 1024;

constexpr int kAgg = 5;      // sum, mean, min, max, std
constexpr int kScalers = 3;  // identity, amplification, attenuation

// Device-side batch dimensions written by the collator: {G, N, E, 0}.
struct DevDims {
  const int *p;  // nullptr: use the host-side sizes
  __device__ __forceinline__ int graphs(int h) const { return p ? p[0] : h; }
  __device__ __forceinline__ int nodes(int h) const { return p ? p[1] : h; }
  __device__ __forceinline__ int edges(int h) const { return p ? p[2] : h; }
};

// ---------------------------------------------------------------- launches
// Programmatic dependent launch.  A kernel launched with the programmatic
// stream-serialisation attribute may be scheduled while its predecessor in the
// stream is still running, so every kernel of the library begins with
// pdl_entry(): griddepcontrol.wait blocks until the predecessor grid has
// completed and its writes are visible (a no-op for a normal launch), then
// griddepcontrol.launch_dependents lets the successor be scheduled.  Every CTA
// executes the wait before it can exit, so the completion of a grid implies the
// completion of every earlier grid in the stream; only work that touches no
// global memory (shared-memory barrier set-up, tensor-map prefetch) may come
// before it.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
// Kernel timeline (gcnn_timeline_*): a device buffer of (clock, kernel id)
// records.  Each translation unit has its own copy of the pointer below,
// set by its timeline_attach_* function (the device code is not linked
// across units).
struct Timeline {
  unsigned n, cap;
  unsigned long long *t;
  unsigned *id;
};
static __device__ Timeline *g_timeline = nullptr;

__device__ __forceinline__ void timeline_stamp(unsigned kid) {
  if (threadIdx.x == 0 && threadIdx.y == 0 && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0) {
    Timeline *tl = g_timeline;
    if (tl) {
      unsigned long long t;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
      const unsigned k = atomicAdd(&tl->n, 1u);
      if (k < tl->cap) {
        tl->t[k] = t;
        tl->id[k] = kid;
      }
    }
  }
}

// kid: the kernel's GCNN_K_* identifier (timeline records)
__device__ __forceinline__ void pdl_entry(unsigned kid) {
  pdl_wait();
  pdl_launch_dependents();
  timeline_stamp(kid);
}

#define GCNN_TIMELINE_ATTACH(unit)                                                        \
  int timeline_attach_##unit(void *tl) {                                                  \
    GCNN_CUDA_TRY(cudaMemcpyToSymbol(g_timeline, &tl, sizeof(tl)));                       \
    return GCNN_OK;                                                                       \
  }

// Launches on the legacy or per-thread default stream keep full serialisation;
// GCNN_PDL=0 in the environment turns the attribute off everywhere.
inline bool pdl_enabled(cudaStream_t s) {
  static const bool on = [] {
    const char *v = std::getenv("GCNN_PDL");
    return !(v && v[0] == '0');
  }();
  return on && s != nullptr && s != cudaStreamLegacy && s != cudaStreamPerThread;
}

// kernel<<<grid, block, smem, s>>>(args...) with programmatic serialisation.
template <typename... P, typename... A>
int launch(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, A &&...args) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = pdl_enabled(s) ? 1 : 0;
  GCNN_CUDA_TRY(cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...));
  return GCNN_OK;
}

inline unsigned ceil_div(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

// Two floats -> packed BF16 pair (round to nearest even), lo in the low half.
__device__ __forceinline__ uint32_t bf16x2(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}

// Four floats -> four BF16 at p (8-byte aligned).
__device__ __forceinline__ void st_bf16x4(uint16_t *p, float a, float b, float c, float d) {
  *reinterpret_cast<uint2 *>(p) = make_uint2(bf16x2(a, b), bf16x2(c, d));
}

}  // namespace gcnn
