// gcnn_op_aggregate_bwd_noalloc: the aggregation backward with its per-edge
// scratch in a fixed, library-owned device array instead of a caller buffer.
//
// Some callers cannot allocate device memory at the point where they need
// this gradient: a host framework that has already reserved the device's
// memory for its own caching allocator (a fresh cudaMalloc would fail or
// fragment its pool), or a latency-critical loop in which cudaMalloc and
// cudaFree are not acceptable because they can synchronise the device.  For
// them this entry point needs only the inputs and outputs; the scratch lives
// in a file-scope __device__ array that every process loading the library
// holds on every GPU it uses until the process exits.
#include <mutex>

#include "kernels.cuh"

namespace gcnn {
namespace {

// Maximum scratch: n_edges * hidden floats (16 MiB).
constexpr long long kNoAllocScratchFloats = 1LL << 22;

__device__ __align__(256) float g_agg_bwd_scratch[kNoAllocScratchFloats];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
float *g_scratch_addr[kMaxDevices] = {};

// Device address of g_agg_bwd_scratch on the current device (the host-side
// symbol is only a stand-in, never a device address).  Looked up once per
// device, with that device current.
int scratch_address(float **out) {
  int dev = 0;
  GCNN_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return set_error(GCNN_EINVAL, "device ordinal %d not supported", dev);
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_agg_bwd_scratch);
    if (e != cudaSuccess || !p)
      return set_error(GCNN_ECUDA, "cudaGetSymbolAddress(scratch) failed: %s", cudaGetErrorString(e));
    g_scratch_addr[dev] = static_cast<float *>(p);
  }
  *out = g_scratch_addr[dev];
  return GCNN_OK;
}

}  // namespace
}  // namespace gcnn

using namespace gcnn;

extern "C" int gcnn_op_aggregate_bwd_noalloc(int32_t n_nodes, int32_t n_edges, int32_t hidden,
                                             const int32_t *row_ptr, const int32_t *col,
                                             const int32_t *rev, const float *PQ, const float *agg,
                                             const float *dagg, float *dPQ, float std_eps,
                                             void *stream) {
  if (n_nodes < 0 || n_edges < 0 || hidden <= 0 || hidden % 4 ||
      (n_nodes > 0 && (!row_ptr || !col || !rev || !PQ || !agg || !dagg || !dPQ)))
    return set_error(GCNN_EINVAL, "aggregate_bwd_noalloc: bad arguments (hidden must be a multiple of 4)");
  if ((reinterpret_cast<uintptr_t>(PQ) | reinterpret_cast<uintptr_t>(agg) | reinterpret_cast<uintptr_t>(dagg) |
       reinterpret_cast<uintptr_t>(dPQ)) % 16)
    return set_error(GCNN_EINVAL, "aggregate_bwd_noalloc: float buffers must be 16-byte aligned");
  const long long need = (long long)n_edges * hidden;
  if (need > kNoAllocScratchFloats)
    return set_error(GCNN_EINVAL,
                     "aggregate_bwd_noalloc: n_edges * hidden = %lld exceeds the fixed scratch of %lld floats; "
                     "use gcnn_op_aggregate_bwd with a caller buffer",
                     need, kNoAllocScratchFloats);
  float *scratch = nullptr;
  GCNN_TRY(scratch_address(&scratch));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the array keeps the previous call's contents: clear the part this call uses
  if (need > 0) GCNN_CUDA_TRY(cudaMemsetAsync(scratch, 0, (size_t)need * sizeof(float), s));
  return launch_aggregate_bwd(n_nodes, n_edges, hidden, DevDims{nullptr}, row_ptr, col, rev, PQ, agg, dagg, dPQ,
                              scratch, std_eps, nullptr, s);
}
