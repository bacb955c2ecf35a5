// All-mode CP gradient for callers that cannot allocate device memory.
//
// Some callers have no way to call cudaMalloc: a plugin loaded into a host
// application that owns every device allocation through its own pool, or
// latency-critical code that must not allocate after start-up (cudaMalloc can
// synchronize the device).  For them this entry point takes its scratch from a
// file-scope device array of fixed size instead of a caller workspace; the
// caller still provides the tensor, the factors and the gradient buffers.
//
// The array belongs to the library image: every GPU that loads the library
// holds CPG_NOALLOC_WORKSPACE_BYTES of it until the process exits.  All calls
// share it and it keeps the contents of the last call, so two calls whose
// work overlaps on the GPU (different streams, or different host threads)
// race on it; calls issued on one stream are ordered and safe.
#include <cuda_runtime.h>

#include "../../include/cpgrad.h"
#include "api_internal.h"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[CPG_NOALLOC_WORKSPACE_BYTES];

constexpr int kMaxDevices = 64;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the array on the current device.  In host code the
// array's name is only a host-side stand-in, so the address is looked up once
// per device (with that device current) and cached.
cpg_status scratch_for_current_device(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CPG_ERR_CUDA;
  if (g_scratch_ptr[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return CPG_ERR_CUDA;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return CPG_OK;
}

}  // namespace

extern "C" cpg_status cp_gradient_all_noalloc(const void* Y, const int64_t* I, int N, const void* const* A, int R,
                                              void* const* G, int precision, int split, void* stream) {
  cpg_opts o{};
  o.precision = precision;
  o.split = split;
  o.stream = stream;
  // The fixed array need not hold the optional pitched copy of Y: without
  // room for it the gradient streams Y itself.
  const size_t need = cpg::workspace_bytes_required(I, N, R, &o, CPG_CALL_GRADIENT_ALL);
  if (need == 0) return CPG_ERR_ARG;
  if (need > size_t(CPG_NOALLOC_WORKSPACE_BYTES)) return CPG_ERR_WORKSPACE;
  void* scratch = nullptr;
  const cpg_status st = scratch_for_current_device(&scratch);
  if (st != CPG_OK) return st;
  o.workspace = scratch;
  o.workspace_bytes = CPG_NOALLOC_WORKSPACE_BYTES;
  // The status word at the start of the array must read zero before use.
  if (cudaMemsetAsync(scratch, 0, 256, static_cast<cudaStream_t>(stream)) != cudaSuccess) return CPG_ERR_CUDA;
  return cp_gradient_all(Y, I, N, A, R, G, &o);
}
