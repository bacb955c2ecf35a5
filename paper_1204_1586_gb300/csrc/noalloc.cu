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

#include <mutex>

#include "../../include/cpgrad.h"
#include "api_internal.h"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[CPG_NOALLOC_WORKSPACE_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the array on the current device.  In host code the
// array's name is only a host-side stand-in, so the address is looked up
// with the device current, once per device (the first call on the device),
// under a lock.  The same set-up clears the device status word at the start
// of the array, synchronously: afterwards only cpg_device_status clears it.
// The cached address is not valid after cudaDeviceReset.
cpg_status scratch_for_current_device(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CPG_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (g_scratch_ptr[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return CPG_ERR_CUDA;
    if (cudaMemset(p, 0, 256) != cudaSuccess) return CPG_ERR_CUDA;
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
  // The argument errors of cp_gradient_all first, with nothing launched.
  const cpg_status arg = cpg::gradient_all_arg_status(Y, I, N, A, R, G, &o);
  if (arg != CPG_OK) return arg;
  // The plan the call runs with this much room, without the optional pitched
  // copy of Y (without room for it the gradient streams Y itself).
  o.workspace_bytes = CPG_NOALLOC_WORKSPACE_BYTES;
  const size_t need = cpg::gradient_all_bytes_for(I, N, R, &o);
  if (need == 0) return CPG_ERR_ARG;
  if (need > size_t(CPG_NOALLOC_WORKSPACE_BYTES)) return CPG_ERR_WORKSPACE;
  void* scratch = nullptr;
  const cpg_status st = scratch_for_current_device(&scratch);
  if (st != CPG_OK) return st;
  o.workspace = scratch;
  return cp_gradient_all(Y, I, N, A, R, G, &o);
}

extern "C" cpg_status cpg_noalloc_scratch(void** ptr, size_t* bytes) {
  if (ptr == nullptr) return CPG_ERR_ARG;
  const cpg_status st = scratch_for_current_device(ptr);
  if (st != CPG_OK) return st;
  if (bytes) *bytes = CPG_NOALLOC_WORKSPACE_BYTES;
  return CPG_OK;
}
