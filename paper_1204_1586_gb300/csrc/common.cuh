// Shared device helpers and launch-parameter structs for the cpgrad kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/cpgrad.h"

namespace cpg {

constexpr int kMaxOrder = CPG_MAX_ORDER;

// Device status word values (stored in the first word of the workspace).
constexpr int kStatusOk = 0;

// Geometry of one leading contraction (Algorithm 2 steps 4/7):
// Y viewed as the J x K column-major matrix reshape(Y, [J_k, K_k]) (eq. 2.3).
// Rows j index modes [0, k), columns c index modes [k, N).
template <typename T>
struct LeadArgs {
  const T* Y;
  int64_t J, K;
  int N, k;                 // order and split (k leading modes in J)
  int R;                    // total rank
  int r0;                   // first rank column handled by this launch
  int64_t I[kMaxOrder];
  const T* A[kMaxOrder];    // factors, column-major I_m x R
  int64_t Kc;               // columns per K-split (multiple of the tile width)
  int nrt;                  // row tiles per J-block (1 whenever the R side runs)
  T* Rpart;                 // [nKs][R][J]  R-side partial sums (per K-split)
  T* Lpart;                 // [nJb][R][K]  L-side partial sums (per J-block)
  double* normpart;         // [nJb*nKs] partial sums of y^2, or nullptr
  int vec_ok;               // 1: 16-byte copies are legal (J*sizeof(T) % 16 == 0, aligned Y)
};

// ---- cp.async (LDGSTS) wrappers ------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

template <int BYTES>
__device__ __forceinline__ void cp_async_small(void* dst, const void* src) {
  static_assert(BYTES == 4 || BYTES == 8, "small cp.async is 4 or 8 bytes");
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(smem_u32(dst)), "l"(src), "n"(BYTES)
               : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Product over modes [m_begin, m_end) of A_m[i_m(idx), r], where idx is the
// column-major linear index over those modes (mode m_begin fastest, eq. 2.1).
// This is one entry of the Khatri-Rao matrix (Notation 2.1) / one element of
// the Kronecker vector built by eq. 3.3.
template <typename T>
__device__ __forceinline__ T kr_entry(const T* const* A, const int64_t* I, int m_begin, int m_end, int64_t idx,
                                      int r) {
  T p = T(1);
  for (int m = m_begin; m < m_end; ++m) {
    const int64_t In = I[m];
    const int64_t q = idx / In;
    const int64_t i = idx - q * In;
    p *= A[m][i + In * r];
    idx = q;
  }
  return p;
}

}  // namespace cpg
