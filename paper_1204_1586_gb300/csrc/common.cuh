// Shared device helpers and launch-parameter structs for the cpgrad kernels.
#pragma once

#include <cstdint>
#include <type_traits>
#include <utility>

#include <cuda_runtime.h>

#include "../../include/cpgrad.h"

namespace cpg {

constexpr int kMaxOrder = CPG_MAX_ORDER;

// Unsigned division by a runtime constant d >= 1 for numerators below 2^31
// (round-up multiply-and-shift method of Granlund and Montgomery, PLDI 1994):
// with l = ceil(log2 d) and m = floor(2^32 (2^l - d) / d) + 1,
// n / d = (umulhi(n, m) + n) >> l.  The sum fits 32 bits because n < 2^31.
struct FastDiv {
  uint32_t d = 1, m = 1, l = 0;
  static FastDiv make(uint32_t d) {
    FastDiv f;
    f.d = d;
    uint32_t l = 0;
    while ((uint64_t(1) << l) < d) ++l;
    f.l = l;
    f.m = uint32_t(((uint64_t(1) << 32) * ((uint64_t(1) << l) - d)) / d + 1);
    return f;
  }
  __device__ __forceinline__ uint32_t div(uint32_t n) const { return (__umulhi(n, m) + n) >> l; }
};

// Khatri-Rao rows over a contiguous run of modes [mb, me) (Notation 2.1), as
// the product of the first mode's factor and a table of the remaining modes:
//   W[idx, r] = A_mb[idx % I_mb, r] * Q[idx / I_mb, r]
// with Q the Kronecker table of modes (mb, me) in [r][o] layout (ld = ldq), or
// no table when the run has a single mode, or W = 1 when the run is empty.
template <typename T>
struct KrRows {
  const T* A = nullptr;   // first mode's factor, column-major (ld = d.d); nullptr: empty run
  const T* Q = nullptr;   // table of the other modes, [r][o]; nullptr: single mode
  int64_t ldq = 0;
  FastDiv d;
  __device__ __forceinline__ T at(uint32_t idx, int r) const {
    if (A == nullptr) return T(1);
    const uint32_t q = d.div(idx);
    const uint32_t i = idx - q * d.d;
    T v = A[i + int64_t(d.d) * r];
    if (Q != nullptr) v *= Q[q + ldq * r];
    return v;
  }
  // Split form for software pipelining: fetch() issues the two loads, the
  // caller multiplies the pair later.
  __device__ __forceinline__ void fetch(uint32_t idx, int r, T& fa, T& fq) const {
    if (A == nullptr) {
      fa = T(1);
      fq = T(1);
      return;
    }
    const uint32_t q = d.div(idx);
    const uint32_t i = idx - q * d.d;
    fa = A[i + int64_t(d.d) * r];
    fq = (Q != nullptr) ? Q[q + ldq * r] : T(1);
  }
};

// Geometry of one leading contraction (Algorithm 2 steps 4/7):
// Y viewed as the J x K column-major matrix reshape(Y, [J_k, K_k]) (eq. 2.3).
// Rows j index modes [0, k), columns c index modes [k, N).  J and K < 2^31.
template <typename T>
struct LeadArgs {
  const T* Y;
  int64_t J, K;
  int64_t ldy;              // elements from one column of Y_(1:k) to the next (>= J)
  int R;                    // total rank
  int r0;                   // first rank column handled by this launch
  KrRows<T> wl;             // W_L rows: Khatri-Rao over modes [0, k)
  KrRows<T> wr;             // W_R rows: Khatri-Rao over modes [k, N)
  int64_t Kc;               // columns per K-split (multiple of the tile width)
  int nrt;                  // row tiles per J-block (1 whenever the R side runs)
  T* Rpart;                 // [nKs][R][J]  R-side partial sums (per K-split)
  T* Lpart;                 // [nJb][R][K]  L-side partial sums (per J-block)
  double* normpart;         // [nJb*nKs] partial sums of y^2, or nullptr
  int use_tma;              // 1: tiles arrive by TMA (set by the launcher); 0: element copies
  // Khatri-Rao rows built once per pass (kr_rows_kernel), copied per stage with
  // the tile when tiles arrive by TMA; nullptr: each CTA generates its own.
  //   wpre_r: [Kpad][RT]                 (column c, rank r at c * RT + r)
  //   wpre_l: [J tiles][RT][TJ] if rank-major, else [J tiles][TJ][RT]
  // for this launch's rank group, zero past K / J and past rank R.
  const T* wpre_r;
  const T* wpre_l;
  int* status;              // device status word (bounded-wait timeouts)
};

// ---- programmatic dependent launch ----------------------------------------------
// Kernels are launched with programmatic stream serialization (launch_pdl), so
// a kernel may start while the previous kernel on its stream is finishing.
// griddep_wait() blocks until that kernel has completed and its writes are
// visible (a no-op after an ordinary launch); every kernel calls it before it
// reads what an earlier kernel wrote or writes what one may still read.
// griddep_launch() lets the next kernel start launching; a kernel that never
// calls it triggers when all its CTAs have exited.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

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
    if (m + 1 < m_end) {
      const int64_t q = idx / In;
      p *= A[m][(idx - q * In) + In * r];
      idx = q;
    } else {
      p *= A[m][idx + In * r];
    }
  }
  return p;
}

}  // namespace cpg
