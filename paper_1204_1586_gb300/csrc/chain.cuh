// Per-mode contractions of Algorithm 2 that follow the leading pass.
//
// The partial tensors of Section 3.3 are held rank-major, X[r][flat], with
// flat the column-major index over the modes X still carries:
//   right side  R^(n): modes [0, n),   flat = a + Alo * i   (i = last mode)
//   left side   L^(n): modes [n, N),   flat = i + In  * b   (i = first mode)
// where a runs over the modes below i and b over the modes above i.
//
//   mode_grad    : g_r^(n)[i] = sum_o X[r][flat(o, i)] * kr[r][o]
//                  -- the 'right' (line 19, eq. 3.12) and 'left' (line 20,
//                  eq. 3.16) finishing contractions of cp_gradient; kr is the
//                  Kronecker vector of the remaining modes (eq. 3.3).
//   mode_contract: X'[r][o] = sum_i X[r][flat(o, i)] * A^(n)[i, r]
//                  -- the recursions of steps 11 (eq. 3.20) and 15 (eq. 3.22).
//   kr_build     : kr[r][o] = prod_m A^(m)[i_m(o), r] over a range of modes.
//
// The first use of R^(k)/L^(k+1) reads the leading pass's partial sums
// (nparts slices) and adds them in a fixed order, so results are
// deterministic run to run.
#pragma once

#include "common.cuh"

namespace cpg {

template <typename T>
struct FacArgs {
  int64_t I[kMaxOrder];
  const T* A[kMaxOrder];
};

template <typename T>
__global__ void kr_build_kernel(T* __restrict__ out, const FacArgs<T> f, int mb, int me, int64_t len, int R) {
  const int64_t total = len * R;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total; t += int64_t(gridDim.x) * blockDim.x) {
    const int r = int(t / len);
    const int64_t o = t - int64_t(r) * len;
    out[t] = kr_entry<T>(f.A, f.I, mb, me, o, r);
  }
}

// One warp per output (i, r).  RIGHT: flat = o + len_o * i.  LEFT: flat = i + In * o.
template <typename T, bool RIGHT>
__global__ void __launch_bounds__(256) mode_grad_kernel(const T* __restrict__ X, int nparts, int64_t part_stride,
                                                         int64_t len_o, int64_t In, int R,
                                                         const T* __restrict__ kr, T* __restrict__ G,
                                                         T* __restrict__ Xred) {
  const int lane = threadIdx.x & 31;
  const int64_t g = int64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (g >= In * R) return;
  const int r = int(g / In);
  const int64_t i = g - int64_t(r) * In;
  const int64_t S = len_o * In;
  const T* Xr = X + int64_t(r) * S;
  const T* w = kr ? kr + int64_t(r) * len_o : nullptr;
  T acc = T(0);
  for (int64_t o = lane; o < len_o; o += 32) {
    const int64_t flat = RIGHT ? (o + len_o * i) : (i + In * o);
    T x = Xr[flat];
    for (int p = 1; p < nparts; ++p) x += Xr[int64_t(p) * part_stride + flat];
    if (Xred) Xred[int64_t(r) * S + flat] = x;
    acc = w ? fma(x, w[o], acc) : acc + x;
  }
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, s);
  if (lane == 0) G[i + In * r] = acc;
}

template <typename T, bool RIGHT>
__global__ void mode_contract_kernel(const T* __restrict__ X, int64_t len_o, int64_t In, int R,
                                     const T* __restrict__ An, T* __restrict__ Xout) {
  const int64_t total = len_o * R;
  const int64_t S = len_o * In;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total; t += int64_t(gridDim.x) * blockDim.x) {
    const int r = int(t / len_o);
    const int64_t o = t - int64_t(r) * len_o;
    const T* Xr = X + int64_t(r) * S;
    const T* a = An + In * int64_t(r);
    T acc = T(0);
    for (int64_t i = 0; i < In; ++i) {
      const int64_t flat = RIGHT ? (o + len_o * i) : (i + In * o);
      acc = fma(Xr[flat], a[i], acc);
    }
    Xout[t] = acc;
  }
}

}  // namespace cpg
