// Consumers of the CP gradient (Section 2.2) that need only G^(n) = Y_(n) KR,
// the factors and their Grams:
//   model_term_kernel  the cost gradient of eq. 2.13 with its model term,
//                      G^(n) <- G^(n) - A^(n) Gamma^(n), Gamma^(n) = Hadamard_{m != n}
//                      A^(m)T A^(m), for every mode in one launch, and optionally
//                      the all-at-once first-order step of eq. 2.15,
//                      A^(n) <- A^(n) + eta G^(n) (G is -1/2 dD/dA, eq. 2.12);
//   mu_update_kernel   the multiplicative nonnegative update of eq. 2.18,
//                      A^(n) <- A^(n) * G^(n) / (A^(n) Gamma^(n)), elementwise
//                      (an entry whose denominator is not positive is left as is);
//   ntf_fit_kernel     the fit of a nonnegative model after a sweep.
// The R x R products and row sums run in FP64 for FP32 and FP64 data alike:
// the work is I_n R^2 multiply-adds per mode, far from any pipe's limit.
#pragma once

#include "chain.cuh"
#include "common.cuh"

namespace cpg {

constexpr int kRowsPerBlock = 8;

template <typename T>
struct ModelTermArgs {
  int N, R;
  int64_t I[kMaxOrder];
  T* A[kMaxOrder];        // factors (updated in place by the step)
  T* G[kMaxOrder];        // in: Y_(n) KR; out: the cost gradient of eq. 2.13
  const double* gammas;   // [N][R][R] Gamma^(n) of the factors before the step
  double eta;             // step length of eq. 2.15
  int step;               // 1: also A <- A + eta G
};

// Gamma = Hadamard_{m != n} Gram_m into g ([R][R]), by the block.
__device__ __forceinline__ void hadamard_of_grams(const double* grams, int N, int n, int R, double* g) {
  for (int t = threadIdx.x; t < R * R; t += blockDim.x) {
    double v = 1.0;
    for (int m = 0; m < N; ++m)
      if (m != n) v *= grams[int64_t(m) * R * R + t];
    g[t] = v;
  }
}

// Gamma^(n) = Hadamard_{m != n} Gram_m for every mode into gammas ([N][R][R]).
// grid = (ceil(R^2 / 256), N), 256 threads.
__global__ void gamma_all_kernel(const double* grams, int N, int R, double* gammas) {
  griddep_wait();
  const int n = blockIdx.y;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= R * R) return;
  double v = 1.0;
  for (int m = 0; m < N; ++m)
    if (m != n) v *= grams[int64_t(m) * R * R + t];
  gammas[int64_t(n) * R * R + t] = v;
}

// grid = (ceil(max I_n / 8), N), 256 threads, shared memory 8 R doubles (the
// block's rows of A^(n), read before any thread writes them); Gamma^(n) is read
// through the cache.
template <typename T>
__global__ void __launch_bounds__(256) model_term_kernel(const ModelTermArgs<T> a) {
  griddep_wait();
  extern __shared__ double sm_mt[];
  const int n = blockIdx.y, R = a.R;
  const int64_t In = a.I[n], i0 = int64_t(blockIdx.x) * kRowsPerBlock;
  if (i0 >= In) return;  // the whole block
  const double* gam = a.gammas + int64_t(n) * R * R;  // Gamma^(n)[p][r] at p + R r
  double* rows = sm_mt;                               // A^(n)[i0 + i][p] at i + 8 p
  const T* An = a.A[n];
  for (int t = threadIdx.x; t < kRowsPerBlock * R; t += blockDim.x) {
    const int i = t % kRowsPerBlock, p = t / kRowsPerBlock;
    rows[t] = (i0 + i < In) ? double(An[i0 + i + In * p]) : 0.0;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < kRowsPerBlock * R; t += blockDim.x) {
    const int i = t % kRowsPerBlock, r = t / kRowsPerBlock;
    const int64_t gi = i0 + i;
    if (gi >= In) continue;
    double d = 0.0;
    for (int p = 0; p < R; ++p) d = fma(rows[i + kRowsPerBlock * p], gam[p + R * r], d);
    const double g = double(a.G[n][gi + In * r]) - d;
    a.G[n][gi + In * r] = T(g);
    if (a.step) a.A[n][gi + In * r] = T(rows[t] + a.eta * g);
  }
}

template <typename T>
struct MuArgs {
  int N, n, R;
  int64_t In;
  const double* grams;  // [N][R][R]
  const T* G;           // Y_(n) KR, In x R column-major
  T* An;                // In x R column-major, updated in place
};

// grid = ceil(In / 8), 256 threads, shared memory (R + 8) R doubles (R <= 64).
template <typename T>
__global__ void __launch_bounds__(256) mu_update_kernel(const MuArgs<T> a) {
  griddep_wait();
  extern __shared__ double sm_mu[];
  const int R = a.R;
  const int64_t In = a.In, i0 = int64_t(blockIdx.x) * kRowsPerBlock;
  double* gam = sm_mu;
  double* rows = gam + R * R;
  hadamard_of_grams(a.grams, a.N, a.n, R, gam);
  for (int t = threadIdx.x; t < kRowsPerBlock * R; t += blockDim.x) {
    const int i = t % kRowsPerBlock, p = t / kRowsPerBlock;
    rows[t] = (i0 + i < In) ? double(a.An[i0 + i + In * p]) : 0.0;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < kRowsPerBlock * R; t += blockDim.x) {
    const int i = t % kRowsPerBlock, r = t / kRowsPerBlock;
    const int64_t gi = i0 + i;
    if (gi >= In) continue;
    double d = 0.0;
    for (int p = 0; p < R; ++p) d = fma(rows[i + kRowsPerBlock * p], gam[p + R * r], d);
    if (d > 0.0) a.An[gi + In * r] = T(rows[t] * double(a.G[gi + In * r]) / d);
  }
}

// fit = 1 - sqrt(max(0, ||Y||^2 - 2 <Y, Yhat> + ||Yhat||^2)) / ||Y|| of the
// model sum_r a_r^(1) o ... o a_r^(N), with <Y, Yhat> = sum_ir A^(n)_ir G_ir
// (the last mode's gradient) and ||Yhat||^2 = sum_pq Hadamard_m Gram_m.
// One block of 256 threads.
template <typename T>
__global__ void __launch_bounds__(256) ntf_fit_kernel(int N, int R, int64_t In, const T* An, const T* G,
                                                       const double* grams, const double* normY2, double* fit) {
  griddep_wait();
  __shared__ double sh[2][8];
  double inner = 0.0, model = 0.0;
  for (int64_t t = threadIdx.x; t < In * R; t += blockDim.x) inner = fma(double(An[t]), double(G[t]), inner);
  for (int t = threadIdx.x; t < R * R; t += blockDim.x) {
    double v = 1.0;
    for (int m = 0; m < N; ++m) v *= grams[int64_t(m) * R * R + t];
    model += v;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    inner += __shfl_xor_sync(0xffffffffu, inner, o);
    model += __shfl_xor_sync(0xffffffffu, model, o);
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    sh[0][w] = inner;
    sh[1][w] = model;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int k = 0; k < int(blockDim.x >> 5); ++k) {
      a += sh[0][k];
      b += sh[1][k];
    }
    const double y2 = *normY2;
    *fit = 1.0 - sqrt(fmax(0.0, y2 - 2.0 * a + b)) / sqrt(y2);
  }
}

}  // namespace cpg
