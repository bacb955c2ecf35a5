// CP_ALS update of one factor (eq. 2.14, fast ALS of Section 4), in FP64.
//
// For mode n, with the gradient G = Y_(n) KR (computed by the chain kernels):
//   V       = Hadamard_{m != n} Gram_m,     Gram_m = A^(m)T A^(m)   (FP64)
//   V       = L L^T                          (Cholesky, FP64)
//   X       = G V^{-1}                       (the pseudo-inverse of eq. 2.14 when
//                                             V is positive definite)
//   lambda_r = ||x_r||_2,  a_r^(n) = x_r / lambda_r   (column normalisation)
//   Gram_n  = A^(n)T A^(n)  of the stored (rounded) factor
// and, after the last mode of a sweep, the fit from R x R quantities:
//   <Y, Yhat> = sum_r lambda_r a_r^(n)T g_r,  ||Yhat||^2 = lambda^T (Hadamard_m Gram_m) lambda,
//   fit = 1 - sqrt(max(0, ||Y||^2 - 2 <Y,Yhat> + ||Yhat||^2)) / ||Y||.
// A V that is not positive definite leaves A^(n), lambda and Gram_n untouched
// and records CPG_ERR_SINGULAR in the device status word.
#pragma once

#include "chain.cuh"
#include "common.cuh"

namespace cpg {

template <typename T>
struct AlsArgs {
  int N, n, R;
  int64_t In;
  double* grams;          // [N][R][R]
  const T* G;             // In x R, column-major
  T* An;                  // In x R, column-major (updated in place)
  double* lambda;         // [R]
  double* X;              // In x R scratch (FP64)
  int* status;            // device status word
  double* fit_out;        // fit of this sweep, or nullptr
  const double* normY2;   // ||Y||^2
};

// Gram matrices of all N factors (FP64).  grid = (ceil(R*R/256), N).
template <typename T>
__global__ void gram_all_kernel(const FacArgs<T> f, int R, double* grams) {
  griddep_wait();
  const int m = blockIdx.y;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= R * R) return;
  const int a = t % R, b = t / R;
  const int64_t In = f.I[m];
  const T* A = f.A[m];
  double s = 0.0;
  for (int64_t i = 0; i < In; ++i) s = fma(double(A[i + In * a]), double(A[i + In * b]), s);
  grams[(int64_t(m) * R + b) * R + a] = s;
}

// Sum of the leading pass's per-CTA partial sums of y^2.  One block.
__global__ void sum_norm_kernel(const double* part, int64_t n, double* out) {
  griddep_wait();
  __shared__ double sh[32];
  double s = 0.0;
  for (int64_t t = threadIdx.x; t < n; t += blockDim.x) s += part[t];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) t += sh[w];
    *out = t;
  }
}

// Shared-memory form of the update for In * (R + 1) doubles that fit on chip:
// one block of 512 threads.  Shared memory (doubles): V / its Cholesky factor
// (R*R), the In x R panel S with row stride R+1 (G, then X, then the rounded
// factor), lambda (R), and one int flag.
//   Cholesky: one warp, lanes own rows, column by column (R <= 32), or all
//             threads, right-looking (R > 32);
//   solve   : one thread per row, forward then backward substitution;
//   norms, Gram, fit: one warp per column / per (p, q) pair, lanes over rows,
//             fixed-order shuffle reductions.
inline size_t als_smem_bytes(int64_t In, int R) {
  return (size_t(R) * R + size_t(In) * (R + 1) + R) * sizeof(double) + 16;
}

template <typename T>
__global__ void __launch_bounds__(512) als_update_smem_kernel(const AlsArgs<T> a) {
  griddep_wait();
  extern __shared__ __align__(16) double sm[];
  const int R = a.R, N = a.N, n = a.n, RS = R + 1;
  const int64_t In = a.In;
  double* V = sm;                   // V, then L (lower, V[i + R*j])
  double* S = sm + R * R;           // S[i*RS + q]
  double* lam = S + In * RS;
  int* fail = reinterpret_cast<int*>(lam + R);
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;

  for (int64_t t = tid; t < In * R; t += nt) {
    const int q = int(t / In);
    const int64_t i = t - int64_t(q) * In;
    S[i * RS + q] = double(a.G[t]);
  }
  for (int t = tid; t < R * R; t += nt) {
    double v = 1.0;
    for (int m = 0; m < N; ++m)
      if (m != n) v *= a.grams[int64_t(m) * R * R + t];
    V[t] = v;
  }
  if (tid == 0) *fail = 0;
  __syncthreads();

  // Cholesky V = L L^T.
  if (R <= 32) {
    if (warp == 0) {
      for (int j = 0; j < R; ++j) {
        double d = 0.0;
        if (lane == j) {
          d = V[j + R * j];
          for (int p = 0; p < j; ++p) d -= V[j + R * p] * V[j + R * p];
        }
        d = __shfl_sync(0xffffffffu, d, j);
        if (!(d > 0.0)) {
          if (lane == 0) *fail = 1;
          break;
        }
        const double piv = sqrt(d);
        if (lane == j) V[j + R * j] = piv;
        if (lane > j && lane < R) {
          double s = V[lane + R * j];
          for (int p = 0; p < j; ++p) s -= V[lane + R * p] * V[j + R * p];
          V[lane + R * j] = s / piv;
        }
        __syncwarp();
      }
    }
    __syncthreads();
  } else {
    for (int j = 0; j < R; ++j) {
      if (tid == 0) {
        const double d = V[j + R * j];
        if (!(d > 0.0)) *fail = 1;
        V[j + R * j] = sqrt(d > 0.0 ? d : 1.0);
      }
      __syncthreads();
      if (*fail) break;
      const double piv = V[j + R * j];
      for (int i = j + 1 + tid; i < R; i += nt) V[i + R * j] /= piv;
      __syncthreads();
      const int m = R - j - 1;  // trailing (m x m) lower triangle
      for (int t = tid; t < m * m; t += nt) {
        const int ii = j + 1 + t % m, ll = j + 1 + t / m;
        if (ll <= ii) V[ii + R * ll] -= V[ii + R * j] * V[ll + R * j];
      }
      __syncthreads();
    }
  }
  if (*fail) {
    if (tid == 0) atomicCAS(a.status, 0, int(CPG_ERR_SINGULAR));
    return;
  }

  // X = G V^{-1}: row i solves L z = g_i, then L^T x = z (in place in S).
  for (int64_t i = tid; i < In; i += nt) {
    double* x = S + i * RS;
    for (int j = 0; j < R; ++j) {
      double s = x[j];
      for (int p = 0; p < j; ++p) s -= V[j + R * p] * x[p];
      x[j] = s / V[j + R * j];
    }
    for (int j = R - 1; j >= 0; --j) {
      double s = x[j];
      for (int p = j + 1; p < R; ++p) s -= V[p + R * j] * x[p];
      x[j] = s / V[j + R * j];
    }
  }
  __syncthreads();

  // lambda_q = ||x_q||.
  for (int q = warp; q < R; q += nw) {
    double s = 0.0;
    for (int64_t i = lane; i < In; i += 32) s = fma(S[i * RS + q], S[i * RS + q], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      lam[q] = sqrt(s);
      a.lambda[q] = lam[q];
    }
  }
  __syncthreads();
  // a_q = x_q / lambda_q, stored rounded; S keeps the rounded values.
  for (int64_t t = tid; t < In * R; t += nt) {
    const int q = int(t / In);
    const int64_t i = t - int64_t(q) * In;
    const double l = lam[q];
    const T v = T(l > 0.0 ? S[i * RS + q] / l : S[i * RS + q]);
    a.An[t] = v;
    S[i * RS + q] = double(v);
  }
  __syncthreads();

  // Gram of the stored factor, one warp per (p <= q) pair.
  double* gn = a.grams + int64_t(n) * R * R;
  const int npairs = R * (R + 1) / 2;
  for (int pq = warp; pq < npairs; pq += nw) {
    int p = 0, rem = pq;
    while (rem >= R - p) {
      rem -= R - p;
      ++p;
    }
    const int q = p + rem;
    double s = 0.0;
    for (int64_t i = lane; i < In; i += 32) s = fma(S[i * RS + p], S[i * RS + q], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      gn[p + R * q] = s;
      gn[q + R * p] = s;
    }
  }
  if (a.fit_out == nullptr) return;
  __syncthreads();
  // <Y, Yhat> = sum_q lambda_q a_q^T g_q, warp per column; ||Yhat||^2 from the Grams.
  double* part = V;  // V is free now: R partial inner products
  for (int q = warp; q < R; q += nw) {
    double s = 0.0;
    for (int64_t i = lane; i < In; i += 32) s = fma(S[i * RS + q], double(a.G[i + In * q]), s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) part[q] = lam[q] * s;
  }
  __syncthreads();
  if (warp == 0) {
    double inner = 0.0, model = 0.0;
    for (int q = lane; q < R; q += 32) inner += part[q];
    for (int t = lane; t < R * R; t += 32) {
      double v = 1.0;
      for (int m = 0; m < N; ++m) v *= a.grams[int64_t(m) * R * R + t];
      model += lam[t % R] * v * lam[t / R];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      inner += __shfl_xor_sync(0xffffffffu, inner, o);
      model += __shfl_xor_sync(0xffffffffu, model, o);
    }
    if (lane == 0) {
      const double y2 = *a.normY2;
      const double res = y2 - 2.0 * inner + model;
      *a.fit_out = 1.0 - sqrt(res > 0.0 ? res : 0.0) / sqrt(y2);
    }
  }
}

// Global-memory form for panels that do not fit on chip.
// One block of 256 threads.  Shared memory: 3 * R * R doubles.
template <typename T>
__global__ void __launch_bounds__(256) als_update_kernel(const AlsArgs<T> a) {
  griddep_wait();
  extern __shared__ __align__(16) double sm[];
  const int R = a.R, N = a.N, n = a.n;
  const int64_t In = a.In;
  double* V = sm;             // V, then its Cholesky factor L (lower) in place
  double* Li = sm + R * R;    // L^{-1} (lower)
  double* Vi = sm + 2 * R * R;  // V^{-1}
  __shared__ int fail;
  const int tid = threadIdx.x, nt = blockDim.x;

  for (int t = tid; t < R * R; t += nt) {
    double v = 1.0;
    for (int m = 0; m < N; ++m)
      if (m != n) v *= a.grams[int64_t(m) * R * R + t];
    V[t] = v;  // V[row + R*col], symmetric
  }
  if (tid == 0) fail = 0;
  __syncthreads();

  // Left-looking Cholesky, column j at a time: V = L L^T, L stored in V's lower part.
  for (int j = 0; j < R; ++j) {
    if (tid == 0) {
      double d = V[j + R * j];
      for (int p = 0; p < j; ++p) d -= V[j + R * p] * V[j + R * p];
      if (!(d > 0.0)) fail = 1;
      V[j + R * j] = sqrt(d > 0.0 ? d : 1.0);
    }
    __syncthreads();
    if (fail) break;
    const double djj = V[j + R * j];
    for (int i = j + 1 + tid; i < R; i += nt) {
      double s = V[i + R * j];
      for (int p = 0; p < j; ++p) s -= V[i + R * p] * V[j + R * p];
      V[i + R * j] = s / djj;
    }
    __syncthreads();
  }
  if (fail) {
    if (tid == 0) atomicCAS(a.status, 0, int(CPG_ERR_SINGULAR));
    return;
  }

  // L^{-1}: column c by forward substitution (one thread per column).
  for (int c = tid; c < R; c += nt) {
    for (int i = 0; i < R; ++i) Li[i + R * c] = 0.0;
    Li[c + R * c] = 1.0 / V[c + R * c];
    for (int i = c + 1; i < R; ++i) {
      double s = 0.0;
      for (int p = c; p < i; ++p) s += V[i + R * p] * Li[p + R * c];
      Li[i + R * c] = -s / V[i + R * i];
    }
  }
  __syncthreads();
  // V^{-1} = L^{-T} L^{-1}.
  for (int t = tid; t < R * R; t += nt) {
    const int p = t % R, q = t / R;
    const int lo = p > q ? p : q;
    double s = 0.0;
    for (int i = lo; i < R; ++i) s += Li[i + R * p] * Li[i + R * q];
    Vi[t] = s;
  }
  __syncthreads();

  // X = G V^{-1}  (X[i, q] = sum_p G[i, p] Vi[p, q]).
  for (int64_t t = tid; t < In * R; t += nt) {
    const int q = int(t / In);
    const int64_t i = t - int64_t(q) * In;
    double s = 0.0;
    for (int p = 0; p < R; ++p) s = fma(double(a.G[i + In * p]), Vi[p + R * q], s);
    a.X[t] = s;
  }
  __syncthreads();
  // lambda_r = ||x_r||, column normalisation (one thread per column, fixed order).
  double* lam = Li;  // reuse
  for (int q = tid; q < R; q += nt) {
    double s = 0.0;
    for (int64_t i = 0; i < In; ++i) {
      const double x = a.X[i + In * q];
      s = fma(x, x, s);
    }
    lam[q] = sqrt(s);
    a.lambda[q] = lam[q];
  }
  __syncthreads();
  for (int64_t t = tid; t < In * R; t += nt) {
    const int q = int(t / In);
    const double l = lam[q];
    a.An[t] = T(l > 0.0 ? a.X[t] / l : a.X[t]);
  }
  __syncthreads();
  // Gram of the stored factor.
  double* gn = a.grams + int64_t(n) * R * R;
  for (int t = tid; t < R * R; t += nt) {
    const int p = t % R, q = t / R;
    if (p > q) continue;
    double s = 0.0;
    for (int64_t i = 0; i < In; ++i) s = fma(double(a.An[i + In * p]), double(a.An[i + In * q]), s);
    gn[p + R * q] = s;
    gn[q + R * p] = s;
  }
  if (a.fit_out == nullptr) return;
  __syncthreads();
  if (tid < 32) {
    // <Y, Yhat> and ||Yhat||^2 in one warp, fixed order.
    double inner = 0.0, model = 0.0;
    for (int q = tid; q < R; q += 32) {
      double s = 0.0;
      for (int64_t i = 0; i < In; ++i) s = fma(double(a.An[i + In * q]), double(a.G[i + In * q]), s);
      inner += lam[q] * s;
    }
    for (int t = tid; t < R * R; t += 32) {
      double v = 1.0;
      for (int m = 0; m < N; ++m) v *= a.grams[int64_t(m) * R * R + t];
      model += lam[t % R] * v * lam[t / R];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      inner += __shfl_xor_sync(0xffffffffu, inner, o);
      model += __shfl_xor_sync(0xffffffffu, model, o);
    }
    if (tid == 0) {
      const double y2 = *a.normY2;
      const double res = y2 - 2.0 * inner + model;
      *a.fit_out = 1.0 - sqrt(res > 0.0 ? res : 0.0) / sqrt(y2);
    }
  }
}

}  // namespace cpg
