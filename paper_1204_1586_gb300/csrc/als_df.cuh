// CP_ALS factor update (eq. 2.14, fast ALS of Section 4) for FP32 tensors,
// with the normal equations carried in double-float arithmetic (dfloat.cuh).
//
// For mode n, with the gradient G = Y_(n) KR from the chain kernels:
//   V        = Hadamard_{m != n} Gram_m          (Gram_m = A^(m)T A^(m))
//   V^{-1}   by Gauss-Jordan elimination of [V | I]
//   X        = G V^{-1}
//   lambda_q = ||x_q||,  a_q = x_q / lambda_q    (column normalisation)
//   Gram_n   = A^(n)T A^(n) of the stored FP32 factor (products exact, sums compensated)
// and after the last mode of a sweep the fit from R x R quantities:
//   <Y, Yhat> = sum_q lambda_q a_q^T g_q,  ||Yhat||^2 = lambda^T (Hadamard_m Gram_m) lambda,
//   fit = 1 - sqrt(max(0, ||Y||^2 - 2 <Y,Yhat> + ||Yhat||^2)) / ||Y||.
// V is symmetric positive definite whenever the Grams are (a Hadamard product
// of positive definite matrices is positive definite, Schur product theorem),
// so the elimination needs no pivoting and its pivots are the positive Schur
// complements that a Cholesky factorisation would take square roots of; a
// pivot that is not positive marks V as not positive definite, and then
// A^(n), lambda and Gram_n are left untouched and CPG_ERR_SINGULAR is
// recorded in the device status word.
// Every quantity of the normal equations is a double-float (about 48-bit
// significand) so that their conditioning is handled at FP64-like accuracy on
// the FP32 pipe; the measured FP64 rate of this GPU (64-cycle dependent FMA,
// ~680-cycle divide) would put tens of microseconds on the critical path of
// every update.
#pragma once

#include "chain.cuh"
#include "common.cuh"
#include "dfloat.cuh"

namespace cpg {

struct AlsDfArgs {
  int N, n, R;
  int64_t In;
  df* grams;              // [N][R][R] double-float Grams
  const float* G;         // In x R, column-major
  float* An;              // In x R, column-major (updated in place)
  double* lambda;         // [R]
  int* status;            // device status word
  double* fit_out;        // fit of this sweep, or nullptr
  const double* normY2;   // ||Y||^2
};

// Gram matrices of all N factors.  grid = (ceil(R*R/256), N).
__global__ void gram_all_df_kernel(const FacArgs<float> f, int R, df* grams) {
  const int m = blockIdx.y;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= R * R) return;
  const int a = t % R, b = t / R;
  const int64_t In = f.I[m];
  const float* A = f.A[m];
  df s{0.f, 0.f};
  for (int64_t i = 0; i < In; ++i) s = df_add_prod_ff(s, A[i + In * a], A[i + In * b]);
  grams[(int64_t(m) * R + b) * R + a] = s;
}

// Threads of the update block: enough for one Gauss-Jordan entry and about two
// entries of X per thread at small ranks.
inline int als_df_threads(int R) { return R <= 16 ? 512 : 1024; }

inline size_t als_df_smem_bytes(int64_t In, int R) {
  const size_t RS = size_t(R) + 1;
  // [V | I] (R x 2R), two column and two row buffers, lambda, 1/lambda, partials, X, the factor panel.
  return (2 * size_t(R) * R + 2 * size_t(R) + 4 * size_t(R) + 3 * size_t(R)) * sizeof(df) +
         size_t(In) * RS * (sizeof(df) + sizeof(float)) + 16;
}

__device__ __forceinline__ df df_warp_sum(df v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = df_add(v, df_shfl_xor(v, o));
  return v;
}

// One block of als_df_threads(R) threads.  Shared memory: als_df_smem_bytes(In, R).
// Phases (each a short dependent chain, all entries in parallel):
//   V^{-1}   R Gauss-Jordan steps on [V | I], one barrier each: step j
//            scales row j by 1 / pivot and removes column j from the other
//            rows, reading row j and column j from the side buffers written
//            by step j - 1 (so every entry updates in place);
//   X        = G V^{-1}, one output per thread;
//   lambda   warp per column; Gram: 8 lanes per (p, q) pair.
__global__ void __launch_bounds__(1024) als_update_df_kernel(const AlsDfArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int R = a.R, N = a.N, n = a.n, RS = R + 1, R2 = 2 * R;
  const int64_t In = a.In;
  df* M = reinterpret_cast<df*>(smraw);      // [V | I], row-major: M[i * 2R + c]
  df* colb = M + R * R2;                     // column j of M, two buffers of R
  df* rowb = colb + 2 * R;                   // row j of M, two buffers of 2R
  df* lam = rowb + 2 * R2;                   // lambda_q
  df* ilam = lam + R;                        // 1 / lambda_q
  df* part = ilam + R;                       // per-column partial inner products
  df* X = part + R;                          // X[i*RS + q]
  float* Af = reinterpret_cast<float*>(X + In * RS);  // G, then the stored factor: Af[i*RS + q]
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;

  for (int64_t t = tid; t < In * R; t += nt) {
    const int q = int(t / In);
    const int64_t i = t - int64_t(q) * In;
    Af[i * RS + q] = a.G[t];
  }
  for (int e = tid; e < R * R2; e += nt) {
    const int i = e / R2, c = e - i * R2;
    df v;
    if (c < R) {
      v = df_make(1.f);
      for (int m = 0; m < N; ++m)
        if (m != n) v = df_mul(v, a.grams[int64_t(m) * R * R + i + R * c]);
    } else {
      v = df_make(c - R == i ? 1.f : 0.f);
    }
    M[e] = v;
    if (c == 0) colb[i] = v;
    if (i == 0) rowb[c] = v;
  }
  __syncthreads();

  // Gauss-Jordan: after step j, columns <= j of the left half are unit
  // vectors (never read again) and the right half holds the running inverse.
  bool fail = false;
  for (int j = 0; j < R; ++j) {
    const df* col = colb + (j & 1) * R;
    const df* row = rowb + (j & 1) * R2;
    df* coln = colb + ((j + 1) & 1) * R;
    df* rown = rowb + ((j + 1) & 1) * R2;
    const df p = col[j];
    if (!(p.hi > 0.f)) {  // every thread read the same pivot
      fail = true;
      break;
    }
    const df inv = df_rcp(p);
    for (int e = tid; e < R * R2; e += nt) {
      const int i = e / R2, c = e - i * R2;
      if (c <= j) continue;
      const df v = (i == j) ? df_mul(row[c], inv) : df_sub(M[e], df_mul(df_mul(col[i], inv), row[c]));
      M[e] = v;
      if (c == j + 1) coln[i] = v;
      if (i == j + 1) rown[c] = v;
    }
    __syncthreads();
  }
  if (fail) {
    if (tid == 0) atomicCAS(a.status, 0, int(CPG_ERR_SINGULAR));
    return;
  }

  // X = G V^{-1}: X[i, q] = sum_p G[i, p] Vi[p, q], Vi[p, q] = M[p * 2R + R + q].
  for (int64_t t = tid; t < In * R; t += nt) {
    const int q = int(t / In);
    const int64_t i = t - int64_t(q) * In;
    const float* g = Af + i * RS;
    const df* vi = M + R + q;
    df s0{0.f, 0.f}, s1{0.f, 0.f};
    int p = 0;
    for (; p + 1 < R; p += 2) {
      s0 = df_add(s0, df_mul_f(vi[p * R2], g[p]));
      s1 = df_add(s1, df_mul_f(vi[(p + 1) * R2], g[p + 1]));
    }
    if (p < R) s0 = df_add(s0, df_mul_f(vi[p * R2], g[p]));
    X[i * RS + q] = df_add(s0, s1);
  }
  __syncthreads();

  // lambda_q = ||x_q||, 1/lambda_q = rsqrt(||x_q||^2).
  for (int q = warp; q < R; q += nw) {
    df s{0.f, 0.f};
    for (int64_t i = lane; i < In; i += 32) s = df_add(s, df_mul(X[i * RS + q], X[i * RS + q]));
    s = df_warp_sum(s);
    if (lane == 0) {
      if (s.hi > 0.f) {
        const df rs = df_rsqrt(s);
        lam[q] = df_mul(s, rs);
        ilam[q] = rs;
      } else {
        lam[q] = df{0.f, 0.f};
        ilam[q] = df_make(1.f);
      }
      a.lambda[q] = df_to_double(lam[q]);
    }
  }
  __syncthreads();
  for (int64_t t = tid; t < In * R; t += nt) {
    const int q = int(t / In);
    const int64_t i = t - int64_t(q) * In;
    const df v = df_mul(X[i * RS + q], ilam[q]);
    const float f = __fadd_rn(v.hi, v.lo);
    a.An[t] = f;
    Af[i * RS + q] = f;
  }
  __syncthreads();

  // Gram of the stored factor: 8 lanes per (p <= q) pair.
  df* gn = a.grams + int64_t(n) * R * R;
  const int npairs = R * (R + 1) / 2;
  const int sub = tid & 7, ngroups = nt >> 3;
  for (int pq0 = 0; pq0 < npairs; pq0 += ngroups) {
    const int pq = pq0 + (tid >> 3);
    int p = 0, q = 0;
    df s{0.f, 0.f};
    if (pq < npairs) {
      int rem = pq;
      while (rem >= R - p) {
        rem -= R - p;
        ++p;
      }
      q = p + rem;
      for (int64_t i = sub; i < In; i += 8) s = df_add_prod_ff(s, Af[i * RS + p], Af[i * RS + q]);
    }
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) s = df_add(s, df_shfl_xor(s, o, 8));
    if (pq < npairs && sub == 0) {
      gn[p + R * q] = s;
      gn[q + R * p] = s;
    }
  }
  if (a.fit_out == nullptr) return;
  __syncthreads();
  for (int q = warp; q < R; q += nw) {
    df s{0.f, 0.f};
    for (int64_t i = lane; i < In; i += 32) s = df_add_prod_ff(s, Af[i * RS + q], a.G[i + In * q]);
    s = df_warp_sum(s);
    if (lane == 0) part[q] = df_mul(lam[q], s);
  }
  __syncthreads();
  if (warp == 0) {
    df inner{0.f, 0.f}, model{0.f, 0.f};
    for (int q = lane; q < R; q += 32) inner = df_add(inner, part[q]);
    for (int t = lane; t < R * R; t += 32) {
      df v = df_mul(lam[t % R], lam[t / R]);
      for (int m = 0; m < N; ++m) v = df_mul(v, a.grams[int64_t(m) * R * R + t]);
      model = df_add(model, v);
    }
    inner = df_warp_sum(inner);
    model = df_warp_sum(model);
    if (lane == 0) {
      const df y2 = df_from_double(*a.normY2);
      df res = df_add(df_sub(y2, df_add(inner, inner)), model);
      if (!(res.hi > 0.f)) res = df{0.f, 0.f};
      const df ratio = df_mul(df_sqrt(res), df_rsqrt(y2));
      *a.fit_out = 1.0 - df_to_double(ratio);
    }
  }
}

}  // namespace cpg
