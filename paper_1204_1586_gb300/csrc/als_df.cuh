// CP_ALS factor update (eq. 2.14, fast ALS of Section 4) for FP32 tensors,
// with the normal equations carried in double-float arithmetic (dfloat.cuh).
//
// For mode n, with the gradient G = Y_(n) KR from the chain:
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
// the FP32 pipe; the sums of products G V^{-1}, ||x_q||^2 and Gram_n are
// accumulated by the compensated dot product of dfloat.cuh, as accurate at
// about half the instructions and a far shorter dependent chain.  The
// measured FP64 rate of this GPU (64-cycle dependent FMA, ~680-cycle divide)
// would put tens of microseconds on the critical path of every update.
//
// The update runs inside the kernel that produces G (als_mode_df_kernel):
// every CTA but one computes its share of G (a finishing contraction or a
// recursion of the chain, chain.cuh) while the extra CTA forms V and V^{-1}
// (they need only the Grams, final before the launch); the CTA that finishes
// last, found by an atomic ticket after a memory fence (no CTA ever waits for
// another), then updates the factor.  One launch per mode, no second stream.
#pragma once

#include "chain.cuh"
#include "common.cuh"
#include "dfloat.cuh"

namespace cpg {

struct AlsDfArgs {
  int N, n, R;
  int64_t In;
  df* grams;              // [N][R][R] double-float Grams
  df* V;                  // [R][R] V of this mode (written by the inverse CTA)
  df* Vi;                 // [R][R] V^{-1}; Vi[0] = 0 marks a V that is not positive definite
  const float* G;         // In x R, column-major (read through L2: other CTAs wrote it)
  float* An;              // In x R, column-major (updated in place)
  double* lambda;         // [R]
  int* status;            // device status word
  double* fit_out;        // fit of this sweep, or nullptr
  const double* normY2;   // ||Y||^2
};

// Gram matrices of all N factors.  grid = (ceil(R*R/256), N).
__global__ void gram_all_df_kernel(const FacArgs<float> f, int R, df* grams) {
  griddep_wait();
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

// ---- V and V^{-1} of one mode, by one block ----------------------------------------
// V = Hadamard_{m != n} Gram_m into V_out and V^{-1} into Vi_out ([R][R],
// symmetric, Vi_out[p + R q]; global memory), by Gauss-Jordan elimination of
// [V | I] in shared `work` ((2 R^2 + 6 R) double-floats).  Step j touches only
// the R columns j+1 .. R+j (earlier left columns are finished unit vectors,
// later right columns are still identity columns) and reads row j and column
// j from side buffers written by step j - 1, so every entry updates in place
// with one barrier per step; when the R x R active block fits the block's
// threads each thread keeps its entry's row and column offset for all steps.
// Returns false (on every thread, Vi_out unwritten) when a pivot is not
// positive.
__device__ bool df_inverse_block(const df* grams, int N, int n, int R, df* V_out, df* Vi_out, df* work) {
  const int R2 = 2 * R;
  df* M = work;            // [V | I], row-major: M[i * 2R + c]
  df* colb = M + R * R2;   // column j of M, two buffers of R
  df* rowb = colb + 2 * R; // row j of M, two buffers of 2R
  const int tid = threadIdx.x, nt = blockDim.x;

  for (int t = tid; t < R * R; t += nt) {
    df g[kMaxOrder];
#pragma unroll
    for (int m = 0; m < kMaxOrder; ++m)
      if (m < N && m != n) g[m] = grams[m * R * R + t];  // every load in flight before the products
    df v = df_make(1.f);
#pragma unroll
    for (int m = 0; m < kMaxOrder; ++m)
      if (m < N && m != n) v = df_mul(v, g[m]);
    const int i = t % R, c = t / R;  // V is symmetric: V[i][c]
    V_out[t] = v;
    M[i * R2 + c] = v;
    M[i * R2 + R + c] = df_make(i == c ? 1.f : 0.f);
    if (c == 0) colb[i] = v;  // column 0 for step 0
    if (i == 0) rowb[c] = v;  // row 0, left half
  }
  // Column R + j of row j still holds the identity's 1 when step j first
  // touches it, and no earlier step writes that side-buffer slot: preset it.
  for (int j = tid; j < R; j += nt) rowb[(j & 1) * R2 + R + j] = df_make(1.f);
  __syncthreads();

  const bool one = R * R <= nt;  // at most one active entry per thread
  const int ei = tid / R, eo = tid - ei * R;
  for (int j = 0; j < R; ++j) {
    const df* col = colb + (j & 1) * R;
    const df* row = rowb + (j & 1) * R2;
    df* coln = colb + ((j + 1) & 1) * R;
    df* rown = rowb + ((j + 1) & 1) * R2;
    const df p = col[j];
    if (!(p.hi > 0.f)) return false;  // every thread read the same pivot
    const df inv = df_rcp(p);
    auto step = [&](int i, int c) {
      const df v = (i == j) ? df_mul(row[c], inv) : df_sub(M[i * R2 + c], df_mul(df_mul(col[i], inv), row[c]));
      M[i * R2 + c] = v;
      if (c == j + 1) coln[i] = v;
      if (i == j + 1) rown[c] = v;
    };
    if (one) {
      if (tid < R * R) step(ei, j + 1 + eo);
    } else {
      for (int e = tid; e < R * R; e += nt) {
        const int i = e / R;
        step(i, j + 1 + (e - i * R));
      }
    }
    __syncthreads();
  }
  for (int t = tid; t < R * R; t += nt) {
    const int p = t % R, q = t / R;
    Vi_out[t] = M[p * R2 + R + q];
  }
  return true;
}

// ---- the update of one mode, by one block ---------------------------------------
constexpr int kModeThreads = 512;

// Shared memory of the update (V^{-1}, V, Gram_n, lambda, partials; then X
// (double-float), G and the new factor (floats), all In x (R + 1)) and of the
// inverse ([V | I] and the pivot row/column buffers); the mode kernel takes
// the larger.
inline size_t als_df_smem_bytes(int64_t In, int R) {
  const size_t RS = size_t(R) + 1, R2 = size_t(R) * R;
  const size_t update = (3 * R2 + 2 * size_t(R)) * sizeof(df) + size_t(In) * RS * (sizeof(df) + 2 * sizeof(float));
  const size_t inverse = (2 * R2 + 6 * size_t(R)) * sizeof(df);
  return (update > inverse ? update : inverse) + 16;
}

__device__ __forceinline__ df df_warp_sum(df v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = df_add(v, df_shfl_xor(v, o));
  return v;
}

// Phases (each a short dependent chain, all entries in parallel):
//   load     V^{-1}, V (from the inverse CTA), G;
//   X        = G V^{-1}, one output per thread (compensated dot product);
//   lambda   warp per column (compensated sum of squares); a_q = x_q / lambda_q;
//   Gram_n   8 lanes per (p, q) pair (compensated dot products);
//   fit      <Y, Yhat> = sum_q lambda_q <a_q, g_q>,
//            ||Yhat||^2 = lambda^T (V * Gram_n) lambda.
__device__ void als_update_block(const AlsDfArgs& a, unsigned char* smraw) {
  const int R = a.R, n = a.n, RS = R + 1;
  const int In = int(a.In);  // In * (R + 1) fits the shared-memory budget, far below 2^31
  df* Vis = reinterpret_cast<df*>(smraw);    // V^{-1}[p][q] at p + R q
  df* Vs = Vis + R * R;                      // V
  df* gn = Vs + R * R;                       // Gram_n of the new factor
  df* lam = gn + R * R;                      // lambda_q
  df* part = lam + R;                        // lambda_q <a_q, g_q>
  df* X = part + R;                          // X[i*RS + q]
  float* Gs = reinterpret_cast<float*>(X + In * RS);  // G[i*RS + p]
  float* Fs = Gs + In * RS;                            // new factor[i*RS + q]
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  const bool want_fit = a.fit_out != nullptr;

  // Written by other CTAs of this launch: read through L2.
  for (int t = tid; t < R * R; t += nt) {
    const float2 vi = __ldcg(reinterpret_cast<const float2*>(a.Vi) + t);
    const float2 v = __ldcg(reinterpret_cast<const float2*>(a.V) + t);
    Vis[t] = df{vi.x, vi.y};
    Vs[t] = df{v.x, v.y};
  }
  // Every load of a round in flight before its stores.
  constexpr int kLoadUnroll = 4;
  for (int t0 = tid; t0 < In * R; t0 += kLoadUnroll * nt) {
    float v[kLoadUnroll];
#pragma unroll
    for (int k = 0; k < kLoadUnroll; ++k) {
      const int t = t0 + k * nt;
      v[k] = (t < In * R) ? __ldcg(a.G + t) : 0.f;
    }
#pragma unroll
    for (int k = 0; k < kLoadUnroll; ++k) {
      const int t = t0 + k * nt;
      if (t < In * R) {
        const int q = t / In, i = t - q * In;
        Gs[i * RS + q] = v[k];
      }
    }
  }
  __syncthreads();
  if (!(Vis[0].hi != 0.f)) return;  // V was not positive definite: leave this mode untouched

  // X = G V^{-1}: X[i, q] = sum_p G[i, p] Vi[p, q], one output per thread
  // (compensated: as accurate as a double-float evaluation).
  for (int t = tid; t < In * R; t += nt) {
    const int q = t / In, i = t - q * In;
    const float* g = Gs + i * RS;
    const df* vi = Vis + R * q;
    dot2 acc;
    for (int p = 0; p < R; ++p) acc.add_fd(g[p], vi[p]);
    X[i * RS + q] = acc.value();
  }
  __syncthreads();

  // lambda_q = ||x_q||, a_q = x_q / lambda_q (1/lambda_q = rsqrt(||x_q||^2)), warp per column.
  for (int q = warp; q < R; q += nw) {
    dot2 sq;
    for (int i = lane; i < In; i += 32) sq.add_sq(X[i * RS + q]);
    const df ss = df_warp_sum(sq.value());
    df lq, il;
    if (ss.hi > 0.f) {
      il = df_rsqrt(ss);
      lq = df_mul(ss, il);
    } else {
      lq = df{0.f, 0.f};
      il = df_make(1.f);
    }
    dot2 ipa;
    for (int r = lane; r < In; r += 32) {
      const df v = df_mul(X[r * RS + q], il);
      const float f = __fadd_rn(v.hi, v.lo);
      a.An[r + In * q] = f;
      Fs[r * RS + q] = f;
      if (want_fit) ipa.add_ff(f, Gs[r * RS + q]);
    }
    df ip{0.f, 0.f};
    if (want_fit) ip = df_warp_sum(ipa.value());
    if (lane == 0) {
      lam[q] = lq;
      part[q] = df_mul(lq, ip);
      a.lambda[q] = df_to_double(lq);
    }
  }
  __syncthreads();

  // Gram of the stored factor: 8 lanes per (p <= q) pair.
  df* gout = a.grams + int64_t(n) * R * R;
  const int npairs = R * (R + 1) / 2;
  const int sub = tid & 7, ngroups = nt >> 3;
  for (int pq0 = 0; pq0 < npairs; pq0 += ngroups) {
    const int pq = pq0 + (tid >> 3);
    int p = 0, q = 0;
    dot2 acc;
    if (pq < npairs) {
      int rem = pq;
      while (rem >= R - p) {
        rem -= R - p;
        ++p;
      }
      q = p + rem;
      for (int i = sub; i < In; i += 8) acc.add_ff(Fs[i * RS + p], Fs[i * RS + q]);
    }
    df s = acc.value();
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) s = df_add(s, df_shfl_xor(s, o, 8));
    if (pq < npairs && sub == 0) {
      gout[p + R * q] = s;
      gout[q + R * p] = s;
      gn[p + R * q] = s;
      gn[q + R * p] = s;
    }
  }
  if (!want_fit) return;
  __syncthreads();

  if (warp == 0) {
    df inner{0.f, 0.f}, model{0.f, 0.f};
    for (int q = lane; q < R; q += 32) inner = df_add(inner, part[q]);
    for (int t = lane; t < R * R; t += 32)
      model = df_add(model, df_mul(df_mul(lam[t % R], lam[t / R]), df_mul(Vs[t], gn[t])));
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

// ---- one mode: G, then the update -------------------------------------------------
struct AlsModeArgs {
  SegDot<float> sd;        // produces G (sd.out == u.G): a finishing contraction or a recursion
  AlsDfArgs u;             // the update of mode u.n
  unsigned int* ticket;    // zero on entry; the last CTA resets it
};

// grid = (CTAs of the segmented dot) + 1 of kModeThreads threads, dynamic
// shared memory als_df_smem_bytes(In, R).  LPO = lanes per output of the
// segmented dot, or 0 for its tiled form (chain.cuh); the last CTA of the
// grid forms V and V^{-1}.
template <int LPO>
__global__ void __launch_bounds__(kModeThreads) als_mode_df_kernel(const AlsModeArgs p) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ unsigned int s_ticket;
  griddep_wait();
  if (blockIdx.x == gridDim.x - 1) {
    const AlsDfArgs& u = p.u;
    const int R = u.R;
    const bool ok = df_inverse_block(u.grams, u.N, u.n, R, u.V, u.Vi, reinterpret_cast<df*>(smraw));
    if (!ok) {
      for (int t = threadIdx.x; t < R * R; t += blockDim.x) u.Vi[t] = df{0.f, 0.f};
      if (threadIdx.x == 0) atomicCAS(u.status, 0, int(CPG_ERR_SINGULAR));
    }
  } else if constexpr (LPO == 0) {
    seg_dot_tiled_run<float>(p.sd, blockIdx.x);
  } else {
    seg_dot_run<float, LPO>(p.sd, blockIdx.x * int64_t(blockDim.x) + threadIdx.x);
  }
  // Publish this CTA's outputs, then take a ticket: the CTA with the last
  // ticket sees every other CTA's outputs and runs the update.
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_ticket = atomicAdd(p.ticket, 1u);
  __syncthreads();
  if (s_ticket != gridDim.x - 1) return;
  __threadfence();
  if (threadIdx.x == 0) *p.ticket = 0u;  // ready for the next launch on this stream
  // No early trigger: the next kernel launches when this one completes (an
  // early launch measured slower, 209.4 against 207.6 us per 100^4 sweep).
  als_update_block(p.u, smraw);
}

}  // namespace cpg
