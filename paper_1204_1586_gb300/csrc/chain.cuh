// Per-mode contractions of Algorithm 2 that follow the leading pass.
//
// The partial tensors of Section 3.3 are held rank-major, X[r][flat], with
// flat the column-major index over the modes X still carries:
//   right side  R^(n): modes [0, n),   flat = a + Alo * i   (i = last mode)
//   left side   L^(n): modes [n, N),   flat = i + In  * b   (i = first mode)
// where a runs over the modes below i and b over the modes above i.
//
// Both per-mode operations are segmented dot products over one index of X:
//   finishing contraction (cp_gradient 'right', line 19 / eq. 3.12, and
//   'left', line 20 / eq. 3.16):
//       g_r^(n)[i] = sum_o X[r][flat(o, i)] * kr[r][o]
//   recursion (steps 11 / eq. 3.20 and 15 / eq. 3.22):
//       X'[r][o]   = sum_i X[r][flat(o, i)] * A^(n)[i, r]
// where kr is the Kronecker vector of the other remaining modes (eq. 3.3).
// In both, output t = a + D * r reads X[r * S + a * astep + u * ustep] for
// u < inner, weighted by w[r * wlen + u] (w = kr, or the factor's column).
//
// The first use of R^(k) / L^(k+1) reads the leading pass's partial sums
// (nparts slices) and adds them in a fixed order (optionally storing the
// sum), so results are deterministic run to run.
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
  griddep_launch();  // the kernels that follow may start launching (they wait for this one)
  griddep_wait();
  const int64_t total = len * R;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total; t += int64_t(gridDim.x) * blockDim.x) {
    const int r = int(t / len);
    const int64_t o = t - int64_t(r) * len;
    out[t] = kr_entry<T>(f.A, f.I, mb, me, o, r);
  }
}

// Khatri-Rao rows of a leading pass (W_R of eq. 3.10 or W_L of eq. 3.9), built
// once per pass for one rank group (ranks r0 .. r0 + RT - 1) in the padded
// layouts the CUDA-core leading kernel copies per stage (LeadArgs::wpre_r /
// wpre_l):
//   rank_major = 0: out[o * RT + r],                        o < len_pad
//   rank_major = 1: out[(o / TJ) * RT * TJ + r * TJ + o % TJ]
// Entry (o, r) is the factor row of the first mode times the Kronecker-table
// entry of the others, the product the kernel would form itself (KrRows),
// and zero for o >= len or r0 + r >= R.  The kernels that follow may launch
// at once: they wait for this one before they read the rows.
template <typename T>
__global__ void kr_rows_kernel(T* __restrict__ out, const KrRows<T> kr, int64_t len, int64_t len_pad, int RT, int r0,
                               int R, int TJ, int rank_major) {
  griddep_launch();
  griddep_wait();
  const int64_t total = len_pad * RT, tile = int64_t(RT) * TJ;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total; t += int64_t(gridDim.x) * blockDim.x) {
    int64_t o;
    int r;
    if (rank_major) {
      const int64_t tb = t / tile, w = t - tb * tile;
      r = int(w / TJ);
      o = tb * TJ + (w - int64_t(r) * TJ);
    } else {
      o = t / RT;
      r = int(t - o * RT);
    }
    T v = T(0);
    if (o < len && r0 + r < R) {
      if (kr.A == nullptr) {
        v = T(1);
      } else {
        const uint32_t q = kr.d.div(uint32_t(o)), i = uint32_t(o) - q * kr.d.d;
        const T fa = kr.A[i + int64_t(kr.d.d) * (r0 + r)];
        const T fq = (kr.Q != nullptr) ? kr.Q[q + kr.ldq * (r0 + r)] : T(1);
        v = fa * fq;
      }
    }
    out[t] = v;
  }
}

// Y_(1:k) (J rows, pitch J) copied into a buffer whose columns start on
// 16-byte boundaries (pitch ldd >= J), so that the leading passes can take TMA
// tiles of a tensor whose own row pitch is not a multiple of 16 bytes.  The
// rows J .. ldd-1 are never read (the tiles' out-of-range rows read as zero).
template <typename T>
__global__ void pitch_copy_kernel(T* __restrict__ dst, int64_t ldd, const T* __restrict__ src, int64_t J, int64_t K) {
  griddep_wait();
  for (int64_t c = blockIdx.x; c < K; c += gridDim.x) {
    const T* s = src + J * c;
    T* d = dst + ldd * c;
#pragma unroll 8
    for (int64_t j = threadIdx.x; j < J; j += blockDim.x) d[j] = s[j];
  }
}

template <typename T>
struct SegDot {
  const T* X;             // [nparts][R][S]
  int nparts;
  int64_t part_stride;    // R * S
  int64_t S;              // elements of X per rank column
  int64_t D;              // outputs per rank column
  int64_t astep, ustep;   // X offset of output a and of reduction index u
  int64_t inner;          // reduction length
  const T* w;             // weights [r][u] (ld = wlen), or nullptr for all ones
  int64_t wlen;
  T* out;                 // out[a + D * r]
  T* Xred;                // if set (and nparts > 1): the summed X is stored here
  int R;
};

// X[0] + X[1] + ... + X[nparts-1] (the partial sums of a leading pass,
// `stride` elements apart, n elements each) into out by a grid over the whole
// GPU, added exactly as the segmented dot products below add them (from zero,
// in the order q = 0, 1, ..., in batches of 8), so the chain's results do not
// change when it reads the sum instead of the parts.
template <typename T>
__global__ void sum_parts_kernel(T* __restrict__ out, const T* __restrict__ X, int nparts, int64_t stride, int64_t n) {
  griddep_wait();
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < n; t += int64_t(gridDim.x) * blockDim.x) {
    T x = T(0);
    for (int q0 = 0; q0 < nparts; q0 += 8) {
      T v[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) v[e] = (q0 + e < nparts) ? __ldcs(X + (q0 + e) * stride + t) : T(0);
#pragma unroll
      for (int e = 0; e < 8; ++e) x += v[e];
    }
    out[t] = x;
  }
}

// LPO lanes cooperate on one output; lanes stride the reduction index.  The
// partial sums of an element are loaded in batches of 8 ahead of their
// additions (which keep the fixed order q = 0, 1, ...), so that the loads
// overlap instead of each waiting for the previous add.  gid = global thread
// index; every lane of a warp must call it (shuffle reduction).
template <typename T, int LPO>
__device__ __forceinline__ void seg_dot_run(const SegDot<T>& p, int64_t gid) {
  const int64_t t = gid / LPO;
  const int sub = int(gid % LPO);
  const int64_t nout = p.D * p.R;
  const bool live = t < nout;
  const T* __restrict__ X = p.X;
  T* __restrict__ Xred = p.Xred;
  const int nparts = p.nparts;
  const int64_t pstride = p.part_stride;
  T acc = T(0);
  if (live) {
    const int r = int(t / p.D);
    const int64_t a = t - int64_t(r) * p.D;
    const int64_t base = int64_t(r) * p.S + a * p.astep;
    const T* __restrict__ w = p.w ? p.w + int64_t(r) * p.wlen : nullptr;
#pragma unroll 2
    for (int64_t u = sub; u < p.inner; u += LPO) {
      const int64_t off = base + u * p.ustep;
      T x;
      if (nparts == 1) {
        x = X[off];
      } else {
        x = T(0);
        for (int q0 = 0; q0 < nparts; q0 += 8) {
          T v[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) v[e] = (q0 + e < nparts) ? X[(q0 + e) * pstride + off] : T(0);
#pragma unroll
          for (int e = 0; e < 8; ++e) x += v[e];
        }
        if (Xred) Xred[off] = x;
      }
      acc = w ? fma(x, w[u], acc) : acc + x;
    }
  }
  if constexpr (LPO > 1) {
#pragma unroll
    for (int s = LPO / 2; s > 0; s >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, s, LPO);
  }
  if (live && sub == 0) p.out[t] = acc;
}

template <typename T, int LPO>
__global__ void __launch_bounds__(256) seg_dot_kernel(const SegDot<T> p) {
  griddep_wait();
  seg_dot_run<T, LPO>(p, blockIdx.x * int64_t(blockDim.x) + threadIdx.x);
}

// The same product when consecutive outputs are consecutive in X (astep == 1)
// and the reduction index is strided (ustep > 1): lanes take 32 consecutive
// outputs of one rank column, so every load of a warp is one contiguous run,
// and the kSegWarps warps of a block take interleaved slices of the
// reduction, summed through shared memory in a fixed order.  Block `blk` of
// seg_tiled_blocks(p) covers outputs [32 g, 32 g + 32) of rank r, with
// g = blk % groups and r = blk / groups.
constexpr int kSegWarps = 16;

template <typename T>
inline int64_t seg_tiled_groups(const SegDot<T>& p) {
  return (p.D + 31) / 32;
}
template <typename T>
inline int64_t seg_tiled_blocks(const SegDot<T>& p) {
  return seg_tiled_groups(p) * p.R;
}

template <typename T>
__device__ __forceinline__ void seg_dot_tiled_run(const SegDot<T>& p, int64_t blk) {
  __shared__ T red[kSegWarps][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t groups = (p.D + 31) / 32;
  const int r = int(blk / groups);
  const int64_t a = (blk - int64_t(r) * groups) * 32 + lane;
  const bool live = a < p.D;
  const T* __restrict__ X = p.X;
  const T* __restrict__ w = p.w ? p.w + int64_t(r) * p.wlen : nullptr;
  const int nparts = p.nparts;
  T acc = T(0);
  if (live) {
    const int64_t base = int64_t(r) * p.S + a;
#pragma unroll 4
    for (int64_t u = warp; u < p.inner; u += kSegWarps) {
      const int64_t off = base + u * p.ustep;
      T x;
      if (nparts == 1) {
        x = X[off];
      } else {
        x = T(0);
        for (int q0 = 0; q0 < nparts; q0 += 8) {
          T v[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) v[e] = (q0 + e < nparts) ? X[(q0 + e) * p.part_stride + off] : T(0);
#pragma unroll
          for (int e = 0; e < 8; ++e) x += v[e];
        }
        if (p.Xred) p.Xred[off] = x;
      }
      acc = w ? fma(x, w[u], acc) : acc + x;
    }
  }
  red[warp][lane] = acc;
  __syncthreads();
  if (warp == 0 && live) {
    T sum = T(0);
#pragma unroll
    for (int k = 0; k < kSegWarps; ++k) sum += red[k][lane];
    p.out[a + p.D * r] = sum;
  }
}

template <typename T>
__global__ void __launch_bounds__(kSegWarps * 32) seg_dot_tiled_kernel(const SegDot<T> p) {
  griddep_wait();
  seg_dot_tiled_run<T>(p, blockIdx.x);
}

// The tiled form when outputs are contiguous and the reduction is strided.
template <typename T>
inline bool seg_use_tiled(const SegDot<T>& p) {
  return p.astep == 1 && p.ustep > 1 && p.inner >= 8;
}

}  // namespace cpg
