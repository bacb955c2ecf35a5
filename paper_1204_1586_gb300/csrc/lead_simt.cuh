// Leading contractions of Algorithm 2 (steps 4 and 7) on CUDA cores.
//
// Y is viewed, without moving data, as the J x K column-major matrix
// Y_(1:k) = reshape(Y, [J_k, K_k]) (eq. 2.3 / 2.11).  From one shared-memory
// tile of Y this kernel can form both
//
//   R-side (step 4, eq. 3.10):  R^(k)[j, r] = sum_c Y[j, c] * W_R[c, r],
//       W_R = A^(N) (.) ... (.) A^(k+1)   (Khatri-Rao over the trailing modes)
//   L-side (step 7, eq. 3.9):   L^(k+1)[r, c] = sum_j W_L[j, r] * Y[j, c],
//       W_L = A^(k) (.) ... (.) A^(1)     (Khatri-Rao over the leading modes)
//
// so that the all-mode gradient streams Y from memory once.  Each Khatri-Rao
// row is one factor row times one entry of a small Kronecker table (eq. 3.3).
// Where a stage's rows are at most a quarter of its tile (WPRE) and the tiles
// come by TMA, W_R and W_L are built once per pass in global memory
// (kr_rows_kernel, 0.4 MB each at 100^4 R=10) and copied with every tile;
// otherwise each CTA generates its rows per stage in shared memory.
//
// Work split: CTA (jb, ks) owns the J-block of nrt row tiles
// [jb*nrt*TJ, (jb+1)*nrt*TJ) and the column range [ks*Kc, ks*Kc+Kc); stage s
// covers column chunk s / nrt and row tile s % nrt.  The R side keeps its
// accumulators for every row of the block in registers, so it runs with
// nrt = 1; the L side alone may use tall blocks (nrt > 1) to cut the number
// of J-block partials.
//
// Tiles arrive through a ring of STAGES buffers.  When columns start on
// 16-byte boundaries (a.ldy, the column pitch, may exceed J for a pitched copy
// of Y) one thread issues TMA copies (cp.async.bulk.tensor, 128-byte swizzle,
// L2 evict-first: the tensor is read once) per stage; otherwise all threads
// issue element copies (cp.async with zero fill) into the same layout.  Entries outside Y read as zero, and
// Khatri-Rao rows outside Y are zero, so the arithmetic needs no bounds tests.
// The layout (tile_off) stores each 128-byte run of a column as one line whose
// 16-byte chunks are XOR-permuted by the column index, which serves both access
// patterns without bank conflicts:
//   R side: warp w takes columns w, w+8, ...; each lane holds RPL rows and
//           accumulates all RT ranks over the CTA's columns in registers.
//   L side: warp (wr, wc) takes a band of rows and TCL columns per lane and
//           accumulates over rows; the WR row bands are summed through shared
//           memory once per finished column chunk.
// Outputs are deterministic partial sums: Rpart[ks] (over K-splits) and
// Lpart[jb] (over J-blocks), summed in a fixed order by the chain kernels.
//
// Every wait on a TMA barrier is bounded; on expiry the CTA records
// CPG_ERR_TIMEOUT in the status word, waits (bounded) for its own copies and
// returns.
#pragma once

#include <cuda.h>

#include "common.cuh"
#include "tc_common.cuh"

namespace cpg {

template <typename T, int RT, int TJ, int SIDES>
struct SimtCfg {
  static constexpr bool DO_R = (SIDES & 1) != 0;
  static constexpr bool DO_L = (SIDES & 2) != 0;
  static constexpr int NT = 256;
  static constexpr int VEC = 16 / int(sizeof(T));        // elements per 16-byte chunk
  static constexpr int SEG = 128 / int(sizeof(T));       // elements per 128-byte line
  static constexpr int STAGE_BYTES = (TJ * int(sizeof(T)) <= 128) ? 16384 : 32768;
  static constexpr int STAGES = (STAGE_BYTES == 16384) ? 4 : 3;
  static constexpr int TK = STAGE_BYTES / (TJ * int(sizeof(T)));  // columns per stage
  static constexpr int NSEG = TJ / SEG;                  // 128-byte lines per column
  static constexpr int RPL = TJ / 32;                    // R side: rows per lane
  static constexpr int VECR = RPL < VEC ? RPL : VEC;     // R side: elements per load
  static constexpr int NLD = RPL / VECR;                 // R side: loads per column
  static constexpr int CPW = TK / 8;                     // R side: columns per warp per stage
  static constexpr int TCL = (TK >= 64 && RT <= 32) ? 2 : 1;  // L side: columns per lane
  static constexpr int WC = TK / (32 * TCL);             // L side: column groups
  static constexpr int WR = 8 / WC;                      // L side: row bands
  static constexpr int ROWS_PW = TJ / WR;                // L side: rows per warp
  // FP32 products run two at a time (fma.rn.f32x2); FP64 ranks in chunks of VEC.
  static constexpr bool F2 = sizeof(T) == 4;
  // L side, FP32, up to 20 (column, rank) accumulators per lane: a register
  // pair holds the even-row and odd-row partial sums of one (column, rank);
  // W_L is stored rank-major ([r][j]) so that one 16-byte load gives two row
  // pairs of a rank.  Wider lanes keep rank pairs (W_L row-major, [j][r]).
  static constexpr bool LP = F2 && TCL * RT <= 20;
  static_assert(F2 ? (RT % 2 == 0) : (RT % VEC == 0), "rank tile must be a multiple of the pair / vector width");
  static_assert(TJ % SEG == 0, "row tile must hold whole 128-byte lines");
  static_assert(WC >= 1 && 8 % WC == 0, "bad L-side warp grid");
  static_assert(ROWS_PW % VEC == 0, "row band must hold whole chunks");
  static_assert(8 * RT <= STAGES * TK, "R-side reduction must fit in the tile buffers");
  static_assert(NT % TK == 0 && NT % TJ == 0, "Khatri-Rao row generation maps whole rows / columns");
  static_assert(TK <= 256 && SEG <= 256, "TMA box extent");

  // Khatri-Rao entries per thread and stage: thread t generates column
  // t % TK of W_R for ranks t / TK + u * (NT / TK), and row t % TJ of W_L for
  // ranks t / TJ + u * (NT / TJ).
  static constexpr int RSTEP = NT / TK, EWR = DO_R ? (RT + RSTEP - 1) / RSTEP : 1;
  static constexpr int LSTEP = NT / TJ, EWL = DO_L ? (RT + LSTEP - 1) / LSTEP : 1;

  // The L-side row-band reduction reuses the stage buffer it has just consumed
  // when it fits there.
  static constexpr bool RED_ALIAS = size_t(WR) * RT * TK <= size_t(TK) * TJ;
  static constexpr size_t y_elems = size_t(STAGES) * TK * TJ;
  // Khatri-Rao row buffers.  When a stage's rows are at most half of its
  // tile (WPRE), rows built once per pass (LeadArgs::wpre_r / wpre_l) come
  // with each tile into a ring of STAGES slots; otherwise (and when no rows
  // are built) the CTA writes slots 0 and 1 itself (one W_L slot when both
  // sides run: W_L is then fixed per CTA).
  static constexpr size_t wr_slot = size_t(TK) * RT, wl_slot = size_t(TJ) * RT;
  static constexpr bool WPRE = 2 * ((DO_R ? wr_slot : 0) + (DO_L ? wl_slot : 0)) * sizeof(T) <= size_t(STAGE_BYTES);
  static constexpr size_t wr_elems = DO_R ? size_t(WPRE ? STAGES : 2) * wr_slot : 0;
  static constexpr size_t wl_elems = DO_L ? size_t(WPRE ? STAGES : DO_R ? 1 : 2) * wl_slot : 0;
  static_assert(STAGES >= 2, "two Khatri-Rao slots at least");
  static_assert((wr_slot * sizeof(T)) % 16 == 0 && (wl_slot * sizeof(T)) % 16 == 0,
                "Khatri-Rao slots are whole 16-byte units (bulk copies)");
  static constexpr size_t red_elems = (DO_L && WR > 1 && !RED_ALIAS) ? size_t(WR) * RT * TK : 0;
  // + slack to align the tile ring to 1024 bytes (128-byte swizzle atoms).
  static constexpr size_t smem_bytes = (y_elems + wr_elems + wl_elems + red_elems) * sizeof(T) + 1024;
  static_assert(smem_bytes <= 227 * 1024, "shared memory budget");
  // Two CTAs per SM when both shared memory and a 128-register budget allow.
  static constexpr int MIN_BLOCKS = (SIDES != 3 && RT <= 16 && 2 * (smem_bytes + 1024) <= 228 * 1024) ? 2 : 1;
};

// Paired FP32 arithmetic: two floats in one 64-bit register, one fused
// multiply-add instruction for both lanes of the pair (sm_100 family).
__device__ __forceinline__ uint64_t f2_pack(float a, float b) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void f2_unpack(uint64_t v, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// The RT/2 rank pairs of a W row (RT floats, 8-byte aligned), 16 bytes at a
// time where the pair count allows.
template <int NP>
__device__ __forceinline__ void lds_pairs(const float* row, uint64_t (&w)[NP]) {
  const uint64_t* p = reinterpret_cast<const uint64_t*>(row);
  if constexpr (NP % 2 == 0) {
#pragma unroll
    for (int i = 0; i < NP; i += 2) {
      const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(p + i);
      w[i] = v.x;
      w[i + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < NP; ++i) w[i] = p[i];
  }
}

// Position of element (column c, row j) inside one stage of the tile: line
// j / SEG of every column forms a TK x 128-byte block (one TMA box of the
// 128-byte-swizzle mode), and the 16-byte chunk index within a line is XORed
// with c mod 8.
template <int TK, int SEG, int VEC>
__device__ __forceinline__ int tile_off(int c, int j) {
  return (j / SEG) * (TK * SEG) + c * SEG + ((((j % SEG) / VEC) ^ (c & 7)) * VEC) + (j % VEC);
}

template <typename T, int N>
__device__ __forceinline__ void lds_vec(const T* p, T (&out)[N]) {
  constexpr int B = int(sizeof(T)) * N;
  if constexpr (B == 16) {
    const uint4 v = *reinterpret_cast<const uint4*>(p);
    const T* s = reinterpret_cast<const T*>(&v);
#pragma unroll
    for (int i = 0; i < N; ++i) out[i] = s[i];
  } else if constexpr (B == 8) {
    const uint2 v = *reinterpret_cast<const uint2*>(p);
    const T* s = reinterpret_cast<const T*>(&v);
#pragma unroll
    for (int i = 0; i < N; ++i) out[i] = s[i];
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) out[i] = p[i];
  }
}

template <typename T, int N>
__device__ __forceinline__ void sts_vec(T* p, const T (&in)[N]) {
  constexpr int B = int(sizeof(T)) * N;
  if constexpr (B == 16) {
    uint4 v;
    T* d = reinterpret_cast<T*>(&v);
#pragma unroll
    for (int i = 0; i < N; ++i) d[i] = in[i];
    *reinterpret_cast<uint4*>(p) = v;
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) p[i] = in[i];
  }
}

// Element copy global -> shared with zero fill: src_bytes = 0 writes zeros
// and reads nothing.
template <int BYTES>
__device__ __forceinline__ void cp_async_zfill(void* dst, const void* src, int src_bytes) {
  static_assert(BYTES == 4 || BYTES == 8, "element copy is 4 or 8 bytes");
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(smem_u32(dst)), "l"(src), "n"(BYTES),
               "r"(src_bytes)
               : "memory");
}

// SIDES: bit 0 = R side (step 4), bit 1 = L side (step 7).
// tmap: Y as the 2-D tensor {J, K} (rows contiguous), box {SEG, TK}, 128-byte
// swizzle, zero fill; used when a.use_tma is set.
template <typename T, int RT, int TJ, int SIDES>
__global__ void __launch_bounds__(256, (SimtCfg<T, RT, TJ, SIDES>::MIN_BLOCKS))
    lead_simt_kernel(const __grid_constant__ CUtensorMap tmap, const LeadArgs<T> a) {
  using C = SimtCfg<T, RT, TJ, SIDES>;
  constexpr bool DO_R = C::DO_R, DO_L = C::DO_L;
  constexpr int NT = C::NT, VEC = C::VEC, TK = C::TK, STAGES = C::STAGES, SEG = C::SEG;

  extern __shared__ unsigned char smem_dyn[];
  // Align by an offset from the shared-memory base (not through an integer
  // round trip), so that accesses keep the shared state space.
  T* Ys = reinterpret_cast<T*>(smem_dyn + ((1024u - (smem_u32(smem_dyn) & 1023u)) & 1023u));
  T* WRs = Ys + C::y_elems;
  T* WLs = WRs + C::wr_elems;
  T* red_sep = WLs + C::wl_elems;
  __shared__ uint64_t bar_full[STAGES];
  __shared__ uint64_t bar_w;  // Khatri-Rao rows of the prologue stages (built rows only)
  __shared__ int abort_flag;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t J = a.J, K = a.K;
  const int R = a.R, r0 = a.r0;
  const int nrt = DO_R ? 1 : a.nrt;                 // row tiles per J-block
  const int jb = blockIdx.x, ks = blockIdx.y;
  const int64_t jblk = int64_t(jb) * TJ * nrt;      // first row of the J-block
  const int64_t kbeg = int64_t(ks) * a.Kc;
  const int64_t kend = (kbeg + a.Kc < K) ? (kbeg + a.Kc) : K;
  const int nchunk = int((kend - kbeg + TK - 1) / TK);
  const int nst = nchunk * nrt;
  const bool do_norm = DO_R && (a.normpart != nullptr);
  const bool use_tma = a.use_tma != 0;
  // Khatri-Rao rows built once per pass arrive with the tiles (TMA mode only).
  const bool wpre = C::WPRE && use_tma && (!DO_R || a.wpre_r != nullptr) && (!DO_L || a.wpre_l != nullptr);

  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) tc::mbar_init(&bar_full[s], 1);
    tc::mbar_init(&bar_w, 1);
    tc::mbar_fence_init();
    abort_flag = 0;
  }

  // Stage `it` (column chunk it / nrt, row tile it % nrt) into buffer it % STAGES.
  // Element copies commit one cp.async group per call, empty past the last
  // stage, so that "all but STAGES - 2 groups complete" always means "stage
  // it has landed".
  int issued = 0;               // stages issued so far
  int iss_ci = 0, iss_rt = 0;   // column chunk and row tile of stage `issued`
  constexpr uint32_t WR_BYTES = uint32_t(C::wr_slot * sizeof(T)), WL_BYTES = uint32_t(C::wl_slot * sizeof(T));
  constexpr uint32_t W_BYTES = (DO_R ? WR_BYTES : 0u) + (DO_L ? WL_BYTES : 0u);
  const uint64_t y_policy = tc::policy_evict_first();  // the tiles are read once
  // Built Khatri-Rao rows of stage s (column chunk ci, row tile rt) into ring slot s % STAGES.
  auto load_w = [&](int s, int ci, int rt, uint64_t* bar) {
    if constexpr (DO_R)
      tc::bulk_load(WRs + size_t(s % STAGES) * C::wr_slot, a.wpre_r + (kbeg + int64_t(ci) * TK) * RT, WR_BYTES, bar);
    if constexpr (DO_L)
      tc::bulk_load(WLs + size_t(s % STAGES) * C::wl_slot, a.wpre_l + (int64_t(jb) * nrt + rt) * C::wl_slot, WL_BYTES,
                    bar);
  };
  // The prologue stages are issued before the previous kernel's results are
  // awaited: their Khatri-Rao rows follow on bar_w once it has completed.
  bool w_with_tile = false;
  auto issue = [&](int it) {    // it == issued, or past the last stage
    if (it >= nst) {
      if (!use_tma) cp_async_commit();
      return;
    }
    issued = it + 1;
    T* dst = Ys + size_t(it % STAGES) * TK * TJ;
    const int64_t cbase = kbeg + int64_t(iss_ci) * TK;
    const int64_t j0 = jblk + int64_t(iss_rt) * TJ;
    const int ci_it = iss_ci, rt_it = iss_rt;
    if (++iss_rt == nrt) {
      iss_rt = 0;
      ++iss_ci;
    }
    if (use_tma) {
      if (tid == 0) {
        tc::fence_async_smem();
        uint64_t* bar = &bar_full[it % STAGES];
        const bool w = wpre && w_with_tile;
        tc::mbar_arrive_expect_tx(bar, uint32_t(C::STAGE_BYTES) + (w ? W_BYTES : 0u));
#pragma unroll
        for (int s = 0; s < C::NSEG; ++s)
          tc::tma_load_2d_hint(dst + s * TK * SEG, &tmap, int(j0) + s * SEG, int(cbase), bar, y_policy);
        if (w) load_w(it, ci_it, rt_it, bar);
      }
    } else {
#pragma unroll 4
      for (int f = tid; f < TK * TJ; f += NT) {
        const int c = f / TJ, j = f % TJ;
        const int64_t cg = cbase + c, jg = j0 + j;
        const bool in = cg < K && jg < J;
        cp_async_zfill<int(sizeof(T))>(dst + tile_off<TK, SEG, VEC>(c, j), in ? a.Y + jg + a.ldy * cg : a.Y,
                                       in ? int(sizeof(T)) : 0);
      }
      cp_async_commit();
    }
  };

  // ---- Khatri-Rao rows ----
  const int cw = tid % TK, rw = tid / TK;  // W_R: column cw, ranks rw + RSTEP * u
  const int jw = tid % TJ, rl = tid / TJ;  // W_L: row jw, ranks rl + LSTEP * u
  T pwa[C::EWR], pwq[C::EWR], pla[C::EWL], plq[C::EWL];
  // Loads (not yet products) of the rows of `kr` at index idx (< lim) for
  // ranks rbase + rstep * u: one division per thread and stage.
  auto fetch_rows = [&](const KrRows<T>& kr, int64_t idx, int64_t lim, int rbase, int rstep, auto ne_tag, T* fa,
                        T* fq) {
    constexpr int NE = decltype(ne_tag)::value;
    const bool in = idx < lim;
    uint32_t i = 0, q = 0;
    if (in && kr.A != nullptr) {
      q = kr.d.div(uint32_t(idx));
      i = uint32_t(idx) - q * kr.d.d;
    }
#pragma unroll
    for (int u = 0; u < NE; ++u) {
      const int r = rbase + rstep * u;
      if (in && r < RT && r0 + r < R) {
        if (kr.A == nullptr) {
          fa[u] = T(1);
          fq[u] = T(1);
        } else {
          fa[u] = kr.A[i + int64_t(kr.d.d) * (r0 + r)];
          fq[u] = (kr.Q != nullptr) ? kr.Q[q + kr.ldq * (r0 + r)] : T(1);
        }
      } else {
        fa[u] = T(0);
        fq[u] = T(0);
      }
    }
  };
  auto fetch_wr = [&](int it2) {
    if (it2 < nst)
      fetch_rows(a.wr, kbeg + int64_t(it2) * TK + cw, K, rw, C::RSTEP,  // R side: one row tile per J-block
                 std::integral_constant<int, C::EWR>{}, pwa, pwq);
  };
  auto store_wr = [&](int it2) {
    T* Wr = WRs + size_t(it2 & 1) * TK * RT;
#pragma unroll
    for (int u = 0; u < C::EWR; ++u) {
      const int r = rw + C::RSTEP * u;
      if (r < RT) Wr[cw * RT + r] = pwa[u] * pwq[u];
    }
  };
  // W_L rows of row tile t of this J-block.
  auto fetch_wl = [&](int t) {
    fetch_rows(a.wl, jblk + int64_t(t) * TJ + jw, J, rl, C::LSTEP, std::integral_constant<int, C::EWL>{}, pla, plq);
  };
  auto store_wl = [&](T* Wl) {
#pragma unroll
    for (int u = 0; u < C::EWL; ++u) {
      const int r = rl + C::LSTEP * u;
      if (r < RT) Wl[C::LP ? r * TJ + jw : jw * RT + r] = pla[u] * plq[u];
    }
  };
  const bool wl_per_stage = DO_L && !DO_R && nrt > 1;
  __syncthreads();  // barriers initialised
  // The first stages read only Y, which no kernel writes: they are in flight
  // before the previous kernel's results (the factors) are awaited.
#pragma unroll 1
  for (int s = 0; s < STAGES - 1; ++s) issue(s);
  griddep_wait();
  w_with_tile = true;
  if (wpre) {
    if (tid == 0) {
      const int np = (nst < STAGES - 1) ? nst : STAGES - 1;
      tc::mbar_arrive_expect_tx(&bar_w, uint32_t(np) * W_BYTES);
      int ci = 0, rt = 0;
      for (int s = 0; s < np; ++s) {
        load_w(s, ci, rt, &bar_w);
        if (++rt == nrt) {
          rt = 0;
          ++ci;
        }
      }
      if (!tc::mbar_wait(&bar_w, 0)) abort_flag = 1;
    }
  } else {
    if constexpr (DO_L) {
      fetch_wl(0);
      store_wl(WLs);
    }
    if constexpr (DO_R) {
      fetch_wr(0);
      store_wr(0);
    }
  }
  __syncthreads();  // first Khatri-Rao rows stored or landed

  constexpr int NP = RT / 2;  // rank pairs (FP32)
  T racc[C::NLD][C::VECR][(DO_R && !C::F2) ? RT : 1];                          // FP64 accumulators
  T lacc[C::TCL][DO_L ? RT : 1];
  uint64_t racc2[C::NLD][C::VECR][(DO_R && C::F2) ? NP : 1];              // rank pairs
  uint64_t lacc2[C::TCL][(DO_L && C::F2) ? (C::LP ? RT : NP) : 1];         // row pairs (LP) or rank pairs
  T ss = T(0);  // this thread's sum of y^2 (fixed order); summed in FP64 across threads
  if constexpr (DO_R) {
#pragma unroll
    for (int m = 0; m < C::NLD; ++m)
#pragma unroll
      for (int e = 0; e < C::VECR; ++e) {
        if constexpr (C::F2) {
#pragma unroll
          for (int r = 0; r < NP; ++r) racc2[m][e][r] = 0ull;
        } else {
#pragma unroll
          for (int r = 0; r < RT; ++r) racc[m][e][r] = T(0);
        }
      }
  }
  auto zero_lacc = [&]() {
#pragma unroll
    for (int t = 0; t < C::TCL; ++t) {
      if constexpr (C::F2) {
#pragma unroll
        for (int r = 0; r < (C::LP ? RT : NP); ++r) lacc2[t][r] = 0ull;
      } else {
#pragma unroll
        for (int r = 0; r < RT; ++r) lacc[t][r] = T(0);
      }
    }
  };
  if constexpr (DO_L) zero_lacc();

  // L-side lane placement.
  const int wr = warp % C::WR, wc = warp / C::WR;
  const int cl0 = wc * 32 * C::TCL + lane;

  int ci = 0, rt = 0;  // column chunk and row tile of stage it
#pragma unroll 1
  for (int it = 0; it < nst; ++it) {
    // One thread waits for the TMA barrier (acquiring the copied tile) and the
    // block barrier orders every other thread after it, so that 255 threads do
    // not poll shared memory while the tile is in flight.
    if (use_tma) {
      if (tid == 0 && !tc::mbar_wait(&bar_full[it % STAGES], uint32_t(it / STAGES) & 1u)) abort_flag = 1;
    } else {
      cp_async_wait<STAGES - 2>();
    }
    __syncthreads();  // stage it is complete for every thread; stage it - 1 is consumed
    if (abort_flag) break;
    const int64_t cbase = kbeg + int64_t(ci) * TK;
    issue(it + STAGES - 1);
    // Khatri-Rao rows of the next stage: loads now, products stored after this
    // stage's arithmetic (into the buffer the previous stage used).
    if (!wpre) {
      if constexpr (DO_R) fetch_wr(it + 1);
      if (wl_per_stage && it + 1 < nst) fetch_wl(rt + 1 == nrt ? 0 : rt + 1);
    }

    T* Yst = Ys + size_t(it % STAGES) * TK * TJ;
    if constexpr (DO_R) {
      // Lane: RPL rows (one 16-byte chunk per load); pairs hold two ranks of a row.
      const T* Wr = WRs + size_t(wpre ? it % STAGES : it & 1) * C::wr_slot;
#pragma unroll 2
      for (int i = 0; i < C::CPW; ++i) {
        const int c = warp + 8 * i;
        T y[C::NLD][C::VECR];
#pragma unroll
        for (int m = 0; m < C::NLD; ++m) {
          const int j = lane * C::VECR + 32 * C::VECR * m;
          lds_vec<T, C::VECR>(Yst + tile_off<TK, SEG, VEC>(c, j), y[m]);
        }
        if constexpr (C::F2) {
          uint64_t yy[C::NLD][C::VECR];
#pragma unroll
          for (int m = 0; m < C::NLD; ++m)
#pragma unroll
            for (int e = 0; e < C::VECR; ++e) yy[m][e] = f2_pack(float(y[m][e]), float(y[m][e]));
          uint64_t w[NP];
          lds_pairs<NP>(reinterpret_cast<const float*>(Wr) + c * RT, w);
#pragma unroll
          for (int r = 0; r < NP; ++r)
#pragma unroll
            for (int m = 0; m < C::NLD; ++m)
#pragma unroll
              for (int e = 0; e < C::VECR; ++e) racc2[m][e][r] = f2_fma(yy[m][e], w[r], racc2[m][e][r]);
        } else {
#pragma unroll
          for (int r4 = 0; r4 < RT; r4 += VEC) {
            T w[VEC];
            lds_vec<T, VEC>(Wr + c * RT + r4, w);
#pragma unroll
            for (int m = 0; m < C::NLD; ++m)
#pragma unroll
              for (int e = 0; e < C::VECR; ++e)
#pragma unroll
                for (int v = 0; v < VEC; ++v) racc[m][e][r4 + v] = fma(y[m][e], w[v], racc[m][e][r4 + v]);
          }
        }
        if (do_norm) {
#pragma unroll
          for (int m = 0; m < C::NLD; ++m)
#pragma unroll
            for (int e = 0; e < C::VECR; ++e) ss = fma(y[m][e], y[m][e], ss);
        }
      }
    }

    if constexpr (DO_L) {
      const T* Wl = WLs + (wpre ? size_t(it % STAGES) * C::wl_slot : wl_per_stage ? size_t(it & 1) * C::wl_slot : 0);
      // Lanes read 16-byte chunks of consecutive columns at the same rows: the
      // XOR permutation puts 8 consecutive columns on 8 distinct bank groups.
      if constexpr (C::LP) {
#pragma unroll 2
        for (int q = 0; q < C::ROWS_PW / VEC; ++q) {
          const int jl = wr * C::ROWS_PW + q * VEC;
          uint64_t yq[C::TCL][2];  // rows (jl, jl+1) and (jl+2, jl+3) of each column
#pragma unroll
          for (int t = 0; t < C::TCL; ++t) {
            const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(Yst + tile_off<TK, SEG, VEC>(cl0 + 32 * t, jl));
            yq[t][0] = v.x;
            yq[t][1] = v.y;
          }
          const T* wl = Wl + jl;  // rank-major: W_L[j][r] at r * TJ + j
#pragma unroll
          for (int r = 0; r < RT; ++r) {
            const ulonglong2 w = *reinterpret_cast<const ulonglong2*>(wl + r * TJ);
#pragma unroll
            for (int t = 0; t < C::TCL; ++t) {
              lacc2[t][r] = f2_fma(yq[t][0], w.x, lacc2[t][r]);
              lacc2[t][r] = f2_fma(yq[t][1], w.y, lacc2[t][r]);
            }
          }
        }
      } else {
#pragma unroll 2
        for (int q = 0; q < C::ROWS_PW / VEC; ++q) {
          const int jl = wr * C::ROWS_PW + q * VEC;
          T y[C::TCL][VEC];
#pragma unroll
          for (int t = 0; t < C::TCL; ++t) lds_vec<T, VEC>(Yst + tile_off<TK, SEG, VEC>(cl0 + 32 * t, jl), y[t]);
#pragma unroll
          for (int e = 0; e < VEC; ++e) {
            if constexpr (C::F2) {
              uint64_t yy[C::TCL];
#pragma unroll
              for (int t = 0; t < C::TCL; ++t) yy[t] = f2_pack(float(y[t][e]), float(y[t][e]));
              uint64_t w[NP];
              lds_pairs<NP>(reinterpret_cast<const float*>(Wl) + (jl + e) * RT, w);
#pragma unroll
              for (int r = 0; r < NP; ++r)
#pragma unroll
                for (int t = 0; t < C::TCL; ++t) lacc2[t][r] = f2_fma(yy[t], w[r], lacc2[t][r]);
            } else {
#pragma unroll
              for (int r4 = 0; r4 < RT; r4 += VEC) {
                T w[VEC];
                lds_vec<T, VEC>(Wl + (jl + e) * RT + r4, w);
#pragma unroll
                for (int t = 0; t < C::TCL; ++t)
#pragma unroll
                  for (int v = 0; v < VEC; ++v) lacc[t][r4 + v] = fma(y[t][e], w[v], lacc[t][r4 + v]);
              }
            }
          }
        }
      }
      if (rt == nrt - 1) {
        if constexpr (C::LP) {
#pragma unroll
          for (int t = 0; t < C::TCL; ++t)
#pragma unroll
            for (int r = 0; r < RT; ++r) {
              float a0, a1;
              f2_unpack(lacc2[t][r], a0, a1);
              lacc[t][r] = a0 + a1;  // even rows + odd rows
            }
        } else if constexpr (C::F2) {
#pragma unroll
          for (int t = 0; t < C::TCL; ++t)
#pragma unroll
            for (int r = 0; r < NP; ++r) {
              float a0, a1;
              f2_unpack(lacc2[t][r], a0, a1);
              lacc[t][2 * r] = a0;
              lacc[t][2 * r + 1] = a1;
            }
        }
        // The chunk's columns are complete over this J-block: sum the row bands.
        if constexpr (C::WR > 1) {
          T* red = C::RED_ALIAS ? Yst : red_sep;
          if constexpr (C::RED_ALIAS) __syncthreads();  // every warp is done reading this stage
#pragma unroll
          for (int t = 0; t < C::TCL; ++t)
#pragma unroll
            for (int r = 0; r < RT; ++r) red[(size_t(wr) * RT + r) * TK + cl0 + 32 * t] = lacc[t][r];
          __syncthreads();
          for (int f = tid; f < RT * TK; f += NT) {
            const int r = f / TK, c = f % TK;
            T sum = T(0);
#pragma unroll
            for (int w = 0; w < C::WR; ++w) sum += red[(size_t(w) * RT + r) * TK + c];
            const int64_t cg = cbase + c;
            if (r0 + r < R && cg < kend) a.Lpart[(int64_t(jb) * R + r0 + r) * K + cg] = sum;
          }
          // This buffer is refilled by TMA (the async proxy) after the next barrier.
          if constexpr (C::RED_ALIAS) tc::fence_async_smem();
        } else {
#pragma unroll
          for (int t = 0; t < C::TCL; ++t) {
            const int64_t cg = cbase + cl0 + 32 * t;
#pragma unroll
            for (int r = 0; r < RT; ++r)
              if (r0 + r < R && cg < kend) a.Lpart[(int64_t(jb) * R + r0 + r) * K + cg] = lacc[t][r];
          }
        }
        zero_lacc();
      }
    }
    if (!wpre) {
      if constexpr (DO_R) {
        if (it + 1 < nst) store_wr(it + 1);
      }
      if (wl_per_stage && it + 1 < nst) store_wl(WLs + size_t((it + 1) & 1) * C::wl_slot);
    }
    if (++rt == nrt) {
      rt = 0;
      ++ci;
    }
  }

  if (!use_tma) cp_async_wait<0>();
  __syncthreads();  // every thread has left the loop
  if (abort_flag) {
    if (tid == 0) {
      atomicCAS(a.status, 0, int(CPG_ERR_TIMEOUT));
      // Let this CTA's own copies land (bounded) before its memory is released:
      // the newest phase of every stage buffer (older phases have completed).
      for (int q = (issued > STAGES ? issued - STAGES : 0); q < issued; ++q)
        tc::mbar_wait(&bar_full[q % STAGES], uint32_t(q / STAGES) & 1u, 1u << 16);
      if (wpre) tc::mbar_wait(&bar_w, 0, 1u << 16);
    }
    return;
  }

  if constexpr (DO_R) {
    // Sum the 8 warps' column-split partials through the (now idle) tile buffers.
    T* redR = Ys;
#pragma unroll
    for (int m = 0; m < C::NLD; ++m) {
      const int j = lane * C::VECR + 32 * C::VECR * m;
#pragma unroll
      for (int r = 0; r < RT; ++r) {
        T v[C::VECR];
#pragma unroll
        for (int e = 0; e < C::VECR; ++e) {
          if constexpr (C::F2) {
            float a0, a1;
            f2_unpack(racc2[m][e][r / 2], a0, a1);
            v[e] = (r & 1) ? a1 : a0;
          } else {
            v[e] = racc[m][e][r];
          }
        }
        sts_vec<T, C::VECR>(redR + (size_t(warp) * RT + r) * TJ + j, v);
      }
    }
    __syncthreads();
    for (int f = tid; f < RT * TJ; f += NT) {
      const int r = f / TJ, j = f % TJ;
      T sum = T(0);
#pragma unroll
      for (int w = 0; w < 8; ++w) sum += redR[(size_t(w) * RT + r) * TJ + j];
      const int64_t jg = jblk + j;
      if (r0 + r < R && jg < J) a.Rpart[(int64_t(ks) * R + r0 + r) * J + jg] = sum;
    }
    if (do_norm) {
      double sd = double(ss);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sd += __shfl_xor_sync(0xffffffffu, sd, o);
      __syncthreads();
      double* wsum = reinterpret_cast<double*>(Ys);
      if (lane == 0) wsum[warp] = sd;
      __syncthreads();
      if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += wsum[w];
        a.normpart[int64_t(ks) * gridDim.x + jb] = t;
      }
    }
  }
}

}  // namespace cpg
