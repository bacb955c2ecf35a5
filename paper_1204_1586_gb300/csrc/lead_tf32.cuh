// Leading contractions of Algorithm 2 (steps 4 and 7) on the tensor cores
// (tcgen05, kind::tf32) with the 3-term split-TF32 product and FP32
// accumulation, one side per pass.
//
// Every FP32 value x is split as x = hi + lo with hi = tf32(x) and
// lo = tf32(x - hi) (round to nearest, ties away); x - hi is exact in FP32,
// so hi + lo carries 22 significant bits.  Each product sums
//     y_hi w_hi + y_hi w_lo + y_lo w_hi,
// dropping only y_lo w_lo (about 2^-22 relative).
//
// Y is the J x K column-major matrix reshape(Y, [J_k, K_k]) (eq. 2.3).  A
// super-stage is a (TJS rows) x (TKS columns) tile that TMA writes as TJS/32
// boxes of {32 rows, TKS columns} with the 128-byte swizzle: column c of box
// x is one 128-byte line (rows 32x..32x+31), its 16-byte chunks XORed with
// c mod 8.  Both steps feed the tensor cores K-major A operands (a TF32
// operand that is MN-major in shared memory reads as zeros on this GPU):
//   step 7 (L side, 64 rows x 128 columns): A has M = columns and K = rows,
//     so the raw tile already is a K-major layout (8-column atoms 1 KB apart
//     along M, K steps of 8 rows inside a line, one box per 32 rows).  All
//     threads round it in place to hi and write lo into a second region of
//     the same layout;
//   step 4 (R side, 128 rows x 64 columns): A has M = rows and K = columns,
//     so every thread transposes 4 x 4 blocks in registers and writes hi and
//     lo into one K-major buffer (8-row atoms of 32 columns); the raw buffer
//     is free for the next copy as soon as it is converted.
// The Khatri-Rao rows (eqs. 3.9 / 3.10) are generated per super-stage into a
// K-major B tile [W_hi ; W_lo].  One thread issues, per K step of 8,
//     D += A_hi [W_hi | W_lo]   (N = 2 RTP)   and   D[:, :RTP] += A_lo W_hi,
// and the epilogue adds the two halves of D.
//
// Accumulators live in tensor memory: step 4 walks column chunks outer and
// keeps one accumulator per row tile of its J-block; step 7 walks row tiles
// outer and keeps one per column chunk, so each Khatri-Rao tile is built once
// per chunk (step 4) or per row tile (step 7).  Outputs are the same
// deterministic partial sums as the other leading kernels.
//
// Every mbarrier wait is bounded; on expiry the CTA records CPG_ERR_TIMEOUT in
// the status word, waits (bounded) for its own operations, frees its tensor
// memory and returns.
#pragma once

#include <cuda.h>

#include "common.cuh"
#include "lead_ws.cuh"
#include "tc_common.cuh"

namespace cpg {

template <int RTP, int SIDES>
struct Tf32Cfg {
  static_assert(SIDES == 1 || SIDES == 2, "the split-TF32 kernel runs one side per pass");
  static_assert(RTP % 16 == 0 && RTP <= 64, "MMA N must be a multiple of 16");
  static constexpr bool DO_R = SIDES == 1;
  static constexpr int NT = 256;
  static constexpr int TJS = DO_R ? 128 : 64;          // rows per super-stage
  static constexpr int TKS = DO_R ? 64 : 128;          // columns per super-stage
  static constexpr int KS = DO_R ? TKS : TJS;          // contraction length per super-stage
  static constexpr int NKSTEP = KS / 8;                // MMA K steps per super-stage
  static constexpr int NBOX = TJS / 32;                // {32 rows, TKS columns} boxes
  static constexpr uint32_t BOX_BYTES = uint32_t(TKS) * 128;
  static constexpr uint32_t RAW_BYTES = uint32_t(TJS) * TKS * 4;
  static constexpr int NW = 2 * RTP;                   // B rows: W_hi, then W_lo
  static constexpr uint32_t W_BYTES = uint32_t(NW) * KS * 4;
  static constexpr uint32_t budget = 227u * 1024u - 1024u;
  // Step 4: NB raw buffers, one converted buffer [hi | lo], one W tile (the
  // conversion of a super-stage waits for the previous MMAs).  Step 7: NB
  // buffers [hi (in place) | lo], two W tiles where they fit.
  static constexpr uint32_t BUF_BYTES = DO_R ? RAW_BYTES : 2 * RAW_BYTES;
  static constexpr uint32_t CONV_BYTES = DO_R ? 2 * RAW_BYTES : 0;
  static constexpr int WB = DO_R ? 1 : ((3u * BUF_BYTES + 2u * W_BYTES <= budget) ? 2 : 1);
  static constexpr int NB_MAX = DO_R ? 4 : 3;
  static constexpr int NB = (NB_MAX * BUF_BYTES + CONV_BYTES + uint32_t(WB) * W_BYTES <= budget) ? NB_MAX : NB_MAX - 1;
  static constexpr int NMB = DO_R ? 1 : NB;            // MMA-completion barriers
  static constexpr uint32_t OFF_CONV = NB * BUF_BYTES;
  static constexpr uint32_t OFF_W = OFF_CONV + CONV_BYTES;
  static constexpr size_t smem_bytes = OFF_W + WB * W_BYTES + 1024;  // + alignment slack
  static_assert(smem_bytes <= 227 * 1024, "shared memory budget");
  static_assert(RAW_BYTES / 16 % NT == 0, "conversion maps whole 16-byte chunks to threads");
};

// Byte offset of element (row j, column c) of a super-stage tile.
template <int TKS>
__device__ __forceinline__ uint32_t tf32_tile_off(int j, int c) {
  return uint32_t((j >> 5) * (TKS * 128) + c * 128 + ((((j & 31) >> 2) ^ (c & 7)) << 4) + ((j & 3) << 2));
}
// Byte offset of element (row n, k) of a K-major operand tile with 64 K
// entries per row (the Khatri-Rao B tiles, and step 4's converted A tile with
// n = row, k = column): 8-row groups of two 1 KB atoms (k < 32, k >= 32),
// 2 KB apart.
__device__ __forceinline__ uint32_t tf32_wtile_off(int n, int k) {
  return uint32_t(((n >> 3) * 2 + (k >> 5)) * 1024 + (n & 7) * 128 + ((((k & 31) >> 2) ^ (n & 7)) << 4) +
                  ((k & 3) << 2));
}

__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
__device__ __forceinline__ void split_tf32(float x, float& hi, float& lo) {
  hi = to_tf32(x);
  lo = to_tf32(x - hi);
}

template <int RTP, int SIDES>
__global__ void __launch_bounds__(256, 1) lead_tf32_kernel(const __grid_constant__ CUtensorMap tmap, const TcArgs a) {
  using C = Tf32Cfg<RTP, SIDES>;
  constexpr bool DO_R = C::DO_R;
  constexpr int NT = C::NT;
  extern __shared__ unsigned char smem_dyn[];
  // Align by an offset from the shared-memory base (not through an integer
  // round trip), so that accesses keep the shared state space.
  unsigned char* sm = smem_dyn + ((1024u - (tc::smem_addr(smem_dyn) & 1023u)) & 1023u);
  __shared__ uint64_t bar_full[C::NB];
  __shared__ uint64_t bar_mma[C::NMB];
  __shared__ uint32_t tslot;
  __shared__ int abort_flag;
  __shared__ double wsum[NT / 32];

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t J = a.J, K = a.K;
  const int R = a.R, r0 = a.r0;
  const int nrt = a.nrt;
  const int jb = blockIdx.x, ks = blockIdx.y;
  const int64_t jblk = int64_t(jb) * C::TJS * nrt;
  const int64_t kbeg = int64_t(ks) * a.Kc;
  const int64_t kend = (kbeg + a.Kc < K) ? (kbeg + a.Kc) : K;
  const int nchunk = int((kend - kbeg + C::TKS - 1) / C::TKS);
  const int nss = nchunk * nrt;
  // Step 4: chunks outer, accumulator per row tile.  Step 7: row tiles outer,
  // accumulator per chunk.
  auto chunk_of = [&](int ss) { return DO_R ? ss / nrt : ss % nchunk; };
  auto tile_of = [&](int ss) { return DO_R ? ss % nrt : ss / nchunk; };
  const int nacc = DO_R ? nrt : nchunk;
  uint32_t tcols = 32;
  while (tcols < uint32_t(nacc * C::NW)) tcols <<= 1;

  const bool use_tma = a.use_tma != 0;
  if (tid == 0) {
    for (int b = 0; b < C::NB; ++b) {
      // TMA: one arrival with the byte count; element copies: one arrival per
      // thread when its copies have landed.
      tc::mbar_init(&bar_full[b], use_tma ? 1 : NT);
      if (b < C::NMB) tc::mbar_init(&bar_mma[b], 1);
    }
    tc::mbar_fence_init();
    abort_flag = 0;
  }
  if (warp == 0) tc::tmem_alloc(&tslot, tcols);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tbase = tslot;

  int last_issued = 0;  // super-stages whose copies have been issued
  int mma_issued = 0;   // super-stages whose MMAs thread 0 has issued
  auto issue_tma = [&](int ss) {  // thread 0 only
    last_issued = ss + 1;
    const int b = ss % C::NB;
    const int64_t cb = kbeg + int64_t(chunk_of(ss)) * C::TKS;
    const int64_t j0 = jblk + int64_t(tile_of(ss)) * C::TJS;
    uint64_t* bar = &bar_full[b];
    tc::mbar_arrive_expect_tx(bar, C::RAW_BYTES);
    // Row coordinates are multiples of 32 elements (128 bytes), as TMA requires.
    const uint64_t pol = tc::policy_evict_first();  // the tiles are read once
#pragma unroll
    for (int x = 0; x < C::NBOX; ++x)
      tc::tma_load_2d_hint(sm + b * C::BUF_BYTES + x * C::BOX_BYTES, &tmap, int(j0) + 32 * x, int(cb), bar, pol);
  };
  // The same tile by element copies (every thread), in the boxes' layout;
  // entries outside Y are zero-filled.
  auto issue_copies = [&](int ss) {
    last_issued = ss + 1;
    const int b = ss % C::NB;
    const int64_t cb = kbeg + int64_t(chunk_of(ss)) * C::TKS;
    const int64_t j0 = jblk + int64_t(tile_of(ss)) * C::TJS;
    unsigned char* dst = sm + b * C::BUF_BYTES;
#pragma unroll 4
    for (int f = tid; f < C::TJS * C::TKS; f += NT) {
      const int c = f / C::TJS, j = f % C::TJS;
      const int64_t cg = cb + c, jg = j0 + j;
      const bool in = cg < K && jg < J;
      cp_async_zfill4(dst + tf32_tile_off<C::TKS>(j, c), in ? a.Y + jg + a.ldy * cg : a.Y, in ? 4 : 0);
    }
    tc::cp_async_mbar_arrive(&bar_full[b]);
  };
  auto issue = [&](int ss) {
    if (use_tma) {
      if (tid == 0) issue_tma(ss);
    } else {
      issue_copies(ss);
    }
  };
  // The first super-stages read only Y, which no kernel writes: they are in
  // flight before the previous kernel's results (the factors) are awaited.
  for (int ss = 0; ss < C::NB && ss < nss; ++ss) issue(ss);
  griddep_wait();

  // Khatri-Rao B tile [W_hi ; W_lo] over KS contraction indices from `base`:
  // a task is 4 consecutive indices of one rank (one 16-byte chunk per part);
  // consecutive threads take consecutive indices, so factor loads coalesce.
  const KrRows<float>& kr = DO_R ? a.wr : a.wl;
  auto gen_w = [&](unsigned char* tile, int64_t base, int64_t limit) {
    for (int task = tid; task < RTP * (C::KS / 4); task += NT) {
      const int n = task / (C::KS / 4), k4 = (task % (C::KS / 4)) * 4;
      const bool rok = r0 + n < R;
      float4 h, l;
      float* hp = &h.x;
      float* lp = &l.x;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int64_t g = base + k4 + e;
        const float w = (rok && g < limit) ? kr.at(uint32_t(g), r0 + n) : 0.f;
        split_tf32(w, hp[e], lp[e]);
      }
      *reinterpret_cast<float4*>(tile + tf32_wtile_off(n, k4)) = h;
      *reinterpret_cast<float4*>(tile + tf32_wtile_off(RTP + n, k4)) = l;
    }
  };

  // MMA-completion barrier of super-stage ss: one for step 4 (a single
  // converted buffer, at most one phase in flight), one per buffer for step 7.
  auto mma_bar = [&](int ss) { return &bar_mma[DO_R ? 0 : ss % C::NB]; };
  auto mma_parity = [&](int ss) { return uint32_t(DO_R ? ss : ss / C::NB) & 1u; };

  const bool do_norm = DO_R && a.normpart != nullptr;
  float ysq = 0.f;  // this thread's share of sum y^2 (entries outside Y are zero)
  bool ok = true;
  for (int ss = 0; ss < nss; ++ss) {
    const int q = chunk_of(ss), rt = tile_of(ss), b = ss % C::NB;
    const bool rebuild = DO_R ? rt == 0 : q == 0;  // first super-stage of a chunk (step 4) / row tile (step 7)
    if (!tc::mbar_wait(&bar_full[b], uint32_t(ss / C::NB) & 1u)) ok = false;
    // Step 4: the converted buffer and the W tile are free once the MMAs of
    // ss - 1 have completed.  Step 7 with one W tile: those MMAs read it.
    if (ss > 0 && (DO_R || (C::WB == 1 && rebuild))) {
      if (!tc::mbar_wait(mma_bar(ss - 1), mma_parity(ss - 1))) ok = false;
      tc::tc_fence_after();
    }
    if (!ok) atomicExch(&abort_flag, 1);
    __syncthreads();  // abort_flag is settled
    if (abort_flag) {
      ok = false;
      break;
    }
    unsigned char* buf = sm + b * C::BUF_BYTES;
    const int64_t cb = kbeg + int64_t(q) * C::TKS;
    const int64_t j0 = jblk + int64_t(rt) * C::TJS;
    // 1. Split the tile into hi and lo.
    if constexpr (DO_R) {
      // Blocks of 4 rows x 4 columns, transposed in registers into the
      // K-major [hi | lo] buffer (row j, column c at tf32_wtile_off(j, c)).
      // Lane l of an 8-lane group g takes row quad jq = l and column quad
      // (g + l / 2) mod 16: its reads (chunk jq ^ (column mod 8)) and its
      // writes (chunk (column quad mod 8) ^ (row mod 8)) then fall on 8
      // distinct 16-byte bank groups, so 16-byte accesses are conflict-free.
      unsigned char* conv = sm + C::OFF_CONV;
#pragma unroll
      for (int u = 0; u < (C::TJS / 4) * (C::TKS / 4) / NT; ++u) {
        const int blk = tid + NT * u;
        const int jq = blk & 7, cq = (((blk >> 3) & 15) + (jq >> 1)) & 15, x = blk >> 7;
        const int j = 32 * x + 4 * jq, c = 4 * cq;
        float4 v[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) v[e] = *reinterpret_cast<const float4*>(buf + tf32_tile_off<C::TKS>(j, c + e));
        if (do_norm) {
#pragma unroll
          for (int e = 0; e < 4; ++e)
            if (cb + c + e < kend)
              ysq = fmaf(v[e].x, v[e].x, fmaf(v[e].y, v[e].y, fmaf(v[e].z, v[e].z, fmaf(v[e].w, v[e].w, ysq))));
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float r0v = (&v[0].x)[i], r1v = (&v[1].x)[i], r2v = (&v[2].x)[i], r3v = (&v[3].x)[i];
          float4 h, l;
          split_tf32(r0v, h.x, l.x);
          split_tf32(r1v, h.y, l.y);
          split_tf32(r2v, h.z, l.z);
          split_tf32(r3v, h.w, l.w);
          const uint32_t off = tf32_wtile_off(j + i, c);
          *reinterpret_cast<float4*>(conv + off) = h;
          *reinterpret_cast<float4*>(conv + C::RAW_BYTES + off) = l;
        }
      }
    } else {
      // The raw tile is already K-major: hi in place, lo in the second region.
#pragma unroll 4
      for (int u = 0; u < int(C::RAW_BYTES / 16) / NT; ++u) {
        const int f = tid + NT * u;
        float4* p = reinterpret_cast<float4*>(buf) + f;
        const float4 v = *p;
        float4 h, l;
        split_tf32(v.x, h.x, l.x);
        split_tf32(v.y, h.y, l.y);
        split_tf32(v.z, h.z, l.z);
        split_tf32(v.w, h.w, l.w);
        *p = h;
        *(reinterpret_cast<float4*>(buf + C::RAW_BYTES) + f) = l;
      }
    }
    // 2. Khatri-Rao tile (W_R per column chunk, W_L per row tile).  With two
    //    tiles, the one being rebuilt was last read by MMAs two super-stages
    //    back at least, which have completed.
    const int wb = (DO_R ? q : rt) % C::WB;
    unsigned char* wtile = sm + C::OFF_W + wb * C::W_BYTES;
    if (rebuild) {
      if constexpr (DO_R) gen_w(wtile, cb, kend);
      else gen_w(wtile, j0, J);
    }
    tc::fence_async_smem();
    tc::tc_fence_before();
    __syncthreads();
    // Step 4: the raw buffer is consumed; refill it.
    if constexpr (DO_R) {
      if (ss + C::NB < nss) issue(ss + C::NB);
    }
    // 3. MMAs of this super-stage (K-major A: K step = 32 bytes inside the
    //    128-byte line, the next atom (step 4) or box (step 7) every 4 steps).
    if (tid == 0) {
      tc::tc_fence_after();
      const uint32_t hi0 = tc::smem_addr(DO_R ? sm + C::OFF_CONV : buf), lo0 = hi0 + C::RAW_BYTES;
      const uint32_t w0 = tc::smem_addr(wtile);
      const uint32_t d = tbase + uint32_t(DO_R ? rt : q) * C::NW;
      const bool first = DO_R ? q == 0 : rt == 0;
      constexpr uint32_t a_sbo = DO_R ? 2048u : 1024u;  // 8-row (M) group stride
#pragma unroll
      for (int s = 0; s < C::NKSTEP; ++s) {
        const uint32_t koff = uint32_t(s & 3) * 32u;
        const uint64_t bd = tc::smem_desc_sw128(w0 + (s >> 2) * 1024 + koff, 16, 2048);
        const uint32_t aoff = (DO_R ? uint32_t(s >> 2) * 1024u : uint32_t(s >> 2) * C::BOX_BYTES) + koff;
        tc::mma_tf32(d, tc::smem_desc_sw128(hi0 + aoff, 16, a_sbo), bd, tc::idesc_tf32_f32(128, C::NW, 0, 0),
                     (!first || s > 0) ? 1u : 0u);
        tc::mma_tf32(d, tc::smem_desc_sw128(lo0 + aoff, 16, a_sbo), bd, tc::idesc_tf32_f32(128, RTP, 0, 0), 1u);
      }
      tc::mma_commit(mma_bar(ss));
      mma_issued = ss + 1;
    }
    // 4. Step 7: retire super-stage ss - 1; its MMAs are done, so its buffer
    //    can be refilled.
    if constexpr (!DO_R) {
      if (ss > 0) {
        const int p = ss - 1;
        if (!tc::mbar_wait(mma_bar(p), mma_parity(p))) atomicExch(&abort_flag, 1);
        tc::tc_fence_after();
        if (p + C::NB < nss && !abort_flag) issue(p + C::NB);
      }
    }
  }

  __syncthreads();  // every thread has left the loop
  bool aborted = abort_flag != 0;
  if (!aborted && nss > 0) {
    if (!tc::mbar_wait(mma_bar(nss - 1), mma_parity(nss - 1))) atomicExch(&abort_flag, 1);
    tc::tc_fence_after();
    __syncthreads();
    aborted = abort_flag != 0;
    if (!aborted) {
      // Epilogue: warp w reads tensor-memory lanes 32 (w % 4) ..; warps 0-3 and
      // 4-7 take alternate accumulators.  D rows are rows of R^(k) (step 4) or
      // columns of L^(k+1) (step 7).
      const int sub = warp & 3;
      for (int t = warp >> 2; t < nacc; t += 2) {
        const int64_t idx = DO_R ? jblk + int64_t(t) * 128 + 32 * sub + lane
                                 : kbeg + int64_t(t) * 128 + 32 * sub + lane;
        const uint32_t col = tbase + (uint32_t(32 * sub) << 16) + uint32_t(t) * C::NW;
        float v[16], u[16];
#pragma unroll 1
        for (int r16 = 0; r16 < RTP; r16 += 16) {
          tc::tmem_ld16(col + r16, v);
          tc::tmem_ld16(col + RTP + r16, u);
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const int r = r0 + r16 + i;
            if constexpr (DO_R) {
              if (r < R && idx < J) a.Rpart[(int64_t(ks) * R + r) * J + idx] = v[i] + u[i];
            } else {
              if (r < R && idx < kend) a.Lpart[(int64_t(jb) * R + r) * K + idx] = v[i] + u[i];
            }
          }
        }
      }
    }
  }
  if constexpr (DO_R) {
    if (do_norm) {
      double sd = double(ysq);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sd += __shfl_xor_sync(0xffffffffu, sd, o);
      if (lane == 0) wsum[warp] = sd;
      __syncthreads();
      if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < NT / 32; ++w) t += wsum[w];
        a.normpart[int64_t(ks) * gridDim.x + jb] = t;
      }
    }
  }
  if (aborted && tid == 0) {
    atomicCAS(a.status, 0, int(CPG_ERR_TIMEOUT));
    // Let this CTA's own copies and MMAs drain (bounded) before its memory is
    // released: the newest phase of every buffer's barriers.
    for (int ss = (last_issued > C::NB ? last_issued - C::NB : 0); ss < last_issued; ++ss)
      tc::mbar_wait(&bar_full[ss % C::NB], uint32_t(ss / C::NB) & 1u, 1u << 16);
    for (int ss = (mma_issued > C::NMB ? mma_issued - C::NMB : 0); ss < mma_issued; ++ss)
      tc::mbar_wait(mma_bar(ss), mma_parity(ss), 1u << 16);
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, tcols);
}

}  // namespace cpg
