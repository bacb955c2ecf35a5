// Leading contractions of Algorithm 2 (steps 4 and 7) on the 5th-generation
// tensor cores (tcgen05), with split-BF16 operands and FP32 accumulation.
//
// Y is the J x K column-major matrix reshape(Y, [J_k, K_k]) (eq. 2.3); one
// CTA owns a J-block of nrt row tiles of 128 rows and a range of columns, and
// walks it in super-stages of (128 columns) x (one row tile), each in its own
// 64 KB shared buffer (NB buffers in a ring):
//
//   TMA      two 128 x 64 FP32 boxes fill the buffer (issued NB - 1 ahead);
//   convert  all threads read the FP32 tile into registers, then overwrite the
//            same buffer with y = hi + lo (BF16 round-to-nearest each), hi and
//            lo each a 128 x 128 tile of 1 KB atoms
//            [column group of 8][row half][8 columns][64 rows, 128-byte swizzle]
//            which is at once the MN-major A operand of step 4 (M = rows,
//            K = columns) and the K-major A operand of step 7 (M = columns,
//            K = rows);
//   KR rows  the Khatri-Rao rows W_R (columns) and W_L (rows) of eq. 3.9/3.10
//            are generated per tile (factor row x Kronecker-table entry) and
//            split into BF16 hi / lo rows of a K-major B operand;
//   MMA      one thread issues tcgen05.mma (M = 128, K = 16 per step):
//            step 4: D_R[row tile] += A_hi [W_hi | W_lo] + A_lo W_hi
//            step 7: D_L           += A_hi [W_hi | W_lo] + A_lo W_hi
//            (the BF16x3 split product; the plain BF16 form keeps A_hi W_hi);
//            D_R of every row tile of the block and D_L live in tensor memory;
//   epilogue D_L (two buffers, alternating by column chunk) is read back
//            (tcgen05.ld) after each chunk's last row tile; D_R after the CTA's
//            last column.  Outputs are the same deterministic partial sums as
//            the CUDA-core kernel.
// Converting super-stage s + 1 overlaps the MMAs of s; every buffer has its own
// MMA-completion barrier so that no wait can miss a phase.
//
// Every mbarrier wait is bounded; on expiry the CTA records CPG_ERR_TIMEOUT in
// the status word, waits (bounded) for its own operations, frees its tensor
// memory and returns.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include "common.cuh"
#include "tc_common.cuh"

namespace cpg {

struct TcArgs {
  int64_t J, K;
  int R, r0;
  KrRows<float> wl, wr;
  int64_t Kc;      // columns per CTA (multiple of 128)
  int nrt;         // row tiles per J-block
  float* Rpart;    // [nKs][R][J]
  float* Lpart;    // [nJb][R][K]
  double* normpart;  // [nJb*nKs] partial sums of y^2 (R side only), or nullptr
  int* status;
  const float* Y;  // the tensor (element copies when use_tma == 0)
  int64_t ldy;     // elements from one column of Y_(1:k) to the next (>= J)
  int use_tma;     // 1: TMA boxes; 0: every thread copies elements (rows not 16-byte aligned)
};

template <int RTP, int SIDES, int PREC>
struct TcCfg {
  static constexpr bool DO_R = (SIDES & 1) != 0;
  static constexpr bool DO_L = (SIDES & 2) != 0;
  static constexpr bool X3 = PREC == 0;                 // BF16x3; else plain BF16
  static constexpr int NT = 256;
  static constexpr int NW = X3 ? 2 * RTP : RTP;         // B rows (hi, then lo)
  static constexpr uint32_t BUF_BYTES = 128 * 128 * 4;  // one super-stage: fp32, then hi | lo
  static constexpr uint32_t HALF = 128 * 64 * 4;        // one TMA box (64 columns)
  static constexpr uint32_t W_BYTES = uint32_t(NW) * 128 * 2;
  static constexpr int NSIDE = (DO_R ? 1 : 0) + (DO_L ? 1 : 0);
  static constexpr uint32_t budget = 227u * 1024u - 1024u;
  // W tiles double-buffered and three stage buffers where they fit.
  static constexpr int WB = (2u * NSIDE * W_BYTES + 2u * BUF_BYTES <= budget) ? 2 : 1;
  static constexpr int NB = (uint32_t(WB) * NSIDE * W_BYTES + 3u * BUF_BYTES <= budget) ? 3 : 2;
  static constexpr uint32_t OFF_BUF = 0;
  static constexpr uint32_t OFF_WR = OFF_BUF + NB * BUF_BYTES;
  static constexpr uint32_t OFF_WL = OFF_WR + (DO_R ? WB * W_BYTES : 0);
  static constexpr uint32_t OFF_END = OFF_WL + (DO_L ? WB * W_BYTES : 0);
  static constexpr size_t smem_bytes = OFF_END + 1024;  // + alignment slack
  static_assert(smem_bytes <= 227 * 1024, "shared memory budget");
  static_assert(RTP % 16 == 0 && RTP <= 64, "MMA N must be a multiple of 16");
};

// Byte offset of element (row j, column c) of the split tile.
__device__ __forceinline__ uint32_t split_off(int j, int c) {
  const int atom = (c >> 3) * 2 + (j >> 6);
  const int row = c & 7, chunk = ((j & 63) >> 3) ^ row;
  return uint32_t(atom * 1024 + row * 128 + chunk * 16 + (j & 7) * 2);
}
// Byte offset of element (B row n, k) of a W tile (K-major, 2 K atoms per 8 rows).
__device__ __forceinline__ uint32_t wtile_off(int n, int k) {
  const int atom = (n >> 3) * 2 + (k >> 6);
  const int row = n & 7, chunk = ((k & 63) >> 3) ^ row;
  return uint32_t(atom * 1024 + row * 128 + chunk * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&v);
}

// hi = bf16(x), lo = bf16(x - hi) (round-to-nearest each) for a pair, with
// one paired conversion per limb; hi is unpacked exactly to form x - hi.
__device__ __forceinline__ uint32_t split2(float x0, float x1, uint32_t& lo) {
  const uint32_t hp = pack_bf16(x0, x1);
  const float h0 = __uint_as_float(hp << 16), h1 = __uint_as_float(hp & 0xffff0000u);
  lo = pack_bf16(x0 - h0, x1 - h1);
  return hp;
}
// The same for 8 values; packed 16 bytes each.
__device__ __forceinline__ void split8(const float (&x)[8], uint4& hi, uint4& lo) {
  hi.x = split2(x[0], x[1], lo.x);
  hi.y = split2(x[2], x[3], lo.y);
  hi.z = split2(x[4], x[5], lo.z);
  hi.w = split2(x[6], x[7], lo.w);
}

// 4-byte copy global -> shared with zero fill (src_bytes = 0 writes zeros and
// reads nothing).
__device__ __forceinline__ void cp_async_zfill4(void* dst, const void* src, int src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(tc::smem_addr(dst)), "l"(src), "r"(src_bytes)
               : "memory");
}

template <int RTP, int SIDES, int PREC>
__global__ void __launch_bounds__(256, 1) lead_tc_kernel(const __grid_constant__ CUtensorMap tmap, const TcArgs a) {
  using C = TcCfg<RTP, SIDES, PREC>;
  constexpr bool DO_R = C::DO_R, DO_L = C::DO_L, X3 = C::X3;
  constexpr int NT = C::NT;
  extern __shared__ unsigned char smem_dyn[];
  // Align by an offset from the shared-memory base (not through an integer
  // round trip), so that accesses keep the shared state space.
  unsigned char* sm = smem_dyn + ((1024u - (tc::smem_addr(smem_dyn) & 1023u)) & 1023u);
  __shared__ uint64_t bar_full[C::NB];
  __shared__ uint64_t bar_mma[C::NB];
  __shared__ uint32_t tslot;
  __shared__ int abort_flag;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t J = a.J, K = a.K;
  const int R = a.R, r0 = a.r0;
  const int nrt = a.nrt;
  const int jb = blockIdx.x, ks = blockIdx.y;
  const int64_t jblk = int64_t(jb) * 128 * nrt;
  const int64_t kbeg = int64_t(ks) * a.Kc;
  const int64_t kend = (kbeg + a.Kc < K) ? (kbeg + a.Kc) : K;
  const int nchunk = int((kend - kbeg + 127) / 128);
  const int nss = nchunk * nrt;
  // Step 7 alone walks row tiles in the outer loop and keeps one accumulator
  // per column chunk in tensor memory (the mirror of step 4, which keeps one
  // per row tile): W_L is then built once per row tile, not per super-stage.
  constexpr bool LOUT = SIDES == 2;
  const int tcols_needed = LOUT ? nchunk * C::NW : (DO_R ? nrt : 0) * C::NW + (DO_L ? 2 * C::NW : 0);
  uint32_t tcols = 32;
  while (tcols < uint32_t(tcols_needed)) tcols <<= 1;
  const uint32_t colL0 = (DO_R ? nrt : 0) * C::NW;

  const bool use_tma = a.use_tma != 0;
  if (tid == 0) {
    for (int b = 0; b < C::NB; ++b) {
      // TMA: one arrival with the byte count; element copies: one arrival per
      // thread when its copies have landed.
      tc::mbar_init(&bar_full[b], use_tma ? 1 : NT);
      tc::mbar_init(&bar_mma[b], 1);
    }
    tc::mbar_fence_init();
    abort_flag = 0;
  }
  if (warp == 0) tc::tmem_alloc(&tslot, tcols);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tbase = tslot;

  int last_issued = 0;  // super-stages whose TMA thread 0 has issued
  int mma_issued = 0;   // super-stages whose MMAs thread 0 has issued
  // Super-stage ss -> (column chunk, row tile).
  auto chunk_of = [&](int ss) { return LOUT ? ss % nchunk : ss / nrt; };
  auto tile_of = [&](int ss) { return LOUT ? ss / nchunk : ss % nrt; };
  auto issue_tma = [&](int ss) {  // thread 0 only
    last_issued = ss + 1;
    const int b = ss % C::NB;
    const int64_t cb = kbeg + int64_t(chunk_of(ss)) * 128;
    const int64_t j0 = jblk + int64_t(tile_of(ss)) * 128;
    uint64_t* bar = &bar_full[b];
    tc::mbar_arrive_expect_tx(bar, C::BUF_BYTES);
    const uint64_t pol = tc::policy_evict_first();  // the tiles are read once
    for (int h = 0; h < 2; ++h)
      tc::tma_load_2d_hint(sm + C::OFF_BUF + b * C::BUF_BYTES + h * C::HALF, &tmap, int(j0), int(cb + 64 * h), bar,
                           pol);
  };
  // The same tile by element copies (every thread), in the TMA boxes' layout:
  // column c at (c / 64) * HALF + (c % 64) * 512 bytes, rows contiguous;
  // entries outside Y are zero-filled.
  auto issue_copies = [&](int ss) {
    last_issued = ss + 1;
    const int b = ss % C::NB;
    const int64_t cb = kbeg + int64_t(chunk_of(ss)) * 128;
    const int64_t j0 = jblk + int64_t(tile_of(ss)) * 128;
    unsigned char* dst = sm + C::OFF_BUF + b * C::BUF_BYTES;
#pragma unroll 4
    for (int f = tid; f < 128 * 128; f += NT) {
      const int c = f >> 7, j = f & 127;
      const int64_t cg = cb + c, jg = j0 + j;
      const bool in = cg < K && jg < J;
      cp_async_zfill4(dst + (c >> 6) * C::HALF + (c & 63) * 512 + j * 4, in ? a.Y + jg + a.ldy * cg : a.Y, in ? 4 : 0);
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

  // Khatri-Rao B tile: rows n < RTP are hi, rows RTP + n are lo (X3).  Lanes
  // take consecutive index pairs of one rank, so factor loads coalesce and
  // every lane stores one packed BF16 pair per row.
  auto gen_w = [&](unsigned char* tile, const KrRows<float>& kr, int64_t base, int64_t limit) {
    for (int task = tid; task < RTP * 64; task += NT) {
      const int n = task >> 6, kp = task & 63;
      const int64_t g = base + 2 * kp;
      const bool rok = r0 + n < R;
      const float w0 = (rok && g < limit) ? kr.at(uint32_t(g), r0 + n) : 0.f;
      const float w1 = (rok && g + 1 < limit) ? kr.at(uint32_t(g + 1), r0 + n) : 0.f;
      const float h0 = __bfloat162float(__float2bfloat16_rn(w0)), h1 = __bfloat162float(__float2bfloat16_rn(w1));
      *reinterpret_cast<uint32_t*>(tile + wtile_off(n, 2 * kp)) = pack_bf16(h0, h1);
      if constexpr (X3) *reinterpret_cast<uint32_t*>(tile + wtile_off(RTP + n, 2 * kp)) = pack_bf16(w0 - h0, w1 - h1);
    }
  };

  // L epilogue: D_L rows are the chunk's 128 columns.
  auto dl_col = [&](int q) { return colL0 + uint32_t(LOUT ? q : (q & 1)) * C::NW; };
  auto epilogue_L = [&](int q) {
    if (warp < 4) {
      const uint32_t col = dl_col(q);
      const int64_t c = kbeg + int64_t(q) * 128 + 32 * warp + lane;
      float v[16], u[16];
#pragma unroll
      for (int r16 = 0; r16 < RTP; r16 += 16) {
        tc::tmem_ld16(tbase + (uint32_t(32 * warp) << 16) + col + r16, v);
        if constexpr (X3) tc::tmem_ld16(tbase + (uint32_t(32 * warp) << 16) + col + RTP + r16, u);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int r = r0 + r16 + i;
          const float val = X3 ? v[i] + u[i] : v[i];
          if (r < R && c < kend) a.Lpart[(int64_t(jb) * R + r) * K + c] = val;
        }
      }
    }
  };

  const bool do_norm = DO_R && a.normpart != nullptr;
  float ysq = 0.f;  // this thread's share of sum y^2 (rows beyond J are zero)
  bool ok = true;
  for (int ss = 0; ss < nss; ++ss) {
    const int q = chunk_of(ss), rt = tile_of(ss), b = ss % C::NB;
    if (!tc::mbar_wait(&bar_full[b], uint32_t(ss / C::NB) & 1u)) ok = false;
    if (C::WB == 1 && ss > 0) {  // single W tiles: MMA(ss - 1) must be done before they are rewritten
      if (!tc::mbar_wait(&bar_mma[(ss - 1) % C::NB], uint32_t((ss - 1) / C::NB) & 1u)) ok = false;
    }
    if (!ok) atomicExch(&abort_flag, 1);
    unsigned char* buf = sm + C::OFF_BUF + b * C::BUF_BYTES;
    // 1. FP32 tile -> registers (two half-chunk reads ordered to avoid bank conflicts).
    const int64_t cb = kbeg + int64_t(q) * 128;
    float x[8][8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int task = tid + NT * u;
      const int c = task >> 4, jq = task & 15;
      const int first = (jq >> 2) & 1;
      const float* src = reinterpret_cast<const float*>(buf + (c >> 6) * C::HALF + (c & 63) * 512 + jq * 32);
      const float4 pa = reinterpret_cast<const float4*>(src)[first];
      const float4 pb = reinterpret_cast<const float4*>(src)[first ^ 1];
      const float4 p0 = first ? pb : pa, p1 = first ? pa : pb;
      x[u][0] = p0.x; x[u][1] = p0.y; x[u][2] = p0.z; x[u][3] = p0.w;
      x[u][4] = p1.x; x[u][5] = p1.y; x[u][6] = p1.z; x[u][7] = p1.w;
      if constexpr (DO_R) {
        if (do_norm && cb + c < kend) {
#pragma unroll
          for (int e = 0; e < 8; ++e) ysq = fmaf(x[u][e], x[u][e], ysq);
        }
      }
    }
    __syncthreads();  // the whole FP32 tile is in registers; abort_flag is settled
    if (abort_flag) {
      ok = false;
      break;
    }
    // 2. Overwrite the buffer with the BF16 hi | lo split tile.
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int task = tid + NT * u;
      const int c = task >> 4, jq = task & 15;
      uint4 hi, lo;
      split8(x[u], hi, lo);
      const uint32_t off = split_off(jq * 8, c);
      *reinterpret_cast<uint4*>(buf + off) = hi;
      if constexpr (X3) *reinterpret_cast<uint4*>(buf + 128 * 128 * 2 + off) = lo;
    }
    // 3. Khatri-Rao tiles of this super-stage.
    const int64_t j0 = jblk + int64_t(rt) * 128;
    // W_R depends on the column chunk only (buffer q % WB, rebuilt at its first
    // row tile); W_L on the row tile (buffer rt % WB at the first chunk of the
    // row tile when rows are outer, else buffer ss % WB).  The buffer being
    // rebuilt was last read by MMAs that have completed.
    const int wbr = q % C::WB, wbl = LOUT ? rt % C::WB : ss % C::WB;
    if constexpr (DO_R) {
      if (rt == 0) gen_w(sm + C::OFF_WR + wbr * C::W_BYTES, a.wr, cb, kend);
    }
    if constexpr (DO_L) {
      if (LOUT ? q == 0 : (nrt > 1 || ss == 0 || C::WB == 1)) gen_w(sm + C::OFF_WL + wbl * C::W_BYTES, a.wl, j0, J);
    }
    tc::fence_async_smem();
    tc::tc_fence_before();
    __syncthreads();
    // 4. MMAs of this super-stage.
    if (tid == 0) {
      tc::tc_fence_after();
      const uint32_t hi0 = tc::smem_addr(buf), lo0 = hi0 + 128 * 128 * 2;
      if constexpr (DO_R) {
        const uint32_t w0 = tc::smem_addr(sm + C::OFF_WR + wbr * C::W_BYTES);
        const uint32_t d = tbase + uint32_t(rt) * C::NW;
        for (int s = 0; s < 8; ++s) {
          const uint64_t bd = tc::smem_desc_sw128(w0 + (s >> 2) * 1024 + (s & 3) * 32, 16, 2048);
          tc::mma_bf16(d, tc::smem_desc_sw128(hi0 + s * 4096, 1024, 2048), bd, tc::idesc_bf16_f32(128, C::NW, 1, 0),
                       (q > 0 || s > 0) ? 1u : 0u);
          if constexpr (X3)
            tc::mma_bf16(d, tc::smem_desc_sw128(lo0 + s * 4096, 1024, 2048), bd, tc::idesc_bf16_f32(128, RTP, 1, 0), 1u);
        }
      }
      if constexpr (DO_L) {
        const uint32_t w0 = tc::smem_addr(sm + C::OFF_WL + (LOUT || nrt > 1 || C::WB == 1 ? wbl : 0) * C::W_BYTES);
        const uint32_t d = tbase + dl_col(q);
        for (int s = 0; s < 8; ++s) {
          const uint32_t koff = (s >> 2) * 1024 + (s & 3) * 32;
          const uint64_t bd = tc::smem_desc_sw128(w0 + koff, 16, 2048);
          tc::mma_bf16(d, tc::smem_desc_sw128(hi0 + koff, 16, 2048), bd, tc::idesc_bf16_f32(128, C::NW, 0, 0),
                       (rt > 0 || s > 0) ? 1u : 0u);
          if constexpr (X3)
            tc::mma_bf16(d, tc::smem_desc_sw128(lo0 + koff, 16, 2048), bd, tc::idesc_bf16_f32(128, RTP, 0, 0), 1u);
        }
      }
      tc::mma_commit(&bar_mma[b]);
      mma_issued = ss + 1;
    }
    // 5. Retire super-stage ss - 1: its MMAs are done, so its chunk's D_L can be
    //    read and its buffer refilled.
    if (ss > 0) {
      const int p = ss - 1;
      if (!tc::mbar_wait(&bar_mma[p % C::NB], uint32_t(p / C::NB) & 1u)) atomicExch(&abort_flag, 1);
      tc::tc_fence_after();
      if constexpr (DO_L && !LOUT) {
        if (p % nrt == nrt - 1 && !abort_flag) epilogue_L(p / nrt);
      }
      if (p + C::NB < nss && !abort_flag) issue(p + C::NB);
    }
  }

  __syncthreads();  // every thread has left the loop
  bool aborted = abort_flag != 0;
  if (!aborted && nss > 0) {
    if (!tc::mbar_wait(&bar_mma[(nss - 1) % C::NB], uint32_t((nss - 1) / C::NB) & 1u)) atomicExch(&abort_flag, 1);
    tc::tc_fence_after();
    __syncthreads();
    aborted = abort_flag != 0;
    if (!aborted) {
      if constexpr (LOUT) {
        for (int q = 0; q < nchunk; ++q) epilogue_L(q);
      } else if constexpr (DO_L) {
        epilogue_L(nchunk - 1);
      }
      if constexpr (DO_R) {
        if (warp < 4) {
          for (int rt = 0; rt < nrt; ++rt) {
            const int64_t j = jblk + int64_t(rt) * 128 + 32 * warp + lane;
            float v[16], u[16];
#pragma unroll
            for (int r16 = 0; r16 < RTP; r16 += 16) {
              tc::tmem_ld16(tbase + (uint32_t(32 * warp) << 16) + uint32_t(rt) * C::NW + r16, v);
              if constexpr (X3) tc::tmem_ld16(tbase + (uint32_t(32 * warp) << 16) + uint32_t(rt) * C::NW + RTP + r16, u);
#pragma unroll
              for (int i = 0; i < 16; ++i) {
                const int r = r0 + r16 + i;
                const float val = X3 ? v[i] + u[i] : v[i];
                if (r < R && j < J) a.Rpart[(int64_t(ks) * R + r) * J + j] = val;
              }
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
      __shared__ double wsum[8];
      if (lane == 0) wsum[warp] = sd;
      __syncthreads();
      if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += wsum[w];
        a.normpart[int64_t(ks) * gridDim.x + jb] = t;
      }
    }
  }
  if (aborted && tid == 0) {
    atomicCAS(a.status, 0, int(CPG_ERR_TIMEOUT));
    // Let this CTA's own copies and MMAs drain (bounded) before its memory is released.
    // Newest phase of every buffer's barriers only (older phases have completed).
    for (int ss = (last_issued > C::NB ? last_issued - C::NB : 0); ss < last_issued; ++ss)
      tc::mbar_wait(&bar_full[ss % C::NB], uint32_t(ss / C::NB) & 1u, 1u << 16);
    for (int ss = (mma_issued > C::NB ? mma_issued - C::NB : 0); ss < mma_issued; ++ss)
      tc::mbar_wait(&bar_mma[ss % C::NB], uint32_t(ss / C::NB) & 1u, 1u << 16);
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, tcols);
}

}  // namespace cpg
