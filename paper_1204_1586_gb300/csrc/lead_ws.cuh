// Leading contractions of Algorithm 2 (steps 4 and 7) on the 5th-generation
// tensor cores (tcgen05) with split-BF16 operands, warp-specialised.
//
// Y is the J x K column-major matrix reshape(Y, [J_k, K_k]) (eq. 2.3).  A CTA
// owns a J-block of nrt row tiles and a range of columns and walks it in
// stages (SR rows x SC columns):
//   step 4 alone  (SIDES 1): 128 x 64,  column chunks outer, row tiles inner;
//   step 7 alone  (SIDES 2):  64 x 128, row tiles outer, column chunks inner;
//   both, fused   (SIDES 3): 128 x 128, column chunks outer, row tiles inner.
//
// Every FP32 value x (of Y and of the Khatri-Rao rows) is split into L BF16
// limbs, each rounded to nearest: x0 = bf16(x), x1 = bf16(x - x0),
// x2 = bf16(x - x0 - x1); the differences are exact in FP32.  The products
// kept are those of total limb order below L (Henry, Tang and Heinecke,
// "Leveraging the bfloat16 AI datatype for higher-precision computations",
// 2019):
//   L = 1 (BF16):   y0 w0;
//   L = 2 (BF16x3): y0 w0 + y0 w1 + y1 w0;
//   L = 3 (BF16x6): y0 w0 + y0 w1 + y1 w0 + y0 w2 + y1 w1 + y2 w0.
// They are issued as L MMAs per K step, y_l [w_0 | ... | w_{L-1-l}] with
// N = (L - l) RTP, all into one tensor-memory slot whose column block b then
// holds sum_{l <= L-1-b} y_l w_b.
//
// Warp roles (one CTA per SM):
//   warp 0      TMA producer: 32 KB FP32 boxes of Y into a ring of NRU units;
//   warp 1      MMA issuer (one thread) and tensor-memory owner;
//   warps 2-5   promotion: after every stage, read the slot (tcgen05.ld),
//               add its column blocks, unscale, and add the stage's result
//               into a running sum in tensor memory with FP32 round-to-nearest
//               adds; at the end write the deterministic partial sums;
//   warps 6-13  converters: FP32 boxes -> BF16 limb tiles (a ring of NL
//               stages), and the Khatri-Rao B tiles of eqs. 3.9 / 3.10.
// Stages hand over on mbarriers (full / empty pairs); there is no block-wide
// barrier inside the loop.  The tensor cores only ever accumulate one stage
// (at most 8 K steps of 16) in a slot: the running sums are FP32 adds, so the
// accumulation error does not grow with the number of columns a CTA covers.
//
// Per-column power-of-two scaling: every Khatri-Rao B tile is built with each
// rank column multiplied by 2^-e, e the binary exponent of the column's
// largest entry in the tile, and the promotion multiplies the stage's result
// by 2^e.  Both are exact, so the result equals the unscaled product; the
// scaling keeps the limbs of columns of any magnitude far from the BF16
// range limits.
//
// Limb tile layout (one per limb, SR x SC): 1 KB atoms
//   [column group of 8][64-row half][8 columns][64 rows, 128-byte swizzle],
// which is at once the MN-major A operand of step 4 (M = rows, K = columns)
// and the K-major A operand of step 7 (M = columns, K = rows).  B tiles are
// K-major: B row n (limb block b = n / RTP, rank n % RTP) holds KW contraction
// entries in 128-byte swizzled lines, 8 rows per atom.
//
// Tiles arrive by TMA (use_tma = 1) or, when Y's column pitch is not a multiple
// of 16 bytes, the converters load their elements straight from global memory.
//
// Every wait is bounded (time and iterations) and observes a CTA-wide abort
// flag: on expiry the CTA records CPG_ERR_TIMEOUT in the status word, waits
// (bounded) for its own copies and MMAs, frees its tensor memory and returns.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include "common.cuh"
#include "tc_common.cuh"

namespace cpg {

// Arguments of the tensor-core leading kernels (split BF16 and split TF32).
struct TcArgs {
  int64_t J, K;
  int R, r0;
  KrRows<float> wl, wr;
  int64_t Kc;      // columns per CTA (multiple of the stage width)
  int nrt;         // row tiles per J-block
  float* Rpart;    // [nKs][R][J]
  float* Lpart;    // [nJb][R][K]
  double* normpart;  // [nJb*nKs] partial sums of y^2 (R side only), or nullptr
  int* status;
  const float* Y;  // the tensor (element loads when use_tma == 0)
  int64_t ldy;     // elements from one column of Y_(1:k) to the next (>= J)
  int use_tma;     // 1: TMA boxes; 0: element loads (rows not 16-byte aligned)
  // Split-BF16 kernel: the Khatri-Rao B tiles of the pass, prebuilt in their
  // shared-memory layout (ws_wimg_kernel), tile t at t * (tile bytes + 64):
  // W_R tiles of KWR contraction entries (columns of Y), W_L of KWL (rows).
  unsigned char* wimg_r;
  unsigned char* wimg_l;
};

// 4-byte copy global -> shared with zero fill (src_bytes = 0 writes zeros and
// reads nothing).
__device__ __forceinline__ void cp_async_zfill4(void* dst, const void* src, int src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(tc::smem_addr(dst)), "l"(src), "r"(src_bytes)
               : "memory");
}

template <int RTP_, int SIDES_, int L_>
struct WsCfg {
  static constexpr int RTP = RTP_, SIDES = SIDES_, L = L_;
  static_assert(RTP % 16 == 0 && RTP <= 64, "MMA N must be a multiple of 16");
  static_assert(L >= 1 && L <= 3, "one to three BF16 limbs");
  static_assert(L * RTP <= 256, "MMA N at most 256");
  static constexpr bool DO_R = (SIDES & 1) != 0;
  static constexpr bool DO_L = (SIDES & 2) != 0;
  static constexpr int NSIDE = (DO_R ? 1 : 0) + (DO_L ? 1 : 0);
  static constexpr int SR = SIDES == 2 ? 64 : 128;  // rows per stage
  static constexpr int SC = SIDES == 1 ? 64 : 128;  // columns per stage
  static constexpr int NH = SR / 64;                // 64-row halves
  static constexpr int RU = SIDES == 2 ? 64 : 128;  // rows of one TMA box
  static constexpr int CU = 8192 / RU;              // columns of one TMA box (32 KB)
  static constexpr int UNITS = SR * SC / 8192;      // boxes per stage
  static constexpr uint32_t UNIT_BYTES = 32768;
  static constexpr uint32_t LIMB_BYTES = uint32_t(SR) * SC * 2;
  static constexpr uint32_t STAGE_BYTES = L * LIMB_BYTES;
  static constexpr int KWR = SC, KWL = SR;          // contraction entries per B tile
  static constexpr int NW = L * RTP;                // B rows, slot columns
  static constexpr uint32_t WR_BYTES = DO_R ? uint32_t(NW) * KWR * 2 : 0;
  static constexpr uint32_t WL_BYTES = DO_L ? uint32_t(NW) * KWL * 2 : 0;
  // Prebuilt B tiles in global memory: the limbs, then RTP exponent bytes
  // (padded to 64).
  static constexpr uint32_t WIMG_R_STRIDE = WR_BYTES + 64, WIMG_L_STRIDE = WL_BYTES + 64;
  // Converter warps.
  static constexpr int CW = 8;
  static constexpr int CT = CW * 32;                // converter threads
  static constexpr int OPT = 1024 / CT;             // octets (8 rows of a column) per thread per box
  // Fused pass: the W_L tiles of every row tile of the J-block stay in shared
  // memory (built during the first column chunk).
  static constexpr int NWLC = SIDES == 3 ? (RTP <= 16 ? 4 : 2) : 0;
  static constexpr int WBR = 2;                     // W_R ring
  static constexpr int WBL = SIDES == 2 ? 2 : (SIDES == 3 ? NWLC : 0);
  // Dynamic shared memory, leaving room for the alignment slack and the
  // kernel's static shared memory (barriers, exponent rings).
  static constexpr uint32_t budget = 227u * 1024u - 3072u;
  static constexpr uint32_t W_TOTAL = WBR * WR_BYTES + WBL * WL_BYTES;
  static constexpr int NL = (2u * STAGE_BYTES + W_TOTAL + uint32_t(UNITS) * UNIT_BYTES <= budget) ? 2 : 1;
  static constexpr int NRU_FIT = int((budget - NL * STAGE_BYTES - W_TOTAL) / UNIT_BYTES);
  static constexpr int NRU = NRU_FIT > 6 ? 6 : NRU_FIT;
  static_assert(NRU >= UNITS, "shared memory budget: a stage's boxes must fit");
  static constexpr uint32_t OFF_RAW = 0;
  static constexpr uint32_t OFF_LIMB = OFF_RAW + NRU * UNIT_BYTES;
  static constexpr uint32_t OFF_WR = OFF_LIMB + NL * STAGE_BYTES;
  static constexpr uint32_t OFF_WL = OFF_WR + WBR * WR_BYTES;
  static constexpr uint32_t OFF_END = OFF_WL + WBL * WL_BYTES;
  static constexpr size_t smem_bytes = OFF_END + 1024;  // + alignment slack
  static_assert(smem_bytes <= 227 * 1024, "shared memory budget");
  // Tensor memory: running sums (RTP columns each), then NSLOT slots per side.
  static constexpr int NSLOT = (2 * NSIDE * NW <= 512 - 2 * RTP) ? 2 : 1;
  static constexpr int SLOT_COLS = NSIDE * NSLOT * NW;
  static constexpr int MAX_ACC = (512 - SLOT_COLS) / RTP;
  // One side with as many limb stages as slots: "stage ss's MMAs completed"
  // frees limb stage ss % NL and fills slot ss % NSLOT at once, so one
  // barrier (limb_empty) carries both.  Its phases cannot run ahead of either
  // waiter: the MMAs of stage ss + NL need the converters' stage ss + NL and
  // the promotion's release of slot ss.
  static constexpr bool ONE_COMMIT = NSIDE == 1 && NL == NSLOT;
  // MMA-issuing warps: with two limb stages and two slots, a second issuer
  // takes the odd stages, so that one issuer's waits and bookkeeping overlap
  // the other's MMAs in the tensor pipe.
  static constexpr int NISS = (NL == 2 && NSLOT == 2) ? 2 : 1;
  // Warps: producer, MMA issuer 0, 4 promotion, CW converters, MMA issuer 1.
  static constexpr int NWARP = 2 + 4 + CW + (NISS - 1);
  static constexpr int NT = NWARP * 32;
  static constexpr int NEXP = 8;                    // ring of per-tile scale exponents
};

// Byte offset of element (row j, column c) of a limb tile with NH row halves.
template <int NH>
__device__ __forceinline__ uint32_t ws_aoff(int j, int c) {
  const int atom = (c >> 3) * NH + (j >> 6);
  const int row = c & 7, chunk = ((j & 63) >> 3) ^ row;
  return uint32_t(atom * 1024 + row * 128 + chunk * 16 + (j & 7) * 2);
}
// Byte offset of element (B row n, contraction index k) of a K-major B tile
// with KW entries per row.
template <int KW>
__device__ __forceinline__ uint32_t ws_boff(int n, int k) {
  const int atom = (n >> 3) * (KW / 64) + (k >> 6);
  const int row = n & 7, chunk = ((k & 63) >> 3) ^ row;
  return uint32_t(atom * 1024 + row * 128 + chunk * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint32_t ws_pack_bf16(float a, float b) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&v);
}

// Splits a pair into L BF16 limbs (packed pairs): limb l of (x0, x1) in p[l];
// x is updated to the exact remainder after each limb.
template <int L>
__device__ __forceinline__ void ws_split_pair(float x0, float x1, uint32_t (&p)[L]) {
#pragma unroll
  for (int l = 0; l < L; ++l) {
    const uint32_t h = ws_pack_bf16(x0, x1);
    p[l] = h;
    if (l + 1 < L) {
      x0 -= __uint_as_float(h << 16);
      x1 -= __uint_as_float(h & 0xffff0000u);
    }
  }
}

// 8 values -> one 16-byte chunk per limb.
template <int L>
__device__ __forceinline__ void ws_split8(const float (&x)[8], uint4 (&out)[L]) {
  uint32_t p[4][L];
#pragma unroll
  for (int q = 0; q < 4; ++q) ws_split_pair<L>(x[2 * q], x[2 * q + 1], p[q]);
#pragma unroll
  for (int l = 0; l < L; ++l) out[l] = make_uint4(p[0][l], p[1][l], p[2][l], p[3][l]);
}

// One Khatri-Rao B tile: rank columns r0 .. r0 + RTP - 1 of `kr` over
// contraction indices [base, base + KW) (zero past `limit` and past rank R),
// each column scaled by 2^-e (e = floor(log2) of the column's largest
// magnitude in the tile, so the scaling is exact), split into L BF16 limbs
// and stored in the K-major swizzled layout of ws_boff; exps[r] = e.  Thread
// t of nth (a multiple of 32) takes tasks of 8 consecutive indices of one
// rank; the KW / 8 tasks of a rank are adjacent lanes of one warp.
template <int RTP, int L, int KW>
__device__ __forceinline__ void ws_build_w(unsigned char* tile, signed char* exps, const KrRows<float>& kr,
                                           int64_t base, int64_t limit, int r0, int R, int t, int nth) {
  constexpr int KWO = KW / 8;
  const int lane = t & 31;
  for (int t0 = t & ~31; t0 < RTP * KWO; t0 += nth) {
    const int task = t0 + lane;
    const int r = task / KWO, ko = task % KWO;
    const bool rok = r0 + r < R;
    float w[8];
    float m = 0.f;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int64_t g = base + ko * 8 + e;
      w[e] = (rok && g < limit) ? kr.at(uint32_t(g), r0 + r) : 0.f;
      m = fmaxf(m, fabsf(w[e]));
    }
#pragma unroll
    for (int o = KWO / 2; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    int ex = 0;
    if (m > 0.f) {
      ex = int((__float_as_uint(m) >> 23) & 0xffu) - 127;  // floor(log2 m) for normal m
      ex = ex < -100 ? -100 : (ex > 100 ? 100 : ex);
    }
    const float sc = __int_as_float((127 - ex) << 23);  // 2^-ex
#pragma unroll
    for (int e = 0; e < 8; ++e) w[e] *= sc;
    uint4 limbs[L];
    ws_split8<L>(w, limbs);
#pragma unroll
    for (int l = 0; l < L; ++l) *reinterpret_cast<uint4*>(tile + ws_boff<KW>(l * RTP + r, ko * 8)) = limbs[l];
    if (ko == 0) exps[r] = static_cast<signed char>(ex);
  }
}

// The B tiles of one pass, built once in global memory (where the leading
// kernel's producer copies them from with one bulk copy each): tile t covers
// contraction indices [t KW, (t + 1) KW), zero from `limit` on.  A CTA's
// column range starts and ends on tile boundaries (or at K), so these are
// the tiles the CTAs would build for themselves.  grid-stride over tiles,
// 256 threads.
template <int RTP, int L, int KW>
__global__ void __launch_bounds__(256) ws_wimg_kernel(unsigned char* img, const KrRows<float> kr, int64_t limit,
                                                      int r0, int R, int64_t ntiles) {
  griddep_wait();
  constexpr uint32_t WB = uint32_t(L * RTP) * KW * 2, STRIDE = WB + 64;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    unsigned char* tile = img + t * STRIDE;
    ws_build_w<RTP, L, KW>(tile, reinterpret_cast<signed char*>(tile + WB), kr, t * KW, limit, r0, R, threadIdx.x,
                           256);
  }
  griddep_launch();
}

__device__ __forceinline__ uint64_t ws_globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Waits for the phase of `bar` with the given parity.  Gives up, sets *abort
// and returns false after about a second (or 2^30 polls); returns false at
// once when another warp has set *abort.
// Between polls the thread sleeps on the barrier (up to 2 us), so waiting
// warps leave the issue slots to the warps that work.
__device__ __forceinline__ bool ws_wait(uint64_t* bar, uint32_t parity, volatile int* abort) {
  if (tc::mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = ws_globaltimer();
  for (uint32_t i = 1; i < (1u << 30); ++i) {
    if (tc::mbar_try_wait_sleep(bar, parity, 2000u)) return true;
    if ((i & 15u) == 0) {
      if (*abort) return false;
      if (ws_globaltimer() - t0 > 1000000000ull) break;
    }
  }
  *abort = 1;
  return false;
}

// D[tmem] (+)= A * B with A and B BF16 in shared memory.
__device__ __forceinline__ void ws_mma(uint32_t d, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  tc::mma_bf16(d, ad, bd, idesc, acc);
}

// 2^e as a float (|e| <= 126).
__device__ __forceinline__ float ws_pow2(int e) { return __int_as_float((127 + e) << 23); }

template <int RTP, int SIDES, int L>
__global__ void __launch_bounds__(WsCfg<RTP, SIDES, L>::NT, 1)
    lead_ws_kernel(const __grid_constant__ CUtensorMap tmap, const TcArgs a) {
  using C = WsCfg<RTP, SIDES, L>;
  constexpr bool DO_R = C::DO_R, DO_L = C::DO_L;
  constexpr int SR = C::SR, SC = C::SC, NH = C::NH, UNITS = C::UNITS;
  constexpr int NRU = C::NRU, NL = C::NL, NSLOT = C::NSLOT, NW = C::NW;
  constexpr int WBR = C::WBR, WBL = C::WBL, NEXP = C::NEXP;
  extern __shared__ unsigned char smem_dyn[];
  // Align by an offset from the shared-memory base (not through an integer
  // round trip), so that accesses keep the shared state space.
  unsigned char* sm = smem_dyn + ((1024u - (tc::smem_addr(smem_dyn) & 1023u)) & 1023u);
  __shared__ uint64_t raw_full[NRU], raw_empty[NRU];
  __shared__ uint64_t limb_full[NL], limb_empty[NL];
  __shared__ uint64_t wr_full[WBR], wr_empty[WBR];
  __shared__ uint64_t wl_full[WBL > 0 ? WBL : 1], wl_empty[WBL > 0 ? WBL : 1];
  __shared__ uint64_t exr_full[NEXP], exl_full[NEXP];
  __shared__ uint64_t slot_full[C::NSIDE][NSLOT], slot_empty[C::NSIDE][NSLOT];
  __shared__ uint64_t mma_done;
  __shared__ __align__(16) signed char expR[NEXP][RTP];
  __shared__ __align__(16) signed char expL[(SIDES == 3 ? C::NWLC : NEXP)][RTP];
  __shared__ uint32_t tslot;
  __shared__ int abort_flag;
  __shared__ double wsum[C::CW];

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t J = a.J, K = a.K;
  const int R = a.R, r0 = a.r0;
  const int nrt = a.nrt;
  const int jb = blockIdx.x, ks = blockIdx.y;
  const int64_t jblk = int64_t(jb) * SR * nrt;
  const int64_t kbeg = int64_t(ks) * a.Kc;
  const int64_t kend = (kbeg + a.Kc < K) ? (kbeg + a.Kc) : K;
  const int nchunk = int((kend - kbeg + SC - 1) / SC);
  const int nss = nchunk * nrt;
  // Stage ss -> (column chunk, row tile).
  constexpr bool ROWS_OUTER = SIDES == 2;
  auto chunk_of = [&](int ss) { return ROWS_OUTER ? ss % nchunk : ss / nrt; };
  auto tile_of = [&](int ss) { return ROWS_OUTER ? ss / nchunk : ss % nrt; };
  // Running sums in tensor memory: step 4 one per row tile, step 7 one per
  // column chunk; the fused pass one per row tile plus one for the current
  // chunk's step-7 sum.
  const int nacc = SIDES == 1 ? nrt : SIDES == 2 ? nchunk : nrt + 1;
  const uint32_t slot0 = uint32_t(C::MAX_ACC) * RTP;  // first slot column
  uint32_t tcols = 32;
  while (tcols < slot0 + C::SLOT_COLS) tcols <<= 1;
  const bool use_tma = a.use_tma != 0;
  volatile int* abort = &abort_flag;

  if (tid == 0) {
    for (int i = 0; i < NRU; ++i) {
      tc::mbar_init(&raw_full[i], 1);
      tc::mbar_init(&raw_empty[i], C::CW);
    }
    for (int i = 0; i < NL; ++i) {
      tc::mbar_init(&limb_full[i], C::CW);
      tc::mbar_init(&limb_empty[i], 1);
    }
    // B tiles and their exponents arrive by the producer's bulk copies.
    for (int i = 0; i < WBR; ++i) {
      tc::mbar_init(&wr_full[i], 1);
      tc::mbar_init(&wr_empty[i], C::NISS);
    }
    for (int i = 0; i < (WBL > 0 ? WBL : 1); ++i) {
      tc::mbar_init(&wl_full[i], 1);
      tc::mbar_init(&wl_empty[i], C::NISS);
    }
    for (int i = 0; i < NEXP; ++i) {
      tc::mbar_init(&exr_full[i], 1);
      tc::mbar_init(&exl_full[i], 1);
    }
    for (int s = 0; s < C::NSIDE; ++s)
      for (int i = 0; i < NSLOT; ++i) {
        tc::mbar_init(&slot_full[s][i], 1);
        tc::mbar_init(&slot_empty[s][i], 4);
      }
    tc::mbar_init(&mma_done, C::NISS);
    tc::mbar_fence_init();
    abort_flag = 0;
  }
  if (warp == 1) tc::tmem_alloc(&tslot, tcols);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tbase = tslot;
  const bool bad_shape = nacc > C::MAX_ACC || (SIDES == 3 && nrt > C::NWLC) || (DO_R && a.wimg_r == nullptr) ||
                         (DO_L && a.wimg_l == nullptr);

  // ---- TMA producer ------------------------------------------------------------------
  // Unit u = box (u % UNITS) of stage u / UNITS.
  const int nunits = nss * UNITS;
  int issued = 0;
  auto issue_unit = [&](int u) {  // warp 0, lane 0
    const int slot = u % NRU;
    const int ss = u / UNITS, h = u % UNITS;
    const int64_t c0 = kbeg + int64_t(chunk_of(ss)) * SC + int64_t(h) * C::CU;
    const int64_t j0 = jblk + int64_t(tile_of(ss)) * SR;
    tc::mbar_arrive_expect_tx(&raw_full[slot], C::UNIT_BYTES);
    tc::tma_load_2d_hint(sm + C::OFF_RAW + slot * C::UNIT_BYTES, &tmap, int(j0), int(c0), &raw_full[slot],
                         tc::policy_evict_first());
  };
  // The first boxes read only Y, which no kernel writes: they are in flight
  // before the previous kernel's results are awaited.
  if (warp == 0 && lane == 0 && use_tma && !bad_shape)
    for (; issued < NRU && issued < nunits; ++issued) issue_unit(issued);
  griddep_wait();

  if (bad_shape) {
    if (tid == 0) abort_flag = 1;
  } else if (warp == 0) {
    if (lane == 0) {
      // In stage order: the stage's B tiles (W_R at the first row tile of a
      // chunk, W_L at the first chunk of a row tile; fused: every row tile's
      // W_L during the first chunk, kept), each a bulk copy of the prebuilt
      // limbs plus one of its exponents, then the stage's boxes of Y.
      int nwr = 0, nwl = 0;  // B tiles copied
      auto copy_w = [&](uint64_t* full, uint64_t* exfull, unsigned char* dst, signed char* edst,
                        const unsigned char* src, uint32_t bytes) {
        tc::mbar_arrive_expect_tx(full, bytes);
        tc::bulk_load(dst, src, bytes, full);
        tc::mbar_arrive_expect_tx(exfull, uint32_t(RTP));
        tc::bulk_load(edst, src + bytes, uint32_t(RTP), exfull);
      };
      for (int ss = 0; ss < nss; ++ss) {
        const int q = chunk_of(ss), rt = tile_of(ss);
        bool ok = true;
        if constexpr (DO_R) {
          if (rt == 0) {
            if (q >= WBR) ok = ws_wait(&wr_empty[q % WBR], uint32_t(q / WBR - 1) & 1u, abort);
            if (ok) {
              copy_w(&wr_full[q % WBR], &exr_full[q % NEXP], sm + C::OFF_WR + (q % WBR) * C::WR_BYTES, expR[q % NEXP],
                     a.wimg_r + (kbeg / SC + q) * int64_t(C::WIMG_R_STRIDE), C::WR_BYTES);
              ++nwr;
            }
          }
        }
        if constexpr (SIDES == 2) {
          if (ok && q == 0) {
            if (rt >= WBL) ok = ws_wait(&wl_empty[rt % WBL], uint32_t(rt / WBL - 1) & 1u, abort);
            if (ok) {
              copy_w(&wl_full[rt % WBL], &exl_full[rt % NEXP], sm + C::OFF_WL + (rt % WBL) * C::WL_BYTES,
                     expL[rt % NEXP], a.wimg_l + (jblk / SR + rt) * int64_t(C::WIMG_L_STRIDE), C::WL_BYTES);
              ++nwl;
            }
          }
        } else if constexpr (SIDES == 3) {
          if (q == 0) {
            copy_w(&wl_full[rt], &exl_full[rt], sm + C::OFF_WL + rt * C::WL_BYTES, expL[rt],
                   a.wimg_l + (jblk / SR + rt) * int64_t(C::WIMG_L_STRIDE), C::WL_BYTES);
            ++nwl;
          }
        }
        if (ok && use_tma) {
          for (int h = 0; h < UNITS && ok; ++h) {
            const int u = ss * UNITS + h;
            if (u < issued) continue;
            const int slot = u % NRU;
            if (u >= NRU) ok = ws_wait(&raw_empty[slot], uint32_t(u / NRU - 1) & 1u, abort);
            if (ok) {
              issue_unit(u);
              issued = u + 1;
            }
          }
        }
        if (!ok) break;
      }
      if (*abort) {  // let this CTA's own copies land before its memory is released
        for (int u = (issued > NRU ? issued - NRU : 0); u < issued; ++u)
          tc::mbar_wait(&raw_full[u % NRU], uint32_t(u / NRU) & 1u, 1u << 16);
        if constexpr (DO_R) {
          for (int i = (nwr > WBR ? nwr - WBR : 0); i < nwr; ++i)
            tc::mbar_wait(&wr_full[i % WBR], uint32_t(i / WBR) & 1u, 1u << 16);
          for (int i = (nwr > NEXP ? nwr - NEXP : 0); i < nwr; ++i)
            tc::mbar_wait(&exr_full[i % NEXP], uint32_t(i / NEXP) & 1u, 1u << 16);
        }
        if constexpr (DO_L) {
          constexpr int NB = SIDES == 3 ? C::NWLC : WBL, NE = SIDES == 3 ? C::NWLC : NEXP;
          for (int i = (nwl > NB ? nwl - NB : 0); i < nwl; ++i)
            tc::mbar_wait(&wl_full[i % NB], uint32_t(i / NB) & 1u, 1u << 16);
          for (int i = (nwl > NE ? nwl - NE : 0); i < nwl; ++i)
            tc::mbar_wait(&exl_full[i % NE], uint32_t(i / NE) & 1u, 1u << 16);
        }
      }
    }
  } else if (warp == 1 || (C::NISS == 2 && warp == 6 + C::CW)) {
    // ---- MMA issuers ----------------------------------------------------------------
    // Issuer p takes stages p, p + NISS, ...  Each tcgen05.commit tracks the
    // MMAs of its own thread, so a B tile that both issuers read is released
    // by one commit of each (a chunk or row tile with a single stage gets
    // both commits from the issuer that has it).
    if (lane == 0) {
      constexpr int NISS = C::NISS;
      const int p = warp == 1 ? 0 : 1;
      // This one thread bounds the pass when its loop is long (a stage's MMAs
      // wait for its scalar work), so the loop is kept short: the stage
      // coordinates advance by counters, and every shared-memory descriptor is
      // a base descriptor built once plus a constant offset.  The start-address
      // field holds address >> 4 and every shared address here is below 2^18,
      // so adding offset >> 4 cannot carry out of the field.
      const uint32_t limb0 = tc::smem_addr(sm + C::OFF_LIMB);
      const uint64_t a_r0 = tc::smem_desc_sw128(limb0, 1024, NH * 1024);  // step 4: MN-major A
      const uint64_t a_l0 = tc::smem_desc_sw128(limb0, 16, NH * 1024);    // step 7: K-major A
      const uint64_t b_r0 = tc::smem_desc_sw128(tc::smem_addr(sm + C::OFF_WR), 16, (C::KWR / 64) * 1024);
      const uint64_t b_l0 = tc::smem_desc_sw128(tc::smem_addr(sm + C::OFF_WL), 16, (C::KWL / 64) * 1024);
      const uint32_t dslot = tbase + slot0;
      int q = chunk_of(p), rt = tile_of(p);  // chunk and row tile of stage ss
      for (int ss = p; ss < nss; ss += NISS) {
        const int ls = ss % NL, sl = ss % NSLOT;
        if constexpr (DO_R) {
          if (!ws_wait(&wr_full[q % WBR], uint32_t(q / WBR) & 1u, abort)) break;
        }
        if constexpr (SIDES == 2) {
          if (!ws_wait(&wl_full[rt % WBL], uint32_t(rt / WBL) & 1u, abort)) break;
        } else if constexpr (SIDES == 3) {
          if (!ws_wait(&wl_full[rt], 0u, abort)) break;
        }
        if (!ws_wait(&limb_full[ls], uint32_t(ss / NL) & 1u, abort)) break;
        bool ok = true;
        if (ss >= NSLOT)
          for (int s = 0; s < C::NSIDE && ok; ++s)
            ok = ws_wait(&slot_empty[s][sl], uint32_t(ss / NSLOT - 1) & 1u, abort);
        if (!ok) break;
        tc::tc_fence_after();
        const uint64_t aoff = uint64_t(ls * C::STAGE_BYTES) >> 4;
        int side = 0;
        if constexpr (DO_R) {
          // Step 4: D[j, n] += A[j, c] B[n, c]; A MN-major (K step = 2 column groups).
          const uint64_t ar = a_r0 + aoff, br = b_r0 + (uint64_t((q % WBR) * C::WR_BYTES) >> 4);
          const uint32_t d = dslot + uint32_t((side * NSLOT + sl) * NW);
#pragma unroll
          for (int s = 0; s < SC / 16; ++s) {
#pragma unroll
            for (int l = 0; l < L; ++l)
              ws_mma(d, ar + uint64_t((l * C::LIMB_BYTES + s * 2 * NH * 1024) >> 4),
                     br + uint64_t(((s >> 2) * 1024 + (s & 3) * 32) >> 4), tc::idesc_bf16_f32(128, (L - l) * RTP, 1, 0),
                     (s > 0 || l > 0) ? 1u : 0u);
          }
          ++side;
        }
        if constexpr (DO_L) {
          // Step 7: D[c, n] += A[c, j] B[n, j]; A K-major (K step = 32 bytes of a line).
          const int wl = SIDES == 2 ? rt % WBL : rt;
          const uint64_t al = a_l0 + aoff, bl = b_l0 + (uint64_t(wl * C::WL_BYTES) >> 4);
          const uint32_t d = dslot + uint32_t((side * NSLOT + sl) * NW);
#pragma unroll
          for (int s = 0; s < SR / 16; ++s) {
            const int koff = (s >> 2) * 1024 + (s & 3) * 32;
#pragma unroll
            for (int l = 0; l < L; ++l)
              ws_mma(d, al + uint64_t((l * C::LIMB_BYTES + koff) >> 4), bl + uint64_t(koff >> 4),
                     tc::idesc_bf16_f32(128, (L - l) * RTP, 0, 0), (s > 0 || l > 0) ? 1u : 0u);
          }
        }
        tc::mma_commit(&limb_empty[ls]);
        if constexpr (!C::ONE_COMMIT)
          for (int s = 0; s < C::NSIDE; ++s) tc::mma_commit(&slot_full[s][sl]);
        if constexpr (DO_R) {  // this issuer's last stage of chunk q
          if (rt + NISS >= nrt) {
            tc::mma_commit(&wr_empty[q % WBR]);
            if (NISS == 2 && nrt == 1) tc::mma_commit(&wr_empty[q % WBR]);
          }
        }
        if constexpr (SIDES == 2) {  // this issuer's last stage of row tile rt
          if (q + NISS >= nchunk) {
            tc::mma_commit(&wl_empty[rt % WBL]);
            if (NISS == 2 && nchunk == 1) tc::mma_commit(&wl_empty[rt % WBL]);
          }
        }
        // this issuer's next stage (the loop order of chunk_of / tile_of)
#pragma unroll
        for (int i = 0; i < NISS; ++i) {
          if constexpr (ROWS_OUTER) {
            if (++q == nchunk) {
              q = 0;
              ++rt;
            }
          } else {
            if (++rt == nrt) {
              rt = 0;
              ++q;
            }
          }
        }
      }
      // Every MMA this thread issued has completed once mma_done flips.
      tc::mma_commit(&mma_done);
      tc::mbar_wait(&mma_done, 0u, 1u << 20);
    }
  } else if (warp < 6) {
    // ---- promotion ------------------------------------------------------------------
    const int qd = warp & 3;  // tensor-memory lanes 32 qd .. 32 qd + 31
    const uint32_t lrow = uint32_t(32 * qd) << 16;
    auto acc_col = [&](int i) { return tbase + lrow + uint32_t(i) * RTP; };
    // Output of running sum i: R side rows j of row tile i (or of the fused
    // pass's row tiles), L side columns c of chunk i.
    auto write_R = [&](int rt, const float (&v)[16], int r16) {
      const int64_t j = jblk + int64_t(rt) * SR + 32 * qd + lane;
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int r = r0 + r16 + i;
        if (r < R && j < J) a.Rpart[(int64_t(ks) * R + r) * J + j] = v[i];
      }
    };
    auto write_L = [&](int q, const float (&v)[16], int r16) {
      const int64_t c = kbeg + int64_t(q) * SC + 32 * qd + lane;
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int r = r0 + r16 + i;
        if (r < R && c < kend) a.Lpart[(int64_t(jb) * R + r) * K + c] = v[i];
      }
    };
    for (int ss = 0; ss < nss && !*abort; ++ss) {
      const int q = chunk_of(ss), rt = tile_of(ss), sl = ss % NSLOT;
      int side = 0;
#pragma unroll
      for (int sd = 0; sd < 2; ++sd) {
        const bool is_r = sd == 0;
        if (is_r ? !DO_R : !DO_L) continue;
        if (!ws_wait(C::ONE_COMMIT ? &limb_empty[sl] : &slot_full[side][sl], uint32_t(ss / NSLOT) & 1u, abort)) break;
        // Scale exponents of the stage's B tile.
        const signed char* ex;
        if (is_r) {
          if (!ws_wait(&exr_full[q % NEXP], uint32_t(q / NEXP) & 1u, abort)) break;
          ex = expR[q % NEXP];
        } else if (SIDES == 2) {
          if (!ws_wait(&exl_full[rt % NEXP], uint32_t(rt / NEXP) & 1u, abort)) break;
          ex = expL[rt % NEXP];
        } else {
          if (!ws_wait(&exl_full[rt], 0u, abort)) break;
          ex = expL[rt];
        }
        tc::tc_fence_after();
        const uint32_t scol = tbase + lrow + slot0 + uint32_t((side * NSLOT + sl) * NW);
        // Accumulator and its role for this stage.
        const int acc = is_r ? (SIDES == 2 ? -1 : rt) : (SIDES == 2 ? q : nrt);
        const bool first = is_r ? q == 0 : rt == 0;
        const bool last_l = !is_r && SIDES == 3 && rt == nrt - 1;  // fused: chunk q's step-7 sum complete
        // Per 16-rank chunk: the slot's column blocks and the running sum are
        // all in flight before one wait; the sum of the blocks (smallest
        // first) is unscaled and added to the running sum.  The slot is free
        // for the stage after next once its last loads have completed.
        tc::tmem_wait_st();  // this thread's stores of the previous stage
#pragma unroll 1
        for (int r16 = 0; r16 < RTP; r16 += 16) {
          uint32_t u[L][16], g[16];
#pragma unroll
          for (int b = 0; b < L; ++b) tc::tmem_ld16_async(scol + uint32_t(b * RTP + r16), u[b]);
          if (!first) tc::tmem_ld16_async(acc_col(acc) + uint32_t(r16), g);
          tc::tmem_wait_ld();
          if (r16 + 16 >= RTP) {
            tc::tc_fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&slot_empty[side][sl]);
          }
          float w[16];
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            float t = __uint_as_float(u[L - 1][i]);
#pragma unroll
            for (int b = L - 2; b >= 0; --b) t += __uint_as_float(u[b][i]);
            t *= ws_pow2(ex[r16 + i]);
            w[i] = first ? t : __uint_as_float(g[i]) + t;
          }
          if (last_l) write_L(q, w, r16);
          else tc::tmem_st16_async(acc_col(acc) + uint32_t(r16), w);
        }
        ++side;
      }
    }
    tc::tmem_wait_st();
    if (!*abort) {
      // Completed running sums -> partial sums in global memory.
      const int nout = SIDES == 2 ? nchunk : nrt;
      for (int i = 0; i < nout; ++i) {
#pragma unroll 1
        for (int r16 = 0; r16 < RTP; r16 += 16) {
          float v[16];
          tc::tmem_ld16(acc_col(i) + uint32_t(r16), v);
          if (SIDES == 2) write_L(i, v, r16);
          else write_R(i, v, r16);
        }
      }
    }
  } else if (warp < 6 + C::CW) {
    // ---- converters -------------------------------------------------------------------
    const int ct = tid - 6 * 32, cw = ct >> 5;
    float ysq = 0.f;
    const bool do_norm = DO_R && a.normpart != nullptr;
    for (int ss = 0; ss < nss; ++ss) {
      const int q = chunk_of(ss), rt = tile_of(ss);
      const int64_t c0 = kbeg + int64_t(q) * SC, j0 = jblk + int64_t(rt) * SR;
      // The stage's FP32 values: octet o of box h is column o / (RU / 8),
      // rows 8 (o % (RU / 8)) .. + 7 of the box.
      float x[UNITS][C::OPT][8];
      bool ok = true;
#pragma unroll
      for (int h = 0; h < UNITS; ++h) {
        if (use_tma) {
          const int u = ss * UNITS + h, slot = u % NRU;
          if (!ws_wait(&raw_full[slot], uint32_t(u / NRU) & 1u, abort)) {
            ok = false;
            break;
          }
          const unsigned char* box = sm + C::OFF_RAW + slot * C::UNIT_BYTES;
#pragma unroll
          for (int o = 0; o < C::OPT; ++o) {
            const int oi = ct + C::CT * o;
            // Two 16-byte halves, in an order that spreads each quarter-warp
            // over eight distinct 16-byte bank groups.
            const float4* src = reinterpret_cast<const float4*>(box + oi * 32);
            const int first = (lane >> 2) & 1;
            const float4 pa = src[first], pb = src[first ^ 1];
            const float4 p0 = first ? pb : pa, p1 = first ? pa : pb;
            x[h][o][0] = p0.x; x[h][o][1] = p0.y; x[h][o][2] = p0.z; x[h][o][3] = p0.w;
            x[h][o][4] = p1.x; x[h][o][5] = p1.y; x[h][o][6] = p1.z; x[h][o][7] = p1.w;
          }
          __syncwarp();
          if (lane == 0) tc::mbar_arrive(&raw_empty[slot]);
        } else {
#pragma unroll
          for (int o = 0; o < C::OPT; ++o) {
            const int oi = ct + C::CT * o;
            const int cu = oi / (C::RU / 8), j8 = oi % (C::RU / 8);
            const int64_t cg = c0 + int64_t(h) * C::CU + cu, jg = j0 + 8 * j8;
            const float* p = a.Y + jg + a.ldy * cg;
#pragma unroll
            for (int e = 0; e < 8; ++e) x[h][o][e] = (cg < kend && jg + e < J) ? __ldg(p + e) : 0.f;
          }
        }
      }
      if (!ok) break;
      if (do_norm) {
        // Entries outside Y are zero (TMA fill, or the element loads' bounds);
        // columns past the CTA's range belong to the next CTA.
#pragma unroll
        for (int h = 0; h < UNITS; ++h)
#pragma unroll
          for (int o = 0; o < C::OPT; ++o) {
            const int cu = (ct + C::CT * o) / (C::RU / 8);
            if (c0 + int64_t(h) * C::CU + cu < kend) {
#pragma unroll
              for (int e = 0; e < 8; ++e) ysq = fmaf(x[h][o][e], x[h][o][e], ysq);
            }
          }
      }
      const int ls = ss % NL;
      if (ss >= NL && !ws_wait(&limb_empty[ls], uint32_t(ss / NL - 1) & 1u, abort)) break;
      unsigned char* limb = sm + C::OFF_LIMB + ls * C::STAGE_BYTES;
#pragma unroll
      for (int h = 0; h < UNITS; ++h)
#pragma unroll
        for (int o = 0; o < C::OPT; ++o) {
          const int oi = ct + C::CT * o;
          const int cu = oi / (C::RU / 8), j8 = oi % (C::RU / 8);
          uint4 lv[L];
          ws_split8<L>(x[h][o], lv);
          const uint32_t off = ws_aoff<NH>(8 * j8, h * C::CU + cu);
#pragma unroll
          for (int l = 0; l < L; ++l) *reinterpret_cast<uint4*>(limb + l * C::LIMB_BYTES + off) = lv[l];
        }
      tc::fence_async_smem();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&limb_full[ls]);
    }
    if (do_norm) {
      double sd = double(ysq);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sd += __shfl_xor_sync(0xffffffffu, sd, o);
      if (lane == 0) wsum[cw] = sd;
    }
  }

  __syncthreads();  // every role has finished (or given up)
  if (tid == 0) {
    if (DO_R && a.normpart != nullptr && !abort_flag) {
      double t = 0.0;
      for (int w = 0; w < C::CW; ++w) t += wsum[w];
      a.normpart[int64_t(ks) * gridDim.x + jb] = t;
    }
    if (abort_flag) atomicCAS(a.status, 0, int(CPG_ERR_TIMEOUT));
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 1) tc::tmem_dealloc(tbase, tcols);
}

}  // namespace cpg
