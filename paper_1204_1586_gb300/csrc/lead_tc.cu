// Host side of the tensor-core leading contractions: the TMA tensor map of Y
// for the split-BF16 kernel (lead_ws.cuh), instance dispatch, and the plan
// limits the planner reads.  The split-TF32 form is forwarded to lead_tf32.cu.
#include "lead_tc_dispatch.cuh"
#include "lead_tf32.cuh"
#include "lead_ws_host.cuh"

namespace cpg {

namespace {

int limbs_of(int prec) { return prec == kTcBf16 ? 1 : prec == kTcBf16x6 ? 3 : 2; }

template <int SIDES, int L>
int ws_max_acc_rtp(int RTP) {
  switch (RTP) {
    case 16: return WsCfg<16, SIDES, L>::MAX_ACC;
    case 32: return WsCfg<32, SIDES, L>::MAX_ACC;
    default:
      if constexpr (SIDES != 3) return WsCfg<64, SIDES, L>::MAX_ACC;
      return 0;
  }
}

template <int SIDES>
int ws_max_acc(int RTP, int L) {
  if (L == 1) return ws_max_acc_rtp<SIDES, 1>(RTP);
  if (L == 2) return ws_max_acc_rtp<SIDES, 2>(RTP);
  if constexpr (SIDES != 3) return ws_max_acc_rtp<SIDES, 3>(RTP);
  return 0;
}

}  // namespace

int tc_rank_tile(int r) { return r <= 16 ? 16 : r <= 32 ? 32 : 64; }

int tc_tile_rows(int prec, int sides) {
  if (prec == kTcTf32x3) return sides == 1 ? 128 : 64;
  return sides == 2 ? 64 : 128;
}
int tc_tile_cols(int prec, int sides) {
  if (prec == kTcTf32x3) return sides == 1 ? 64 : 128;
  return sides == 1 ? 64 : 128;
}

int tc_max_acc(int RTP, int sides, int prec) {
  if (prec == kTcTf32x3) return 512 / (2 * RTP);
  const int L = limbs_of(prec);
  switch (sides) {
    case 1: return ws_max_acc<1>(RTP, L);
    case 2: return ws_max_acc<2>(RTP, L);
    case 3: return ws_max_acc<3>(RTP, L);
    default: return 0;
  }
}

bool tc_fused_ok(int RTP, int prec) { return prec != kTcTf32x3 && limbs_of(prec) <= 2 && RTP <= 32; }

int tc_fused_max_nrt(int RTP, int prec) {
  if (!tc_fused_ok(RTP, prec)) return 0;
  const bool one = limbs_of(prec) == 1;
  const int nwlc = RTP <= 16 ? (one ? WsCfg<16, 3, 1>::NWLC : WsCfg<16, 3, 2>::NWLC)
                             : (one ? WsCfg<32, 3, 1>::NWLC : WsCfg<32, 3, 2>::NWLC);
  return std::min(nwlc, tc_max_acc(RTP, 3, prec) - 1);
}

namespace {

template <int SIDES, int L>
void wimg_bytes_rtp(int RTP, int64_t J, int64_t K, int nrt, size_t* rb, size_t* lb) {
  if (RTP <= 16) return wimg_bytes<16, SIDES, L>(J, K, nrt, rb, lb);
  if (RTP <= 32) return wimg_bytes<32, SIDES, L>(J, K, nrt, rb, lb);
  if constexpr (SIDES != 3) return wimg_bytes<64, SIDES, L>(J, K, nrt, rb, lb);
}

template <int SIDES>
void wimg_bytes_l(int RTP, int L, int64_t J, int64_t K, int nrt, size_t* rb, size_t* lb) {
  if (L == 1) return wimg_bytes_rtp<SIDES, 1>(RTP, J, K, nrt, rb, lb);
  if (L == 2) return wimg_bytes_rtp<SIDES, 2>(RTP, J, K, nrt, rb, lb);
  if constexpr (SIDES != 3) return wimg_bytes_rtp<SIDES, 3>(RTP, J, K, nrt, rb, lb);
}

}  // namespace

void tc_wimg_bytes(int RTP, int sides, int prec, int64_t J, int64_t K, int nrt, size_t* rb, size_t* lb) {
  *rb = 0;
  *lb = 0;
  if (prec == kTcTf32x3) return;
  const int L = limbs_of(prec);
  switch (sides) {
    case 1: return wimg_bytes_l<1>(RTP, L, J, K, nrt, rb, lb);
    case 2: return wimg_bytes_l<2>(RTP, L, J, K, nrt, rb, lb);
    case 3: return wimg_bytes_l<3>(RTP, L, J, K, nrt, rb, lb);
    default: return;
  }
}

cudaError_t launch_lead_tc_prep(const TcArgs& a, int RTP, int sides, int prec, int nsm, cudaStream_t st) {
  if (prec == kTcTf32x3) return cudaSuccess;
  const int L = limbs_of(prec);
  switch (sides) {
    case 1: return prep_ws_sides1(a, RTP, L, nsm, st);
    case 2: return prep_ws_sides2(a, RTP, L, nsm, st);
    case 3: return prep_ws_sides3(a, RTP, L, nsm, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_lead_tc(const float* Y, const TcArgs& a, int RTP, int sides, int prec, dim3 grid, cudaStream_t st) {
  if (prec == kTcTf32x3) return launch_lead_tf32(Y, a, RTP, sides, grid, st);
  CUtensorMap m{};
  TcArgs b = a;
  b.Y = Y;
  // One box = 32 KB: 128 rows x 64 columns (steps 4 and fused), 64 x 128 (step 7).
  const uint32_t ru = sides == 2 ? 64 : 128, cu = 8192 / ru;
  b.use_tma = make_matrix_map(&m, Y, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, a.J, a.K, ru, cu, CU_TENSOR_MAP_SWIZZLE_NONE,
                              a.ldy)
                  ? 1
                  : 0;
  const int L = limbs_of(prec);
  switch (sides) {
    case 1: return launch_ws_sides1(m, b, RTP, L, grid, st);
    case 2: return launch_ws_sides2(m, b, RTP, L, grid, st);
    case 3: return launch_ws_sides3(m, b, RTP, L, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace cpg
