// Host side of the tensor-core leading contraction: TMA tensor map of Y and
// the kernel instances (rank tile 16 / 32 / 64, sides, BF16x3 or BF16); the
// split-TF32 form is forwarded to lead_tf32.cu.
#include "lead_tc.cuh"
#include "lead_tc_dispatch.cuh"
#include "tensor_map.h"

namespace cpg {

namespace {

// Y as a 2-D tensor [K][J] (J contiguous); one box = 128 rows x 64 columns.
bool make_y_map(CUtensorMap* m, const float* Y, int64_t J, int64_t K, int64_t ldy) {
  return make_matrix_map(m, Y, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, J, K, 128, 64, CU_TENSOR_MAP_SWIZZLE_NONE, ldy);
}

template <int RTP, int SIDES, int PREC>
cudaError_t run(const CUtensorMap& m, const TcArgs& a, dim3 grid, cudaStream_t st) {
  using C = TcCfg<RTP, SIDES, PREC>;
  auto kern = lead_tc_kernel<RTP, SIDES, PREC>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(C::smem_bytes));
  if (e != cudaSuccess) return e;
  return launch_pdl(kern, grid, dim3(C::NT), C::smem_bytes, st, m, a);
}

template <int RTP, int PREC>
cudaError_t run_sides(const CUtensorMap& m, const TcArgs& a, int sides, dim3 grid, cudaStream_t st) {
  switch (sides) {
    case 1: return run<RTP, 1, PREC>(m, a, grid, st);
    case 2: return run<RTP, 2, PREC>(m, a, grid, st);
    case 3: return run<RTP, 3, PREC>(m, a, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

template <int RTP>
cudaError_t run_prec(const CUtensorMap& m, const TcArgs& a, int sides, int prec, dim3 grid, cudaStream_t st) {
  return prec == 0 ? run_sides<RTP, 0>(m, a, sides, grid, st) : run_sides<RTP, 1>(m, a, sides, grid, st);
}

}  // namespace

int tc_rank_tile(int r) { return r <= 16 ? 16 : r <= 32 ? 32 : 64; }

int tc_max_nrt(int RTP, int sides, int prec) {
  const int nw = (prec == 1) ? RTP : 2 * RTP;
  if (sides == 2) return 1 << 20;     // row tiles are outer: any number per CTA
  return sides == 1 ? 512 / nw : 512 / nw - 2;  // fused: two step-7 accumulators
}

int tc_tile_rows(int prec, int sides) { return prec == 2 ? (sides == 1 ? 128 : 64) : 128; }
int tc_tile_cols(int prec, int sides) { return prec == 2 ? (sides == 1 ? 64 : 128) : 128; }

cudaError_t launch_lead_tc(const float* Y, const TcArgs& a, int RTP, int sides, int prec, dim3 grid, cudaStream_t st) {
  if (prec == 2) return launch_lead_tf32(Y, a, RTP, sides, grid, st);
  CUtensorMap m{};
  TcArgs b = a;
  b.Y = Y;
  b.use_tma = make_y_map(&m, Y, a.J, a.K, a.ldy) ? 1 : 0;  // else element copies (rows not 16-byte aligned)
  switch (RTP) {
    case 16: return run_prec<16>(m, b, sides, prec, grid, st);
    case 32: return run_prec<32>(m, b, sides, prec, grid, st);
    case 64: return run_prec<64>(m, b, sides, prec, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace cpg
