// Host side of the split-TF32 leading contraction: TMA tensor map of Y and the
// kernel instances (rank tile 16 / 32 / 64, step 4 or step 7).
#include "lead_tc_dispatch.cuh"
#include "lead_tf32.cuh"
#include "tensor_map.h"

namespace cpg {

namespace {

template <int RTP, int SIDES>
cudaError_t run(const TcArgs& a, dim3 grid, cudaStream_t st) {
  using C = Tf32Cfg<RTP, SIDES>;
  // Tensor-memory columns: one accumulator of 2 RTP columns per row tile
  // (step 4) or per column chunk (step 7), at most 512.
  const int64_t nacc = SIDES == 1 ? a.nrt : (a.Kc + C::TKS - 1) / C::TKS;
  if (nacc < 1 || nacc * C::NW > 512) return cudaErrorInvalidValue;
  CUtensorMap m{};
  TcArgs b = a;
  // Box = {32 rows (128 bytes), TKS columns}, 128-byte swizzle; element copies
  // into the same layout when rows are not whole 16-byte chunks.
  b.use_tma = make_matrix_map(&m, a.Y, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, a.J, a.K, 32, uint32_t(C::TKS),
                              CU_TENSOR_MAP_SWIZZLE_128B, a.ldy)
                  ? 1
                  : 0;
  auto kern = lead_tf32_kernel<RTP, SIDES>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(C::smem_bytes));
  if (e != cudaSuccess) return e;
  return launch_pdl(kern, grid, dim3(C::NT), C::smem_bytes, st, m, b);
}

template <int RTP>
cudaError_t run_sides(const TcArgs& a, int sides, dim3 grid, cudaStream_t st) {
  switch (sides) {
    case 1: return run<RTP, 1>(a, grid, st);
    case 2: return run<RTP, 2>(a, grid, st);
    default: return cudaErrorInvalidValue;  // no fused form: two passes
  }
}

}  // namespace

cudaError_t launch_lead_tf32(const float* Y, const TcArgs& a, int RTP, int sides, dim3 grid, cudaStream_t st) {
  TcArgs b = a;
  b.Y = Y;
  switch (RTP) {
    case 16: return run_sides<16>(b, sides, grid, st);
    case 32: return run_sides<32>(b, sides, grid, st);
    case 64: return run_sides<64>(b, sides, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace cpg
