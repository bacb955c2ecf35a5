// FP32 instances of the CUDA-core leading contraction (Algorithm 2 steps 4/7).
#include "lead_dispatch.cuh"
#include "lead_simt.cuh"
#include "tensor_map.h"

namespace cpg {

namespace {
template <int RT, int TJ, int SIDES>
cudaError_t run(const LeadArgs<float>& a, dim3 grid, cudaStream_t st) {
  using C = SimtCfg<float, RT, TJ, SIDES>;
  auto kern = lead_simt_kernel<float, RT, TJ, SIDES>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(C::smem_bytes));
  if (e != cudaSuccess) return e;
  // Tiles by TMA (box = one 128-byte line of TK columns) where Y allows it.
  CUtensorMap m{};
  LeadArgs<float> b = a;
  b.use_tma = make_matrix_map(&m, a.Y, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, int(sizeof(float)), a.J, a.K, uint32_t(C::SEG), uint32_t(C::TK),
                              CU_TENSOR_MAP_SWIZZLE_128B, a.ldy)
                  ? 1
                  : 0;
  return launch_pdl(kern, grid, dim3(C::NT), C::smem_bytes, st, m, b);
}

// TJ: row tile of the R-side and fused instances; TJL: of the L-side-only
// instance (half-height tiles at small ranks: twice the columns per stage, so
// half the Khatri-Rao rows regenerated per stage of tall J-blocks).
template <int RT, int TJ, int TJL>
cudaError_t run_sides(const LeadArgs<float>& a, int sides, dim3 grid, cudaStream_t st) {
  switch (sides) {
    case 1: return run<RT, TJ, 1>(a, grid, st);
    case 2: return run<RT, TJL, 2>(a, grid, st);
    case 3: return run<RT, TJ, 3>(a, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

template <int RT, int TJ, int SIDES>
int bps() {
  using C = SimtCfg<float, RT, TJ, SIDES>;
  int n = 0;
  auto kern = lead_simt_kernel<float, RT, TJ, SIDES>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(C::smem_bytes)) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, C::NT, C::smem_bytes) != cudaSuccess || n < 1) {
    cudaGetLastError();
    return C::MIN_BLOCKS;
  }
  return n;
}

template <int RT, int TJ, int TJL>
int bps_sides(int sides) {
  static int cache[4] = {0, 0, 0, 0};
  if (sides < 1 || sides > 3) return 1;
  if (cache[sides] == 0)
    cache[sides] = sides == 1 ? bps<RT, TJ, 1>() : sides == 2 ? bps<RT, TJL, 2>() : bps<RT, TJ, 3>();
  return cache[sides];
}

template <int RT, int TJ, int TJL>
SimtShape shape(int sides) {
  using C = SimtCfg<float, RT, TJ, 3>;
  using CL = SimtCfg<float, RT, TJL, 2>;
  using CR = SimtCfg<float, RT, TJ, 1>;
  return sides == 2 ? SimtShape{RT, TJL, CL::TK, CL::smem_bytes, CL::LP, CL::WPRE}
         : sides == 1 ? SimtShape{RT, TJ, CR::TK, CR::smem_bytes, CR::LP, CR::WPRE}
                      : SimtShape{RT, TJ, C::TK, C::smem_bytes, C::LP, C::WPRE};
}
}  // namespace

#define CPG_F32_INSTANCES(X) \
  X(4, 256, 128) X(8, 256, 128) X(10, 128, 64) X(12, 128, 64) X(16, 128, 64) X(24, 128, 64) X(32, 64, 64) \
  X(48, 32, 32) X(64, 32, 32)

SimtShape simt_shape_f32(int r, int sides) {
#define CPG_SHAPE(RT, TJ, TJL) \
  if (r <= RT) return shape<RT, TJ, TJL>(sides);
  CPG_F32_INSTANCES(CPG_SHAPE)
#undef CPG_SHAPE
  return shape<64, 32, 32>(sides);
}

int lead_blocks_per_sm_f32(int RT, int sides) {
  switch (RT) {
#define CPG_BPS(RT_, TJ, TJL) \
  case RT_: return bps_sides<RT_, TJ, TJL>(sides);
    CPG_F32_INSTANCES(CPG_BPS)
#undef CPG_BPS
    default: return 1;
  }
}

cudaError_t launch_lead_f32(const LeadArgs<float>& a, int RT, int sides, dim3 grid, cudaStream_t st) {
  switch (RT) {
#define CPG_RUN(RT_, TJ, TJL) \
  case RT_: return run_sides<RT_, TJ, TJL>(a, sides, grid, st);
    CPG_F32_INSTANCES(CPG_RUN)
#undef CPG_RUN
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace cpg
