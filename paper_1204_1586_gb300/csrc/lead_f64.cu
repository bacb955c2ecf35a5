// FP64 instances of the CUDA-core leading contraction (Algorithm 2 steps 4/7).
#include "lead_dispatch.cuh"
#include "lead_simt.cuh"
#include "tensor_map.h"

namespace cpg {

namespace {
template <int RT, int TJ, int SIDES>
cudaError_t run(const LeadArgs<double>& a, dim3 grid, cudaStream_t st) {
  using C = SimtCfg<double, RT, TJ, SIDES>;
  auto kern = lead_simt_kernel<double, RT, TJ, SIDES>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(C::smem_bytes));
  if (e != cudaSuccess) return e;
  // Tiles by TMA (box = one 128-byte line of TK columns) where Y allows it.
  CUtensorMap m{};
  LeadArgs<double> b = a;
  b.use_tma = make_matrix_map(&m, a.Y, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, int(sizeof(double)), a.J, a.K, uint32_t(C::SEG), uint32_t(C::TK),
                              CU_TENSOR_MAP_SWIZZLE_128B, a.ldy)
                  ? 1
                  : 0;
  return launch_pdl(kern, grid, dim3(C::NT), C::smem_bytes, st, m, b);
}

template <int RT, int TJ>
cudaError_t run_sides(const LeadArgs<double>& a, int sides, dim3 grid, cudaStream_t st) {
  switch (sides) {
    case 1: return run<RT, TJ, 1>(a, grid, st);
    case 2: return run<RT, TJ, 2>(a, grid, st);
    case 3: return run<RT, TJ, 3>(a, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

template <int RT, int TJ, int SIDES>
int bps() {
  using C = SimtCfg<double, RT, TJ, SIDES>;
  int n = 0;
  auto kern = lead_simt_kernel<double, RT, TJ, SIDES>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(C::smem_bytes)) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, C::NT, C::smem_bytes) != cudaSuccess || n < 1) {
    cudaGetLastError();
    return C::MIN_BLOCKS;
  }
  return n;
}

template <int RT, int TJ>
int bps_sides(int sides) {
  static int cache[4] = {0, 0, 0, 0};
  if (sides < 1 || sides > 3) return 1;
  if (cache[sides] == 0) cache[sides] = sides == 1 ? bps<RT, TJ, 1>() : sides == 2 ? bps<RT, TJ, 2>() : bps<RT, TJ, 3>();
  return cache[sides];
}

template <int RT, int TJ>
SimtShape shape(int sides) {
  using C = SimtCfg<double, RT, TJ, 3>;
  using CR = SimtCfg<double, RT, TJ, 1>;
  using CL = SimtCfg<double, RT, TJ, 2>;
  return sides == 1 ? SimtShape{RT, TJ, CR::TK, CR::smem_bytes, CR::LP, CR::WPRE}
         : sides == 2 ? SimtShape{RT, TJ, CL::TK, CL::smem_bytes, CL::LP, CL::WPRE}
                      : SimtShape{RT, TJ, C::TK, C::smem_bytes, C::LP, C::WPRE};
}
}  // namespace

SimtShape simt_shape_f64(int r, int sides) {
  if (r <= 4) return shape<4, 128>(sides);
  if (r <= 8) return shape<8, 128>(sides);
  return shape<16, 64>(sides);
}

int lead_blocks_per_sm_f64(int RT, int sides) {
  switch (RT) {
    case 4: return bps_sides<4, 128>(sides);
    case 8: return bps_sides<8, 128>(sides);
    case 16: return bps_sides<16, 64>(sides);
    default: return 1;
  }
}

cudaError_t launch_lead_f64(const LeadArgs<double>& a, int RT, int sides, dim3 grid, cudaStream_t st) {
  switch (RT) {
    case 4: return run_sides<4, 128>(a, sides, grid, st);
    case 8: return run_sides<8, 128>(a, sides, grid, st);
    case 16: return run_sides<16, 64>(a, sides, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace cpg
