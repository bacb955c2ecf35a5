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
                              CU_TENSOR_MAP_SWIZZLE_128B)
                  ? 1
                  : 0;
  kern<<<grid, C::NT, C::smem_bytes, st>>>(m, b);
  return cudaGetLastError();
}

template <int RT, int TJ>
cudaError_t run_sides(const LeadArgs<float>& a, int sides, dim3 grid, cudaStream_t st) {
  switch (sides) {
    case 1: return run<RT, TJ, 1>(a, grid, st);
    case 2: return run<RT, TJ, 2>(a, grid, st);
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

template <int RT, int TJ>
int bps_sides(int sides) {
  static int cache[4] = {0, 0, 0, 0};
  if (sides < 1 || sides > 3) return 1;
  if (cache[sides] == 0) cache[sides] = sides == 1 ? bps<RT, TJ, 1>() : sides == 2 ? bps<RT, TJ, 2>() : bps<RT, TJ, 3>();
  return cache[sides];
}

template <int RT, int TJ>
SimtShape shape() {
  using C = SimtCfg<float, RT, TJ, 3>;
  return SimtShape{RT, TJ, C::TK, C::smem_bytes};
}
}  // namespace

SimtShape simt_shape_f32(int r) {
  if (r <= 4) return shape<4, 256>();
  if (r <= 8) return shape<8, 256>();
  if (r <= 10) return shape<10, 128>();
  if (r <= 12) return shape<12, 128>();
  if (r <= 16) return shape<16, 128>();
  if (r <= 24) return shape<24, 64>();
  if (r <= 32) return shape<32, 64>();
  if (r <= 48) return shape<48, 32>();
  return shape<64, 32>();
}

int lead_blocks_per_sm_f32(int RT, int sides) {
  switch (RT) {
    case 4: return bps_sides<4, 256>(sides);
    case 8: return bps_sides<8, 256>(sides);
    case 10: return bps_sides<10, 128>(sides);
    case 12: return bps_sides<12, 128>(sides);
    case 16: return bps_sides<16, 128>(sides);
    case 24: return bps_sides<24, 64>(sides);
    case 32: return bps_sides<32, 64>(sides);
    case 48: return bps_sides<48, 32>(sides);
    case 64: return bps_sides<64, 32>(sides);
    default: return 1;
  }
}

cudaError_t launch_lead_f32(const LeadArgs<float>& a, int RT, int sides, dim3 grid, cudaStream_t st) {
  switch (RT) {
    case 4: return run_sides<4, 256>(a, sides, grid, st);
    case 8: return run_sides<8, 256>(a, sides, grid, st);
    case 10: return run_sides<10, 128>(a, sides, grid, st);
    case 12: return run_sides<12, 128>(a, sides, grid, st);
    case 16: return run_sides<16, 128>(a, sides, grid, st);
    case 24: return run_sides<24, 64>(a, sides, grid, st);
    case 32: return run_sides<32, 64>(a, sides, grid, st);
    case 48: return run_sides<48, 32>(a, sides, grid, st);
    case 64: return run_sides<64, 32>(a, sides, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace cpg
