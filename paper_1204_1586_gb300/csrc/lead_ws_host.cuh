// Host side of the warp-specialised split-BF16 leading contraction: one
// launcher per (rank tile, sides, limbs) instance.
#pragma once

#include "lead_ws.cuh"
#include "tensor_map.h"

namespace cpg {

template <int RTP, int SIDES, int L>
cudaError_t run_ws(const CUtensorMap& m, const TcArgs& a, dim3 grid, cudaStream_t st) {
  using C = WsCfg<RTP, SIDES, L>;
  auto kern = lead_ws_kernel<RTP, SIDES, L>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(C::smem_bytes));
  if (e != cudaSuccess) return e;
  return launch_pdl(kern, grid, dim3(C::NT), C::smem_bytes, st, m, a);
}

template <int SIDES, int L>
cudaError_t run_ws_rtp(const CUtensorMap& m, const TcArgs& a, int RTP, dim3 grid, cudaStream_t st) {
  switch (RTP) {
    case 16: return run_ws<16, SIDES, L>(m, a, grid, st);
    case 32: return run_ws<32, SIDES, L>(m, a, grid, st);
    case 64:
      if constexpr (SIDES != 3) return run_ws<64, SIDES, L>(m, a, grid, st);
      return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
}

// Instances of one SIDES value (lead_ws1.cu, lead_ws2.cu, lead_ws3.cu).
cudaError_t launch_ws_sides1(const CUtensorMap& m, const TcArgs& a, int RTP, int L, dim3 grid, cudaStream_t st);
cudaError_t launch_ws_sides2(const CUtensorMap& m, const TcArgs& a, int RTP, int L, dim3 grid, cudaStream_t st);
cudaError_t launch_ws_sides3(const CUtensorMap& m, const TcArgs& a, int RTP, int L, dim3 grid, cudaStream_t st);

}  // namespace cpg
