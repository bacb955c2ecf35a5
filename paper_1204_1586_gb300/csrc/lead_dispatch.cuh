// Host-side selection of the leading-contraction kernel instance.
#pragma once

#include "common.cuh"

namespace cpg {

// Tile shapes of the CUDA-core leading contraction for a rank tile RT.
struct SimtShape {
  int RT, TJ, TK;
  size_t smem;
  bool wl_rank_major;  // the instance's W_L rows are stored rank-major ([r][j])
  bool wpre;           // the instance takes Khatri-Rao rows built once per pass
};

// Smallest supported rank tile >= r (r <= max tile), and the row tile TJ and
// columns per stage TK of its instance for `sides`.
SimtShape simt_shape_f32(int r, int sides);
SimtShape simt_shape_f64(int r, int sides);
constexpr int kMaxRankTileF32 = 64;
constexpr int kMaxRankTileF64 = 16;

// Resident CTAs per SM of an instance (occupancy query; its design value
// when no device is present).
int lead_blocks_per_sm_f32(int RT, int sides);
int lead_blocks_per_sm_f64(int RT, int sides);

// sides: 1 = R side, 2 = L side, 3 = both.  grid = (nJb, nKs).
cudaError_t launch_lead_f32(const LeadArgs<float>& a, int RT, int sides, dim3 grid, cudaStream_t st);
cudaError_t launch_lead_f64(const LeadArgs<double>& a, int RT, int sides, dim3 grid, cudaStream_t st);

}  // namespace cpg
