// Host-side entry points of the tensor-core leading contraction.
#pragma once

#include "common.cuh"

namespace cpg {

struct TcArgs;

// Rank tile (MMA N of one product) for r rank columns: 16, 32 or 64.
int tc_rank_tile(int r);
// Largest number of 128-row tiles per J-block the fused kernel can keep in
// tensor memory (no limit for a single side).
int tc_max_nrt(int RTP, int sides, int prec);
// TMA needs a 16-byte aligned tensor and rows of whole 16-byte chunks.
// prec: 0 = BF16x3 split product, 1 = single BF16 product.
cudaError_t launch_lead_tc(const float* Y, const TcArgs& a, int RTP, int sides, int prec, dim3 grid, cudaStream_t st);

}  // namespace cpg
