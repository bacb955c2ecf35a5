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
// prec: 0 = BF16x3 split product, 1 = single BF16 product, 2 = TF32x3 split
// product (one side per pass: sides 1 or 2).
cudaError_t launch_lead_tc(const float* Y, const TcArgs& a, int RTP, int sides, int prec, dim3 grid, cudaStream_t st);
// The split-TF32 kernel (lead_tf32.cu): rows tiles of 128 x 64 (step 4) or
// 64 x 128 (step 7).
cudaError_t launch_lead_tf32(const float* Y, const TcArgs& a, int RTP, int sides, dim3 grid, cudaStream_t st);
// Row and column extent of one super-stage of the tensor-core kernel for
// (prec, sides).
int tc_tile_rows(int prec, int sides);
int tc_tile_cols(int prec, int sides);

}  // namespace cpg
