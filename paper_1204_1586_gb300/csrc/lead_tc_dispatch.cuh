// Host-side entry points of the tensor-core leading contractions.
#pragma once

#include "common.cuh"

namespace cpg {

struct TcArgs;

// Tensor-core precision codes of a leading pass: 0 = BF16x3 (two BF16 limbs),
// 1 = BF16 (one limb), 2 = TF32x3 (split TF32, lead_tf32.cu), 3 = BF16x6
// (three BF16 limbs).
constexpr int kTcBf16x3 = 0, kTcBf16 = 1, kTcTf32x3 = 2, kTcBf16x6 = 3;

// Rank tile (MMA N of one product) for r rank columns: 16, 32 or 64.
int tc_rank_tile(int r);
// Rows and columns of one stage for (prec, sides).
int tc_tile_rows(int prec, int sides);
int tc_tile_cols(int prec, int sides);
// Largest number of running sums a CTA keeps in tensor memory: row tiles of a
// J-block (step 4, and the fused pass, which needs one more for step 7) or
// column chunks (step 7).
int tc_max_acc(int RTP, int sides, int prec);
// Whether one pass can compute steps 4 and 7 for (RTP, prec), and how many row
// tiles per J-block it can keep the step-7 Khatri-Rao tiles of.
bool tc_fused_ok(int RTP, int prec);
int tc_fused_max_nrt(int RTP, int prec);
// Split-BF16 passes: bytes of the prebuilt Khatri-Rao B tiles (R side, L
// side, for J-blocks of nrt row tiles; 0 for TF32x3) and the launches that
// build them (a.wimg_r / a.wimg_l,
// from a.wr / a.wl for ranks a.r0 ..) ahead of the pass.
void tc_wimg_bytes(int RTP, int sides, int prec, int64_t J, int64_t K, int nrt, size_t* rb, size_t* lb);
cudaError_t launch_lead_tc_prep(const TcArgs& a, int RTP, int sides, int prec, int nsm, cudaStream_t st);
// TMA needs a 16-byte aligned tensor and rows of whole 16-byte chunks; other
// tensors are read with element loads.
cudaError_t launch_lead_tc(const float* Y, const TcArgs& a, int RTP, int sides, int prec, dim3 grid, cudaStream_t st);
// The split-TF32 kernel (lead_tf32.cu): row tiles of 128 x 64 (step 4) or
// 64 x 128 (step 7), one side per pass.
cudaError_t launch_lead_tf32(const float* Y, const TcArgs& a, int RTP, int sides, dim3 grid, cudaStream_t st);

}  // namespace cpg
