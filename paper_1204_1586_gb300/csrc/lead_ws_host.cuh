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

// Tiles of the prebuilt B operands: W_R over the K columns of Y (KWR
// entries per tile), W_L over the row tiles of every J-block (nrt tiles of
// KWL rows each; the last J-block's may pass J and are zero).
template <int RTP, int SIDES, int L>
int64_t wimg_tiles_r(int64_t K) {
  using C = WsCfg<RTP, SIDES, L>;
  return C::DO_R ? (K + C::KWR - 1) / C::KWR : 0;
}
template <int RTP, int SIDES, int L>
int64_t wimg_tiles_l(int64_t J, int nrt) {
  using C = WsCfg<RTP, SIDES, L>;
  return C::DO_L ? (J + int64_t(C::KWL) * nrt - 1) / (int64_t(C::KWL) * nrt) * nrt : 0;
}

// The pass's prebuilt B tiles (ws_wimg_kernel).
template <int RTP, int SIDES, int L>
cudaError_t prep_ws(const TcArgs& a, int nsm, cudaStream_t st) {
  using C = WsCfg<RTP, SIDES, L>;
  if constexpr (C::DO_R) {
    const int64_t nt = wimg_tiles_r<RTP, SIDES, L>(a.K);
    const cudaError_t e = launch_pdl(ws_wimg_kernel<RTP, L, C::KWR>, dim3(unsigned(std::min<int64_t>(nt, 4 * nsm))),
                                     dim3(256), 0, st, a.wimg_r, a.wr, a.K, a.r0, a.R, nt);
    if (e != cudaSuccess) return e;
  }
  if constexpr (C::DO_L) {
    const int64_t nt = wimg_tiles_l<RTP, SIDES, L>(a.J, a.nrt);
    const cudaError_t e = launch_pdl(ws_wimg_kernel<RTP, L, C::KWL>, dim3(unsigned(std::min<int64_t>(nt, 4 * nsm))),
                                     dim3(256), 0, st, a.wimg_l, a.wl, a.J, a.r0, a.R, nt);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Bytes of the prebuilt B tiles of one pass (R side, L side).
template <int RTP, int SIDES, int L>
void wimg_bytes(int64_t J, int64_t K, int nrt, size_t* rb, size_t* lb) {
  using C = WsCfg<RTP, SIDES, L>;
  *rb = size_t(wimg_tiles_r<RTP, SIDES, L>(K)) * C::WIMG_R_STRIDE;
  *lb = size_t(wimg_tiles_l<RTP, SIDES, L>(J, nrt)) * C::WIMG_L_STRIDE;
}

template <int SIDES, int L>
cudaError_t prep_ws_rtp(const TcArgs& a, int RTP, int nsm, cudaStream_t st) {
  switch (RTP) {
    case 16: return prep_ws<16, SIDES, L>(a, nsm, st);
    case 32: return prep_ws<32, SIDES, L>(a, nsm, st);
    case 64:
      if constexpr (SIDES != 3) return prep_ws<64, SIDES, L>(a, nsm, st);
      return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
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
cudaError_t prep_ws_sides1(const TcArgs& a, int RTP, int L, int nsm, cudaStream_t st);
cudaError_t prep_ws_sides2(const TcArgs& a, int RTP, int L, int nsm, cudaStream_t st);
cudaError_t prep_ws_sides3(const TcArgs& a, int RTP, int L, int nsm, cudaStream_t st);

}  // namespace cpg
