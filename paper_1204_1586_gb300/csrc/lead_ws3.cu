// Instances of the warp-specialised split-BF16 leading kernel for SIDES = 3.
#include "lead_ws_host.cuh"

namespace cpg {

cudaError_t launch_ws_sides3(const CUtensorMap& m, const TcArgs& a, int RTP, int L, dim3 grid, cudaStream_t st) {
  switch (L) {
    case 1: return run_ws_rtp<3, 1>(m, a, RTP, grid, st);
    case 2: return run_ws_rtp<3, 2>(m, a, RTP, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t prep_ws_sides3(const TcArgs& a, int RTP, int L, int nsm, cudaStream_t st) {
  switch (L) {
    case 1: return prep_ws_rtp<3, 1>(a, RTP, nsm, st);
    case 2: return prep_ws_rtp<3, 2>(a, RTP, nsm, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace cpg
