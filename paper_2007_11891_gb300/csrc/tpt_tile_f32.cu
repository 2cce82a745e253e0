// Tile operator kernel (tpt_tile.cuh) instantiated for FP32 arithmetic and storage,
// degrees n = 2..17, in a translation unit of its own so that the build
// compiles the precisions in parallel.
#include "tpt_tile_launch.cuh"

namespace hdg {

cudaError_t launch_tile_f32(int n, const TptArgs<float, float>& a, int nrhs, cudaStream_t s) {
#define TL(N) tile_dispatch_dz<float, float, N>(a, nrhs, a.sms, a.tile, s)
  TILE_N_SWITCH(n, TL)
#undef TL
  return cudaErrorInvalidValue;
}

}  // namespace hdg
