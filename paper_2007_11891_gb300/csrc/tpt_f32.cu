// FP32 instantiations of the condensed operator.
#include "tpt_launch.cuh"

namespace hdg {

template <>
int tpt_blocks_per_sm<float, float>(int mode, int n, int ppb) {
  return tpt_occupancy_dispatch<float, float>(mode, n, ppb);
}

template <>
cudaError_t launch_tpt<float, float>(int mode, int n, TptArgs<float, float> a, int nrhs, cudaStream_t s) {
  return tpt_dispatch<float, float>(mode, n, a, nrhs, s);
}

}  // namespace hdg
