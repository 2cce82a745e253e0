// FP32 instantiations of the condensed operator: the element-run apply
// kernel (tpt_fast.cuh), the generic kernel (tpt_kernel.cuh) for the other
// modes; the tile kernel (tpt_tile_f32.cu) and the BF16-storage
// instantiations (tpt_bf16.cu) live in translation units of their own so that
// the build compiles them in parallel.
#include "tpt_fast_launch.cuh"
#include "tpt_launch.cuh"

namespace hdg {

template <>
int tpt_blocks_per_sm<float, float>(int mode, int n, int ppb) {
  if (mode == TPT_APPLY) {
    // the table and in-kernel variants have the same footprint
#define OCC(N) fast_occupancy<N, false>(ppb)
    FAST_N_SWITCH(n, OCC)
#undef OCC
    return 1;
  }
  return tpt_occupancy_dispatch<float, float>(mode, n, ppb);
}

// CTAs per SM of the element-run kernel with the fused CG step (its
// staging areas take extra shared memory); the lower of the two D_Z^-1 forms
int fast_fused_blocks_per_sm(int n, int ppb) {
#define OCC(N) std::min(fast_occupancy<N, false, 1>(ppb), fast_occupancy<N, true, 1>(ppb))
  FAST_N_SWITCH(n, OCC)
#undef OCC
  return 1;
}

template <>
cudaError_t launch_tpt<float, float>(int mode, int n, TptArgs<float, float> a, int nrhs, cudaStream_t s) {
  if (n > kMaxSpecialisedN || a.variant == 4) return launch_generic<float>(mode, n, a, nrhs, s);
  if (mode == TPT_APPLY && a.variant == 3) return launch_tile_f32(n, a, nrhs, s);
  if (mode == TPT_APPLY) {
#define FL(N) fast_dispatch_dz<N, float>(a, nrhs, s)
    FAST_N_SWITCH(n, FL)
#undef FL
    return cudaErrorInvalidValue;
  }
  return tpt_dispatch<float, float>(mode, n, a, nrhs, s);
}

}  // namespace hdg
