// BF16-stored traces: the apply only (FP32 arithmetic, the element-run
// kernel of tpt_fast.cuh instantiated for bfloat16 storage).
#include "tpt_fast_launch.cuh"

namespace hdg {

template <>
int tpt_blocks_per_sm<float, float>(int mode, int n, int ppb);

template <>
int tpt_blocks_per_sm<float, __nv_bfloat16>(int mode, int n, int ppb) {
  return tpt_blocks_per_sm<float, float>(mode, n, ppb);
}

template <>
cudaError_t launch_tpt<float, __nv_bfloat16>(int mode, int n, TptArgs<float, __nv_bfloat16> a, int nrhs,
                                             cudaStream_t s) {
  if (mode != TPT_APPLY) return cudaErrorInvalidValue;
  if (a.variant == 3) return launch_tile_bf16(n, a, nrhs, s);
#define FLB(N) fast_dispatch_dz<N, __nv_bfloat16>(a, nrhs, s)
  FAST_N_SWITCH(n, FLB)
#undef FLB
  return cudaErrorInvalidValue;
}

}  // namespace hdg
