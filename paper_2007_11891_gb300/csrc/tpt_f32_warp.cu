// FP32 operator, one warp per element slot (tpt_warp.cuh): launcher and
// occupancy.
#include <algorithm>

#include "tpt_fast_launch.cuh"
#include "tpt_warp.cuh"

namespace hdg {
namespace {

// one warp per element slot, kWarpSlotsPerCta slots per CTA, runs of `chunk`
template <int N, bool DZC>
cudaError_t warp_launch(const TptArgs<float, float>& a, int nrhs, cudaStream_t s) {
  const long long nelem = a.npencils * a.mesh.ne[0];
  if (nelem <= 0) return cudaSuccess;
  if (a.chunk < 1 || a.ppb != kWarpSlotsPerCta) return cudaErrorInvalidValue;
  const int threads = kWarpSlotsPerCta * 32;
  const size_t smem = (size_t)kWarpSlotsPerCta * tpt_smem_per_pencil<float, N>() * sizeof(float);
  if (smem > kSmemOptIn) {
    cudaError_t e = cudaFuncSetAttribute(tpt_warp_kernel<N, DZC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  const long long blocks = (nelem + (long long)a.chunk * a.ppb - 1) / ((long long)a.chunk * a.ppb);
  dim3 grid((unsigned)blocks, (unsigned)nrhs);
  if (a.pdl) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, tpt_warp_kernel<N, DZC>, a);
  }
  tpt_warp_kernel<N, DZC><<<grid, threads, smem, s>>>(a);
  return cudaGetLastError();
}

template <int N>
int warp_occupancy() {
  static int cached = 0;
  if (cached > 0) return cached;
  const size_t smem = (size_t)kWarpSlotsPerCta * tpt_smem_per_pencil<float, N>() * sizeof(float);
  if (smem > kSmemOptIn)
    cudaFuncSetAttribute(tpt_warp_kernel<N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, tpt_warp_kernel<N, false>, kWarpSlotsPerCta * 32, smem) !=
          cudaSuccess ||
      nb < 1) {
    cudaGetLastError();
    nb = 1;
  }
  cached = nb;
  return nb;
}

template <int N>
cudaError_t warp_dispatch_dz(const TptArgs<float, float>& a, int nrhs, cudaStream_t s) {
  return a.dinv ? warp_launch<N, false>(a, nrhs, s) : warp_launch<N, true>(a, nrhs, s);
}

}  // namespace

int warp_slots_blocks_per_sm(int n) {
#define WO(N) warp_occupancy<N>()
  FAST_N_SWITCH(n, WO)
#undef WO
  return 1;
}

cudaError_t launch_tpt_warp_slots(int n, const TptArgs<float, float>& a, int nrhs, cudaStream_t s) {
#define WL(N) warp_dispatch_dz<N>(a, nrhs, s)
  FAST_N_SWITCH(n, WL)
#undef WL
  return cudaErrorInvalidValue;
}

}  // namespace hdg
