// FP32 operator, x2-plane work split (tpt_plane.cuh): launcher.
#include <algorithm>

#include "tpt_fast_launch.cuh"
#include "tpt_plane.cuh"

namespace hdg {
namespace {

// x2-plane kernel: `ppb` elements per CTA (n threads each; 0 = 64 / n),
// one resident wave striding over the elements
template <int N, bool DZC>
cudaError_t plane_launch(const TptArgs<float, float>& a0, int nrhs, cudaStream_t s) {
  TptArgs<float, float> a = a0;
  const long long nelem = a.npencils * a.mesh.ne[0];
  if (nelem <= 0) return cudaSuccess;
  if (a.ppb < 1) return cudaErrorInvalidValue;
  const int threads = (a.ppb * N + 31) / 32 * 32;
  if (threads > 128) return cudaErrorInvalidConfiguration;
  const size_t smem = (size_t)a.ppb * plane_smem_per_elem<N>() * sizeof(float);
  if (smem > kSmemOptIn) {
    cudaError_t e = cudaFuncSetAttribute(tpt_plane_kernel<N, DZC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  static int per_sm[2] = {0, 0};
  static int sms = 0;
  static int cached_ppb[2] = {-1, -1};
  if (cached_ppb[DZC] != a.ppb) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      sms = 152;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[DZC], tpt_plane_kernel<N, DZC>, threads, smem) !=
            cudaSuccess || per_sm[DZC] < 1)
      per_sm[DZC] = 1;
    cudaGetLastError();
    cached_ppb[DZC] = a.ppb;
  }
  long long blocks = (nelem + a.ppb - 1) / a.ppb;
  blocks = std::min<long long>(blocks, (long long)sms * per_sm[DZC]);
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
    return cudaLaunchKernelEx(&cfg, tpt_plane_kernel<N, DZC>, a);
  }
  tpt_plane_kernel<N, DZC><<<grid, threads, smem, s>>>(a);
  return cudaGetLastError();
}

template <int N>
cudaError_t plane_dispatch_dz(const TptArgs<float, float>& a, int nrhs, cudaStream_t s) {
  TptArgs<float, float> b = a;
  b.ppb = a.ppb > 0 ? a.ppb : std::max(1, 64 / N);
  return a.dinv ? plane_launch<N, false>(b, nrhs, s) : plane_launch<N, true>(b, nrhs, s);
}

}  // namespace

cudaError_t launch_tpt_planes(int n, const TptArgs<float, float>& a, int nrhs, cudaStream_t s) {
#define PL(N) plane_dispatch_dz<N>(a, nrhs, s)
  FAST_N_SWITCH(n, PL)
#undef PL
  return cudaErrorInvalidValue;
}

}  // namespace hdg
