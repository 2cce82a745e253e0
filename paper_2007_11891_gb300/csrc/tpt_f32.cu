// FP32 instantiations of the condensed operator: the specialised apply
// kernel (tpt_fast.cuh) for the inner CG, the generic kernel otherwise.
#include <algorithm>

#include "tpt_fast.cuh"
#include "tpt_launch.cuh"
#include "tpt_plane.cuh"
#include "tpt_warp.cuh"

namespace hdg {
namespace {

template <int N, bool DZC>
int fast_occupancy(int ppb) {
  static int cached[65] = {0};
  const int key = ppb < 64 ? ppb : 64;
  if (cached[key] > 0) return cached[key];
  const int threads = fast_threads(N, ppb);
  const size_t smem = (size_t)ppb * tpt_smem_per_pencil<float, N>() * sizeof(float);
  if (smem > kSmemOptIn)
    cudaFuncSetAttribute(tpt_fast_kernel<N, DZC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, tpt_fast_kernel<N, DZC>, threads, smem) !=
          cudaSuccess ||
      nb < 1) {
    cudaGetLastError();
    nb = 1;
  }
  cached[key] = nb;
  return nb;
}

template <int N, bool DZC, typename ST>
cudaError_t fast_launch(const TptArgs<float, ST>& a, int nrhs, cudaStream_t s) {
  const long long nelem = a.npencils * a.mesh.ne[0];
  if (nelem <= 0) return cudaSuccess;
  if (a.chunk < 1 || a.ppb < 1) return cudaErrorInvalidValue;
  const int threads = fast_threads(N, a.ppb);
  const size_t smem = (size_t)a.ppb * tpt_smem_per_pencil<float, N>() * sizeof(float);
  if (threads > fast_max_threads(N) || (fast_aligned(N) && a.ppb > 15)) return cudaErrorInvalidConfiguration;
  if (smem > kSmemOptIn) {
    cudaError_t e = cudaFuncSetAttribute(tpt_fast_kernel<N, DZC, ST>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  // one run of `chunk` elements per slot: every element is covered exactly once
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
    return cudaLaunchKernelEx(&cfg, tpt_fast_kernel<N, DZC, ST>, a);
  }
  tpt_fast_kernel<N, DZC, ST><<<grid, threads, smem, s>>>(a);
  return cudaGetLastError();
}

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

template <int N>
cudaError_t plane_dispatch_dz(const TptArgs<float, float>& a, int nrhs, cudaStream_t s) {
  TptArgs<float, float> b = a;
  b.ppb = a.ppb > 0 ? a.ppb : std::max(1, 64 / N);
  return a.dinv ? plane_launch<N, false>(b, nrhs, s) : plane_launch<N, true>(b, nrhs, s);
}

template <int N, typename ST>
cudaError_t fast_dispatch_dz(const TptArgs<float, ST>& a, int nrhs, cudaStream_t s) {
  return a.dinv ? fast_launch<N, false, ST>(a, nrhs, s) : fast_launch<N, true, ST>(a, nrhs, s);
}

#define FAST_N_SWITCH(n, CALL)                                                  \
  switch (n) {                                                                  \
    case 2: return CALL(2); case 3: return CALL(3); case 4: return CALL(4);     \
    case 5: return CALL(5); case 6: return CALL(6); case 7: return CALL(7);     \
    case 8: return CALL(8); case 9: return CALL(9); case 10: return CALL(10);   \
    case 11: return CALL(11); case 12: return CALL(12); case 13: return CALL(13); \
    case 14: return CALL(14); case 15: return CALL(15); case 16: return CALL(16); \
    case 17: return CALL(17);                                                   \
    default: break;                                                             \
  }

}  // namespace

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

int warp_slots_blocks_per_sm(int n) {
#define WO(N) warp_occupancy<N>()
  FAST_N_SWITCH(n, WO)
#undef WO
  return 1;
}

template <>
cudaError_t launch_tpt<float, float>(int mode, int n, TptArgs<float, float> a, int nrhs, cudaStream_t s) {
  if (mode == TPT_APPLY && a.variant == 2) {
#define WL(N) warp_dispatch_dz<N>(a, nrhs, s)
    FAST_N_SWITCH(n, WL)
#undef WL
    return cudaErrorInvalidValue;
  }
  if (mode == TPT_APPLY && a.variant == 1) {
#define PL(N) plane_dispatch_dz<N>(a, nrhs, s)
    FAST_N_SWITCH(n, PL)
#undef PL
    return cudaErrorInvalidValue;
  }
  if (mode == TPT_APPLY) {
#define FL(N) fast_dispatch_dz<N, float>(a, nrhs, s)
    FAST_N_SWITCH(n, FL)
#undef FL
    return cudaErrorInvalidValue;
  }
  return tpt_dispatch<float, float>(mode, n, a, nrhs, s);
}

// BF16-stored traces: the apply only (FP32 arithmetic, same kernel)
template <>
int tpt_blocks_per_sm<float, __nv_bfloat16>(int mode, int n, int ppb) {
  return tpt_blocks_per_sm<float, float>(mode, n, ppb);
}

template <>
cudaError_t launch_tpt<float, __nv_bfloat16>(int mode, int n, TptArgs<float, __nv_bfloat16> a, int nrhs,
                                             cudaStream_t s) {
  if (mode != TPT_APPLY) return cudaErrorInvalidValue;
#define FLB(N) fast_dispatch_dz<N, __nv_bfloat16>(a, nrhs, s)
  FAST_N_SWITCH(n, FLB)
#undef FLB
  return cudaErrorInvalidValue;
}

}  // namespace hdg
