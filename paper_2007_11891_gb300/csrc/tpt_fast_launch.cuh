// Launch helpers of the FP32 element-run operator kernel (tpt_fast.cuh),
// shared by the FP32- and BF16-storage translation units, and the switch
// over the compiled degrees n = 2..17.
#pragma once

#include <algorithm>

#include "internal.h"
#include "tpt_fast.cuh"

namespace hdg {

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

// Dynamic shared memory of the element-run kernel with `ppb` slots: the
// staged faces and eigenspace solution per slot, and with the fused CG step
// (CGM = 1) each thread's staging area of 36 values.
template <int N, int CGM>
constexpr size_t fast_smem_bytes(int ppb) {
  return (size_t)ppb * (tpt_smem_per_pencil<float, N>() + (CGM ? 36 * fast_slot_threads(N) : 0)) * sizeof(float);
}

template <int N, bool DZC, int CGM = 0>
int fast_occupancy(int ppb) {
  static int cached[65] = {0};
  const int key = ppb < 64 ? ppb : 64;
  if (cached[key] > 0) return cached[key];
  const int threads = fast_threads(N, ppb);
  const size_t smem = fast_smem_bytes<N, CGM>(ppb);
  if (smem > kSmemOptIn)
    cudaFuncSetAttribute(tpt_fast_kernel<N, DZC, float, CGM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, tpt_fast_kernel<N, DZC, float, CGM>, threads, smem) !=
          cudaSuccess ||
      nb < 1) {
    cudaGetLastError();
    nb = 1;
  }
  cached[key] = nb;
  return nb;
}

template <int N, bool DZC, typename ST, int CGM = 0>
cudaError_t fast_launch(const TptArgs<float, ST>& a, int nrhs, cudaStream_t s) {
  const long long nelem = a.npencils * a.mesh.ne[0];
  if (nelem <= 0) return cudaSuccess;
  if (a.chunk < 1 || a.ppb < 1) return cudaErrorInvalidValue;
  const int threads = fast_threads(N, a.ppb);
  const size_t smem = fast_smem_bytes<N, CGM>(a.ppb);
  if (threads > fast_max_threads(N) || (fast_aligned(N) && a.ppb > 15)) return cudaErrorInvalidConfiguration;
  if (smem > kSmemOptIn) {
    cudaError_t e = cudaFuncSetAttribute(tpt_fast_kernel<N, DZC, ST, CGM>,
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
    return cudaLaunchKernelEx(&cfg, tpt_fast_kernel<N, DZC, ST, CGM>, a);
  }
  tpt_fast_kernel<N, DZC, ST, CGM><<<grid, threads, smem, s>>>(a);
  return cudaGetLastError();
}

template <int N, typename ST>
cudaError_t fast_dispatch_dz(const TptArgs<float, ST>& a, int nrhs, cudaStream_t s) {
  if constexpr (std::is_same<ST, float>::value) {
    if (a.cg == 1)
      return a.dinv ? fast_launch<N, false, ST, 1>(a, nrhs, s) : fast_launch<N, true, ST, 1>(a, nrhs, s);
  }
  if (a.cg != 0) return cudaErrorInvalidValue;
  return a.dinv ? fast_launch<N, false, ST>(a, nrhs, s) : fast_launch<N, true, ST>(a, nrhs, s);
}

}  // namespace hdg
