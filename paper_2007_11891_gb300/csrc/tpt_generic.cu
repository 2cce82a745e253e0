// Runtime-degree operator (tpt_generic.cuh) for FP64 and FP32, every mode:
// the degrees above the specialised instantiations (p = 17..32).
#include <algorithm>

#include "internal.h"
#include "tpt_generic.cuh"

namespace hdg {

namespace {

template <typename T, int MODE>
cudaError_t generic_one(int n, const TptArgs<T, T>& a, int nrhs, cudaStream_t s) {
  const long long nelem = (long long)a.mesh.ne[0] * a.mesh.ne[1] * a.mesh.ne[2];
  if (nelem <= 0) return cudaSuccess;
  if (n < 2 || n > kMaxNDev) return cudaErrorInvalidValue;
  const size_t smem = (size_t)6 * n * n * sizeof(T);
  if (smem > kSmemOptIn) {
    const cudaError_t e = cudaFuncSetAttribute(tpt_generic_kernel<T, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem);
    if (e != cudaSuccess) return e;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tpt_generic_kernel<T, MODE>, kGenericThreads, smem) !=
          cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    sms = 152;
  cudaGetLastError();
  // one resident wave of CTAs per right-hand side row (grid-stride over elements)
  const long long per_rhs = std::max(1LL, (long long)sms * per_sm / std::max(nrhs, 1));
  const dim3 grid((unsigned)std::min(nelem, per_rhs), (unsigned)nrhs);
  tpt_generic_kernel<T, MODE><<<grid, kGenericThreads, smem, s>>>(a, n);
  return cudaGetLastError();
}

}  // namespace

template <typename T>
cudaError_t launch_generic(int mode, int n, const TptArgs<T, T>& a, int nrhs, cudaStream_t s) {
  switch (mode) {
    case TPT_APPLY: return generic_one<T, TPT_APPLY>(n, a, nrhs, s);
    case TPT_RHS: return generic_one<T, TPT_RHS>(n, a, nrhs, s);
    case TPT_RECOVER: return generic_one<T, TPT_RECOVER>(n, a, nrhs, s);
    default: return cudaErrorInvalidValue;
  }
}
template cudaError_t launch_generic<double>(int, int, const TptArgs<double, double>&, int, cudaStream_t);
template cudaError_t launch_generic<float>(int, int, const TptArgs<float, float>&, int, cudaStream_t);

}  // namespace hdg
