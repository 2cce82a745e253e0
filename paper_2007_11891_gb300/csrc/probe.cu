// Measurement support (not part of the method): the multiply-add rate this
// device sustains in FP64 and FP32, the denominator of the FP64 kernels'
// "alu" rooflines.  Every thread runs kChains independent dependency chains
// of fused multiply-adds on registers; the grid fills every SM with
// kProbeBlocksPerSm blocks.
#include <string>

#include "../../include/hdg.h"
#include "internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kProbeThreads = 256;
constexpr int kProbeBlocksPerSm = 4;

template <typename T>
__global__ void __launch_bounds__(kProbeThreads) fma_loop_kernel(T b, T c, int iters, T* sink) {
  T v[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) v[k] = T(threadIdx.x + k) * T(1e-3);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) v[k] = fma(v[k], b, c);
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += v[k];
  if (s == T(-12345.678)) sink[threadIdx.x] = s;   // keeps the loop; never true for these inputs
}

template <typename T>
hdg_status measure(int sms, double* out, cudaStream_t s) {
  const dim3 grid(sms * kProbeBlocksPerSm), block(kProbeThreads);
  // b slightly below one and c small: the chains stay finite and non-zero
  const T b = T(0.999999), c = T(1e-7);
  const int iters = sizeof(T) == 8 ? 4096 : 65536;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    hdg::set_last_error("hdg_measure_fma_peak: cudaEventCreate failed");
    return HDG_ERR_CUDA;
  }
  fma_loop_kernel<T><<<grid, block, 0, s>>>(b, c, iters, nullptr);   // warm-up (clocks ramp)
  const int reps = 5;
  cudaEventRecord(e0, s);
  for (int r = 0; r < reps; ++r) fma_loop_kernel<T><<<grid, block, 0, s>>>(b, c, iters, nullptr);
  cudaEventRecord(e1, s);
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) {
    hdg::set_last_error((std::string("hdg_measure_fma_peak: ") + cudaGetErrorString(e)).c_str());
    return HDG_ERR_CUDA;
  }
  const double flops = 2.0 * kChains * (double)iters * grid.x * block.x * reps;
  *out = flops / (ms * 1e-3) / 1e12;
  return HDG_OK;
}

}  // namespace

extern "C" hdg_status hdg_measure_fma_peak(hdg_precision prec, double* h_tflops, void* stream) {
  hdg::begin_entry();
  if (!h_tflops || (prec != HDG_FP64 && prec != HDG_FP32)) {
    hdg::set_last_error("hdg_measure_fma_peak: NULL output or precision other than FP64/FP32");
    return HDG_ERR_INVALID_ARG;
  }
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    hdg::set_last_error("hdg_measure_fma_peak: no device");
    return HDG_ERR_CUDA;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return prec == HDG_FP64 ? measure<double>(sms, h_tflops, s) : measure<float>(sms, h_tflops, s);
}
