// Launch helpers for tpt_kernel: one translation unit per precision includes
// this file and instantiates launch_tpt<T, ST> for n = 2..17.
#pragma once

#include "internal.h"

namespace hdg {

template <typename T, typename ST, int N, int MODE>
cudaError_t tpt_launch_one(const TptArgs<T, ST>& a, int nrhs, cudaStream_t s) {
  if (a.npencils <= 0) return cudaSuccess;
  const int threads = tpt_threads(N, a.ppb);
  const size_t smem = (size_t)a.ppb * tpt_smem_per_pencil<T, N>() * sizeof(T);
  if (threads > 320) return cudaErrorInvalidConfiguration;
  if (smem > kSmemOptIn) {
    cudaError_t e = cudaFuncSetAttribute(tpt_kernel<T, ST, N, MODE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  if (a.seg < 1 || a.nseg < 1) return cudaErrorInvalidValue;
  long long blocks = tpt_blocks(a.npencils * a.nseg, a.ppb);
  if (a.max_grid > 0 && blocks > a.max_grid) blocks = a.max_grid;
  dim3 grid((unsigned)blocks, (unsigned)nrhs);
  tpt_kernel<T, ST, N, MODE><<<grid, threads, smem, s>>>(a);
  return cudaGetLastError();
}

// resident CTAs per SM of one instantiation (cached per process)
template <typename T, typename ST, int N, int MODE>
int tpt_occupancy_one(int ppb) {
  static int cached[65] = {0};
  const int key = ppb < 64 ? ppb : 64;
  if (cached[key] > 0) return cached[key];
  const int threads = tpt_threads(N, ppb);
  const size_t smem = (size_t)ppb * tpt_smem_per_pencil<T, N>() * sizeof(T);
  if (smem > kSmemOptIn)
    cudaFuncSetAttribute(tpt_kernel<T, ST, N, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, tpt_kernel<T, ST, N, MODE>, threads, smem) != cudaSuccess ||
      nb < 1) {
    cudaGetLastError();
    nb = 1;
  }
  cached[key] = nb;
  return nb;
}

template <typename T, typename ST, int N>
int tpt_occupancy_mode(int mode, int ppb) {
  switch (mode) {
    case TPT_APPLY: return tpt_occupancy_one<T, ST, N, TPT_APPLY>(ppb);
    case TPT_RHS: return tpt_occupancy_one<T, ST, N, TPT_RHS>(ppb);
    default: return tpt_occupancy_one<T, ST, N, TPT_RECOVER>(ppb);
  }
}

template <typename T, typename ST>
int tpt_occupancy_dispatch(int mode, int n, int ppb) {
  switch (n) {
    case 2: return tpt_occupancy_mode<T, ST, 2>(mode, ppb);
    case 3: return tpt_occupancy_mode<T, ST, 3>(mode, ppb);
    case 4: return tpt_occupancy_mode<T, ST, 4>(mode, ppb);
    case 5: return tpt_occupancy_mode<T, ST, 5>(mode, ppb);
    case 6: return tpt_occupancy_mode<T, ST, 6>(mode, ppb);
    case 7: return tpt_occupancy_mode<T, ST, 7>(mode, ppb);
    case 8: return tpt_occupancy_mode<T, ST, 8>(mode, ppb);
    case 9: return tpt_occupancy_mode<T, ST, 9>(mode, ppb);
    case 10: return tpt_occupancy_mode<T, ST, 10>(mode, ppb);
    case 11: return tpt_occupancy_mode<T, ST, 11>(mode, ppb);
    case 12: return tpt_occupancy_mode<T, ST, 12>(mode, ppb);
    case 13: return tpt_occupancy_mode<T, ST, 13>(mode, ppb);
    case 14: return tpt_occupancy_mode<T, ST, 14>(mode, ppb);
    case 15: return tpt_occupancy_mode<T, ST, 15>(mode, ppb);
    case 16: return tpt_occupancy_mode<T, ST, 16>(mode, ppb);
    case 17: return tpt_occupancy_mode<T, ST, 17>(mode, ppb);
    default: return 1;
  }
}

template <typename T, typename ST, int N>
cudaError_t tpt_launch_mode(int mode, const TptArgs<T, ST>& a, int nrhs, cudaStream_t s) {
  switch (mode) {
    case TPT_APPLY: return tpt_launch_one<T, ST, N, TPT_APPLY>(a, nrhs, s);
    case TPT_RHS: return tpt_launch_one<T, ST, N, TPT_RHS>(a, nrhs, s);
    case TPT_RECOVER: return tpt_launch_one<T, ST, N, TPT_RECOVER>(a, nrhs, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T, typename ST>
cudaError_t tpt_dispatch(int mode, int n, const TptArgs<T, ST>& a, int nrhs, cudaStream_t s) {
  switch (n) {
    case 2: return tpt_launch_mode<T, ST, 2>(mode, a, nrhs, s);
    case 3: return tpt_launch_mode<T, ST, 3>(mode, a, nrhs, s);
    case 4: return tpt_launch_mode<T, ST, 4>(mode, a, nrhs, s);
    case 5: return tpt_launch_mode<T, ST, 5>(mode, a, nrhs, s);
    case 6: return tpt_launch_mode<T, ST, 6>(mode, a, nrhs, s);
    case 7: return tpt_launch_mode<T, ST, 7>(mode, a, nrhs, s);
    case 8: return tpt_launch_mode<T, ST, 8>(mode, a, nrhs, s);
    case 9: return tpt_launch_mode<T, ST, 9>(mode, a, nrhs, s);
    case 10: return tpt_launch_mode<T, ST, 10>(mode, a, nrhs, s);
    case 11: return tpt_launch_mode<T, ST, 11>(mode, a, nrhs, s);
    case 12: return tpt_launch_mode<T, ST, 12>(mode, a, nrhs, s);
    case 13: return tpt_launch_mode<T, ST, 13>(mode, a, nrhs, s);
    case 14: return tpt_launch_mode<T, ST, 14>(mode, a, nrhs, s);
    case 15: return tpt_launch_mode<T, ST, 15>(mode, a, nrhs, s);
    case 16: return tpt_launch_mode<T, ST, 16>(mode, a, nrhs, s);
    case 17: return tpt_launch_mode<T, ST, 17>(mode, a, nrhs, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace hdg
