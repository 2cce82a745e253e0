// FP64 instantiations of the condensed operator, plus the shared launch
// geometry helpers.
#include "tpt_launch.cuh"

namespace hdg {

int tpt_ppb(int n) {
  const int n2 = n * n;
  int ppb = 256 / n2;
  return ppb < 1 ? 1 : ppb;
}
int tpt_threads(int n, int ppb) { return (ppb * n * n + 31) / 32 * 32; }
long long tpt_blocks(long long npencils, int ppb) { return (npencils + ppb - 1) / ppb; }

template <>
cudaError_t launch_tpt<double, double>(int mode, int n, TptArgs<double, double> a, int nrhs,
                                       cudaStream_t s) {
  return tpt_dispatch<double, double>(mode, n, a, nrhs, s);
}

}  // namespace hdg
