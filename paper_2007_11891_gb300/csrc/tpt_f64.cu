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
long long tpt_blocks(long long nslots, int ppb) { return (nslots + ppb - 1) / ppb; }

void tpt_split(int n, const int ne[3], int nrhs, int* seg, int* nseg) {
  // enough x1-segments that all slots together hold about 152 SMs x 1536
  // threads (each slot has n^2 threads)
  const long long want = 152LL * 1536 / ((long long)n * n);
  const long long pencils = (long long)ne[1] * ne[2] * (nrhs > 0 ? nrhs : 1);
  long long per = (want + pencils - 1) / pencils;
  if (per < 1) per = 1;
  if (per > ne[0]) per = ne[0];
  *seg = (int)((ne[0] + per - 1) / per);
  *nseg = (ne[0] + *seg - 1) / *seg;
}

template <>
cudaError_t launch_tpt<double, double>(int mode, int n, TptArgs<double, double> a, int nrhs,
                                       cudaStream_t s) {
  return tpt_dispatch<double, double>(mode, n, a, nrhs, s);
}

}  // namespace hdg
