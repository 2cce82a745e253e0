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

void tpt_split(int n, const int ne[3], int nrhs, int ctas, int ppb, int* seg, int* nseg) {
  // CTAs hold ppb slots and run persistently (`ctas` resident at once); a
  // slot marches over `seg` elements.  Pick the segment length with the
  // least predicted time ceil(groups / ctas) x seg (in element steps),
  // preferring longer segments (more x1 faces summed in registers) on ties.
  const long long pencils = (long long)ne[1] * ne[2] * (nrhs > 0 ? nrhs : 1);
  if (ctas < 1) ctas = 1;
  long long best_cost = -1;
  int best = 1;
  for (int s = 1; s <= ne[0]; ++s) {
    const long long ns = (ne[0] + s - 1) / s;
    if (s > 1 && (ne[0] + s - 2) / (s - 1) == ns) continue;   // same split as a shorter segment
    const long long groups = (pencils * ns + ppb - 1) / ppb;
    const long long cost = (groups + ctas - 1) / ctas * s;
    if (best_cost < 0 || cost <= best_cost) {
      best_cost = cost;
      best = s;
    }
  }
  *seg = best;
  *nseg = (ne[0] + best - 1) / best;
}

template <>
int tpt_blocks_per_sm<double, double>(int mode, int n, int ppb) {
  return tpt_occupancy_dispatch<double, double>(mode, n, ppb);
}

template <>
cudaError_t launch_tpt<double, double>(int mode, int n, TptArgs<double, double> a, int nrhs,
                                       cudaStream_t s) {
  if (n > kMaxSpecialisedN || a.variant == 4) return launch_generic<double>(mode, n, a, nrhs, s);
  if (mode == TPT_APPLY && a.variant == 3) return launch_tile_f64(n, a, nrhs, s);
  return tpt_dispatch<double, double>(mode, n, a, nrhs, s);
}

}  // namespace hdg
