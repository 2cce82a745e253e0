// Condensed operator for any degree (runtime n, up to kMaxNDev points per
// direction), used above the degrees the specialised kernels are built for
// (arXiv:2007.11891, Alg. (hdg_op_3d_transformed); modes as tpt_kernel.cuh).
//
// One CTA per element (grid-stride over elements).  The element's six faces
// are staged as sums S = x_lo + x_hi and differences D = x_lo - x_hi per
// direction (6 n^2 values in shared memory).  The eigenspace solution
// u = F / D_Z is never stored: for each direction d, every thread takes
// x_d-lines of the element, recomputes u along its line from the staged
// faces,
//   F(i,j,k) = c_i d1 (S1|D1)(j,k) + c_j d2 (S2|D2)(i,k) + c_k d3 (S3|D3)(i,j)
//              [- f-hat(i,j,k) in the RHS / RECOVER modes],
//   D_Z(i,j,k) = lambda d0 + d1 Lambda_i + d2 Lambda_j + d3 Lambda_k,
// and contracts it along the line into the even/odd sums Q+ / Q- of its face
// node, which give the face residuals r_lo + r_hi = d (hs S - 2 Q+),
// r_lo - r_hi = d (hd D - 2 Q-).  That is three evaluations of u per point
// instead of one, in exchange for O(n^2) shared memory per element, which is
// what lets the degree go past the n^3 eigenspace arrays the other kernels
// keep (n = 33: 36k values per element).  D_Z^-1 is a division per point.
// Every face value is added to a zeroed output with red.global.add (two
// contributions per shared face, which commute: deterministic).
#pragma once

#include "tpt_kernel.cuh"

namespace hdg {

constexpr int kGenericThreads = 256;

template <typename T, int MODE>
__global__ void __launch_bounds__(kGenericThreads) tpt_generic_kernel(const TptArgs<T, T> a, int n) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* FS = reinterpret_cast<T*>(smem_raw);   // [d][s][n^2]: S (s = 0) and D (s = 1) of direction d
  const int n2 = n * n, ne_ = (n + 1) / 2;
  const int rhs = blockIdx.y;
  if (a.skip && a.skip[rhs]) return;
  __shared__ CgScalars s_cg;
  const HookPre hpre = (MODE == TPT_APPLY) ? hook_prefetch(a.hook, rhs, &s_cg) : HookPre{0.0};
  const MeshDev& m = a.mesh;
  const int N1e = m.ne[0], N2e = m.ne[1], N3e = m.ne[2];
  const int pl0 = N2e * N3e, pl1 = N1e * N3e, pl2 = N1e * N2e;
  const long long nelem = (long long)N1e * pl0;
  const long long toff = (long long)rhs * a.trace_stride;
  const T* xin = (MODE == TPT_RHS) ? nullptr : a.x + toff;
  T* yout = (MODE == TPT_RECOVER) ? nullptr : a.y + toff;
  const T* gin = (MODE == TPT_APPLY || a.gbd == nullptr) ? nullptr : a.gbd + (long long)rhs * a.bdry_stride;
  const T lam_r = static_cast<T>(a.lam[rhs]);
  const T hs = a.tab.h0 + a.tab.h1, hd = a.tab.h0 - a.tab.h1;
  const T sgn = (MODE == TPT_RHS) ? T(-1) : T(1);
  T dot = T(0);

  for (long long e = blockIdx.x; e < nelem; e += gridDim.x) {
    const int e1 = (int)(e % N1e), rest = (int)(e / N1e), e2 = rest % N2e, e3 = rest / N2e;
    // unknown-face base of direction d on `plane` (or -1), Dirichlet-face base (or -1)
    auto uface = [&](int d, int plane, int fab, int pl) -> long long {
      return (plane >= m.lo[d] && plane <= m.hi[d]) ? (m.blk[d] + (long long)(plane - m.lo[d]) * pl + fab) * n2 : -1;
    };
    auto gface = [&](int d, int plane, int fab) -> long long {
      if (gin == nullptr || (plane >= m.lo[d] && plane <= m.hi[d])) return -1;
      return (m.side[2 * d + (plane == 0 ? 0 : 1)] + fab) * n2;
    };
    const int fab[3] = {e2 + N2e * e3, e1 + N1e * e3, e1 + N1e * e2};
    const int pls[3] = {pl0, pl1, pl2};
    const int ed[3] = {e1, e2, e3};
    long long ou[3][2], og[3][2];
    for (int d = 0; d < 3; ++d)
      for (int s = 0; s < 2; ++s) {
        ou[d][s] = uface(d, ed[d] + s, fab[d], pls[d]);
        og[d][s] = gface(d, ed[d] + s, fab[d]);
      }
    const T* mt = a.metric + (m.uniform ? 0 : 4 * e);
    const T d0 = mt[0], dd[3] = {mt[1], mt[2], mt[3]};
    // stage S and D of the six faces
    for (int t = threadIdx.x; t < 3 * n2; t += blockDim.x) {
      const int d = t / n2, q = t - d * n2;
      T v[2];
      for (int s = 0; s < 2; ++s) {
        v[s] = T(0);
        if (MODE != TPT_RHS && ou[d][s] >= 0) v[s] = xin[ou[d][s] + q];
        else if (MODE != TPT_APPLY && og[d][s] >= 0) v[s] = gin[og[d][s] + q];
      }
      FS[(2 * d) * n2 + q] = v[0] + v[1];
      FS[(2 * d + 1) * n2 + q] = v[0] - v[1];
    }
    __syncthreads();
    const T* src = (MODE == TPT_APPLY) ? nullptr : a.src + (long long)rhs * a.vol_stride + e * (long long)(n2 * n);
    T* wout = (MODE == TPT_RECOVER) ? a.vout + (long long)rhs * a.vol_stride + e * (long long)(n2 * n) : nullptr;
    // lines along direction d (RECOVER: x1 only, writing w = (f-hat - F) / D_Z = -u)
    const int ndir = (MODE == TPT_RECOVER) ? 1 : 3;
    for (int d = 0; d < ndir; ++d) {
      for (int line = threadIdx.x; line < n2; line += blockDim.x) {
        const int la = line % n, lb = line / n;   // the line's face node (lower axis la)
        T Qp = T(0), Qm = T(0);
        for (int t = 0; t < n; ++t) {
          int i, j, k;
          if (d == 0) { i = t; j = la; k = lb; }
          else if (d == 1) { i = la; j = t; k = lb; }
          else { i = la; j = lb; k = t; }
          const T s1 = FS[(i < ne_ ? 0 : 1) * n2 + j + n * k];
          const T s2 = FS[(2 + (j < ne_ ? 0 : 1)) * n2 + i + n * k];
          const T s3 = FS[(4 + (k < ne_ ? 0 : 1)) * n2 + i + n * j];
          T F = a.tab.c[i] * dd[0] * s1;
          F = fma(a.tab.c[j] * dd[1], s2, F);
          F = fma(a.tab.c[k] * dd[2], s3, F);
          if (MODE != TPT_APPLY) F -= src[i + n * j + n2 * k];
          const T den = fma(dd[2], a.tab.lam[k], fma(dd[1], a.tab.lam[j], fma(dd[0], a.tab.lam[i], lam_r * d0)));
          const T u = F / den;
          if (MODE == TPT_RECOVER) {
            wout[i + n * j + n2 * k] = -u;
          } else {
            if (t < ne_) Qp = fma(a.tab.c[t], u, Qp);
            else Qm = fma(a.tab.c[t], u, Qm);
          }
        }
        if (MODE != TPT_RECOVER) {
          const T Sv = FS[(2 * d) * n2 + line], Dv = FS[(2 * d + 1) * n2 + line];
          const T sum = dd[d] * (hs * Sv - T(2) * Qp), dif = dd[d] * (hd * Dv - T(2) * Qm);
          if (ou[d][0] >= 0) red_add(yout + ou[d][0] + line, sgn * T(0.5) * (sum + dif));
          if (ou[d][1] >= 0) red_add(yout + ou[d][1] + line, sgn * T(0.5) * (sum - dif));
          if (MODE == TPT_APPLY) dot = fma(Sv, sum, fma(Dv, dif, dot));
        }
      }
    }
    __syncthreads();   // the next element restages FS
  }
  if (MODE == TPT_APPLY && a.hook.partials != nullptr) hook_finish(a.hook, rhs, dot, hpre, &s_cg);
}

}  // namespace hdg
