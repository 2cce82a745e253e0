// Condensed HDG operator on one- and two-dimensional Cartesian meshes, FP64.
//
// 1D: Alg. (hdg_op_1d).  Per element of width h (d0 = h/2, d1 = 2/h) with
// face values x_lo, x_hi (single points, so the face basis needs no
// transform):
//   F_E = d1 B_S (x_lo, x_hi),  u_E = D_Z^-1 F_E,  D_Z = lambda d0 + d1 Lambda,
//   r   = d1 H (x_lo, x_hi) - d1 B_S^T u_E
// (Eq. (hdgkelement_factorized)).  With the eigenmodes ordered even-first,
// B_S[m] = c_m (1, sigma_m), so only S = x_lo + x_hi reaches the even modes
// and D = x_lo - x_hi the odd ones: the element reduces to the two sums
// a_even = sum c_m^2 / D_Z,m and a_odd, i.e. O(n) work per element.
//
// 2D: the transformed operator of Alg. (hdg_op_3d_transformed) with one
// direction fewer (d0 = h1 h2 / 4, d1 = h2 / h1, d2 = h1 / h2): the four
// edges of an element expand into its n x n eigenspace, D_Z^-1 scales, and
// the contractions give the edge residuals.  In the nodal basis every
// element transforms its own edges in (S^T M) and out (M S) first and last
// (Alg. (hdg_op_3d) with one direction fewer).  n threads per element: the
// thread of node t owns node t of all four edges and the x1-line j = t.
//
// Shared faces receive exactly two red.global.add contributions onto a
// zeroed output (boundary Neumann faces one): order independent.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace hdg {
namespace {

__global__ void lowdim1_kernel(const LowDimArgs a) {
  const int rhs = blockIdx.y;
  const double* x = a.x + (long long)rhs * a.trace_stride;
  double* y = a.y + (long long)rhs * a.trace_stride;
  const int n = a.n, ne = (n + 1) / 2;
  const double lam = a.lam[rhs];
  const double hs = a.tab.h0 + a.tab.h1, hd = a.tab.h0 - a.tab.h1;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < a.ne[0]; e += gridDim.x * blockDim.x) {
    const double d0 = a.metric[4 * e], d1 = a.metric[4 * e + 1];
    const int ol = (e >= a.lo[0] && e <= a.hi[0]) ? (int)a.blk[0] + e - a.lo[0] : -1;
    const int oh = (e + 1 >= a.lo[0] && e + 1 <= a.hi[0]) ? (int)a.blk[0] + e + 1 - a.lo[0] : -1;
    const double xl = ol >= 0 ? x[ol] : 0.0, xh = oh >= 0 ? x[oh] : 0.0;
    double ae = 0.0, ao = 0.0;
    for (int m = 0; m < n; ++m) {
      const double w = a.tab.c[m] * a.tab.c[m] / fma(d1, a.tab.lam[m], lam * d0);
      if (m < ne) ae += w;
      else ao += w;
    }
    const double S = xl + xh, D = xl - xh;
    const double sum = d1 * (hs * S - 2.0 * d1 * ae * S), dif = d1 * (hd * D - 2.0 * d1 * ao * D);
    if (ol >= 0) red_add(y + ol, 0.5 * (sum + dif));
    if (oh >= 0) red_add(y + oh, 0.5 * (sum - dif));
  }
}

template <int N>
__global__ void __launch_bounds__(256) lowdim2_kernel(const LowDimArgs a) {
  constexpr int NE = (N + 1) / 2;
  constexpr int PER = 12 * N + N * N;   // edges F[4][N], work W[4][N], S/D of x2 edges [4][N], U[N][N]
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sm = reinterpret_cast<double*>(smem_raw);
  const int tid = threadIdx.x;
  const int slot = tid / N, t = tid - slot * N;
  const long long nelem = (long long)a.ne[0] * a.ne[1];
  const long long e = (long long)blockIdx.x * a.epb + slot;
  const bool act = slot < a.epb && e < nelem;
  double* F = sm + (act ? slot : 0) * PER;
  double* W = F + 4 * N;
  double* SD = W + 4 * N;
  double* U = SD + 4 * N;
  const int rhs = blockIdx.y;
  const double* x = a.x + (long long)rhs * a.trace_stride;
  double* y = a.y + (long long)rhs * a.trace_stride;

  // offsets of node t of the four edges (x1-lo, x1-hi, x2-lo, x2-hi), -1 on Dirichlet planes
  int off[4] = {-1, -1, -1, -1};
  double d0 = 0.0, d1 = 0.0, d2 = 0.0;
  if (act) {
    const int e1 = (int)(e % a.ne[0]), e2 = (int)(e / a.ne[0]);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int p1 = e1 + s, p2 = e2 + s;
      if (p1 >= a.lo[0] && p1 <= a.hi[0]) off[s] = (int)((a.blk[0] + (long long)(p1 - a.lo[0]) * a.ne[1] + e2) * N + t);
      if (p2 >= a.lo[1] && p2 <= a.hi[1]) off[2 + s] = (int)((a.blk[1] + (long long)(p2 - a.lo[1]) * a.ne[0] + e1) * N + t);
    }
#pragma unroll
    for (int f = 0; f < 4; ++f) F[f * N + t] = off[f] >= 0 ? x[off[f]] : 0.0;
    d0 = a.metric[4 * e];
    d1 = a.metric[4 * e + 1];
    d2 = a.metric[4 * e + 2];
  }
  __syncthreads();
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  if (act) {
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      if (a.nodal) {   // edge transform in: x-hat[t] = sum_c (S^T M)[t][c] x[c]
        double s = 0.0;
#pragma unroll
        for (int c = 0; c < N; ++c) s = fma(a.StM.a[t * N + c], F[f * N + c], s);
        v[f] = s;
      } else {
        v[f] = F[f * N + t];
      }
    }
    SD[t] = v[2] + v[3];       // x2 edges, node i = t: sum and difference
    SD[N + t] = v[2] - v[3];
  }
  __syncthreads();

  // expansion along the x1-line j = t, D_Z^-1, x1 contraction
  const double S1 = v[0] + v[1], D1 = v[0] - v[1];
  double Pe = 0.0, Po = 0.0;
  const double lam = a.lam[rhs];
  if (act) {
    const int j = t;
    const double* src = SD + (j < NE ? 0 : N);
    const double cjd2 = a.tab.c[j] * d2;
    const double base = fma(d2, a.tab.lam[j], lam * d0);
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const double FE = fma(cjd2, src[i], a.tab.c[i] * d1 * (i < NE ? S1 : D1));
      const double u = FE / fma(d1, a.tab.lam[i], base);
      U[i + N * j] = u;
      if (i < NE) Pe = fma(a.tab.c[i], u, Pe);
      else Po = fma(a.tab.c[i], u, Po);
    }
  }
  __syncthreads();
  if (act) {
    const int i = t;
    double Qe = 0.0, Qo = 0.0;
#pragma unroll
    for (int j = 0; j < N; ++j) {
      if (j < NE) Qe = fma(a.tab.c[j], U[i + N * j], Qe);
      else Qo = fma(a.tab.c[j], U[i + N * j], Qo);
    }
    const double hs = a.tab.h0 + a.tab.h1, hd = a.tab.h0 - a.tab.h1;
    const double s1 = d1 * (hs * S1 - 2.0 * Pe), f1 = d1 * (hd * D1 - 2.0 * Po);
    const double s2 = d2 * (hs * SD[i] - 2.0 * Qe), f2 = d2 * (hd * SD[N + i] - 2.0 * Qo);
    W[t] = 0.5 * (s1 + f1);
    W[N + t] = 0.5 * (s1 - f1);
    W[2 * N + t] = 0.5 * (s2 + f2);
    W[3 * N + t] = 0.5 * (s2 - f2);
  }
  __syncthreads();
  if (act) {
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      double r;
      if (a.nodal) {   // edge transform out: r[t] = sum_c (M S)[t][c] r-hat[c]
        r = 0.0;
#pragma unroll
        for (int c = 0; c < N; ++c) r = fma(a.MS.a[t * N + c], W[f * N + c], r);
      } else {
        r = W[f * N + t];
      }
      if (off[f] >= 0) red_add(y + off[f], r);
    }
  }
}

template <int N>
cudaError_t lowdim2_launch(const LowDimArgs& a0, int nrhs, cudaStream_t s) {
  LowDimArgs a = a0;
  const long long nelem = (long long)a.ne[0] * a.ne[1];
  a.epb = std::max(1, 256 / N);
  const int threads = (a.epb * N + 31) / 32 * 32;
  const size_t smem = (size_t)a.epb * (12 * N + N * N) * sizeof(double);
  if (smem > kSmemOptIn) {
    const cudaError_t e =
        cudaFuncSetAttribute(lowdim2_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const long long blocks = (nelem + a.epb - 1) / a.epb;
  lowdim2_kernel<N><<<dim3((unsigned)blocks, (unsigned)nrhs), threads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_lowdim(const LowDimArgs& a, int nrhs, cudaStream_t s) {
  if (a.dim == 1) {
    if (a.ne[0] <= 0) return cudaSuccess;
    const int threads = 256;
    const int blocks = (int)std::min<long long>((a.ne[0] + threads - 1) / threads, 152LL * 8);
    lowdim1_kernel<<<dim3((unsigned)blocks, (unsigned)nrhs), threads, 0, s>>>(a);
    return cudaGetLastError();
  }
  if ((long long)a.ne[0] * a.ne[1] <= 0) return cudaSuccess;
  switch (a.n) {
    case 2: return lowdim2_launch<2>(a, nrhs, s);
    case 3: return lowdim2_launch<3>(a, nrhs, s);
    case 4: return lowdim2_launch<4>(a, nrhs, s);
    case 5: return lowdim2_launch<5>(a, nrhs, s);
    case 6: return lowdim2_launch<6>(a, nrhs, s);
    case 7: return lowdim2_launch<7>(a, nrhs, s);
    case 8: return lowdim2_launch<8>(a, nrhs, s);
    case 9: return lowdim2_launch<9>(a, nrhs, s);
    case 10: return lowdim2_launch<10>(a, nrhs, s);
    case 11: return lowdim2_launch<11>(a, nrhs, s);
    case 12: return lowdim2_launch<12>(a, nrhs, s);
    case 13: return lowdim2_launch<13>(a, nrhs, s);
    case 14: return lowdim2_launch<14>(a, nrhs, s);
    case 15: return lowdim2_launch<15>(a, nrhs, s);
    case 16: return lowdim2_launch<16>(a, nrhs, s);
    case 17: return lowdim2_launch<17>(a, nrhs, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace hdg
