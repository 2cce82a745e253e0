// Nodal-basis condensed operator in one kernel: Alg. (hdg_op_3d), the
// paper's HDG-TP variant (Sec. 4.2), FP64.
//
// Per element, with the six faces in the nodal (GLL) basis:
//   x-hat_f = (S^T M (x) S^T M) x_f                 six face transforms in
//   F_E     = sum_d d_d (B_S along d) x-hat_d       expansion (Sec. 4.1)
//   u_E     = D_Z^-1 F_E
//   r-hat_d = d_d H x-hat_d - d_d (B_S^T along d) u_E
//   r_f     = (M S (x) M S) r-hat_f                 six face transforms out
// and r_f is added onto the two elements' shared faces.  The face transforms
// are the identities S^-1 = S^T M and S^-T = M S of the generalised
// eigenproblem S^T M S = I (Eq. (generalized_eigenvalue_decomposition)), so
// the product equals K = (S^-T (x) S^-T) K-hat (S^-1 (x) S^-1) face by face,
// i.e. Alg. (hdg_op_3d_transformed) between the transforms.
//
// Cost per element: 12 face transforms of 2 n^3 multiply-adds each (the two
// neighbours of a face both transform it) plus the 25 n^3 of the transformed
// operator: the 73 n^3 flops of Tab. (operator_variants).  The face-wise
// alternative (transform every face once before and after the transformed
// kernel, three launches) does 49 n^3 per element and streams two more trace
// vectors; this kernel needs no workspace.
//
// Work split: one element per CTA slot, n^2 threads per slot; thread (a, b)
// owns face node (a, b) of all six faces (and the x1-line (j, k) = (a, b)
// in the expansion).  Shared faces receive exactly two red.global.add
// contributions onto a zeroed output (Neumann boundary faces one), so the
// result does not depend on the order of the elements.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace hdg {
namespace {

constexpr int kNodalMaxThreads = 320;

template <int N>
__host__ __device__ constexpr int nodal_slot_smem() {   // doubles per element slot
  return 12 * N * N + N * N * N;
}

template <int N>
__global__ void __launch_bounds__(kNodalMaxThreads, 1) tp_nodal_kernel(const NodalArgs a) {
  constexpr int N2 = N * N, NE = (N + 1) / 2;
  constexpr int R = dz_row(N, sizeof(double));
  constexpr int PER = nodal_slot_smem<N>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sm = reinterpret_cast<double*>(smem_raw);
  double* As = sm;        // S^T M, [mode][node]
  double* Bs = sm + N2;   // M S,   [node][mode]
  const int tid = threadIdx.x;
  for (int q = tid; q < N2; q += blockDim.x) {
    As[q] = a.StM.a[q];
    Bs[q] = a.MS.a[q];
  }

  const int slot = tid / N2;
  const int line = tid - slot * N2;
  const int lo = line % N, hi = line / N;
  const MeshDev& m = a.mesh;
  const long long nelem = (long long)m.ne[0] * m.ne[1] * m.ne[2];
  const long long e = (long long)blockIdx.x * a.epb + slot;
  const bool act = slot < a.epb && e < nelem;
  double* F = sm + 2 * N2 + (act ? slot : 0) * PER;   // six faces, node a + N b
  double* W = F + 6 * N2;                             // six faces, work
  double* U = W + 6 * N2;                             // eigenspace solution, i + N (j + N k)
  const int rhs = blockIdx.y;
  const double* xin = a.x + (long long)rhs * a.trace_stride;
  double* yout = a.y + (long long)rhs * a.trace_stride;

  // unknown-face offsets of the six faces (2 d + side), -1 on a Dirichlet plane
  int off[6] = {-1, -1, -1, -1, -1, -1};
  int e1 = 0, e2 = 0, e3 = 0;
  if (act) {
    e1 = (int)(e % m.ne[0]);
    e2 = (int)((e / m.ne[0]) % m.ne[1]);
    e3 = (int)(e / ((long long)m.ne[0] * m.ne[1]));
    const int ec[3] = {e1, e2, e3};
    const int fab[3] = {e2 + m.ne[1] * e3, e1 + m.ne[0] * e3, e1 + m.ne[0] * e2};
    const int pl[3] = {m.ne[1] * m.ne[2], m.ne[0] * m.ne[2], m.ne[0] * m.ne[1]};
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const int plane = ec[d] + s;
        if (plane >= m.lo[d] && plane <= m.hi[d])
          off[2 * d + s] = (int)((m.blk[d] + (long long)(plane - m.lo[d]) * pl[d] + fab[d]) * N2 + line);
      }
#pragma unroll
    for (int f = 0; f < 6; ++f) F[f * N2 + line] = off[f] >= 0 ? xin[off[f]] : 0.0;
  }
  __syncthreads();

  // transform in, first face axis: W[f][al + N b] = sum_a (S^T M)[al][a] F[f][a + N b]
  if (act) {
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      double v = 0.0;
#pragma unroll
      for (int c = 0; c < N; ++c) v = fma(As[lo * N + c], F[f * N2 + c + N * hi], v);
      W[f * N2 + line] = v;
    }
  }
  __syncthreads();
  // second face axis, then per direction the sum and difference of the two
  // sides (the parity split of B_S: even modes see S, odd modes D)
  if (act) {
    double v[6];
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      v[f] = 0.0;
#pragma unroll
      for (int c = 0; c < N; ++c) v[f] = fma(As[hi * N + c], W[f * N2 + lo + N * c], v[f]);
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      F[2 * d * N2 + line] = v[2 * d] + v[2 * d + 1];
      F[(2 * d + 1) * N2 + line] = v[2 * d] - v[2 * d + 1];
    }
  }
  __syncthreads();

  const double* mt = a.metric + (m.uniform ? 0 : 4 * e);
  const double d0 = act ? mt[0] : 0.0, d1 = act ? mt[1] : 0.0, d2 = act ? mt[2] : 0.0, d3 = act ? mt[3] : 0.0;
  // expansion and D_Z^-1 along the x1-line (j, k) = (lo, hi), x1 contraction
  double Pp = 0.0, Pm = 0.0;
  const double S1 = act ? F[line] : 0.0, D1 = act ? F[N2 + line] : 0.0;
  if (act) {
    const int j = lo, k = hi;
    const double Ap = d1 * S1, Am = d1 * D1;
    const double cjd2 = a.tab.c[j] * d2, ckd3 = a.tab.c[k] * d3;
    const double* Bsrc = F + (j < NE ? 2 : 3) * N2 + N * k;   // x2 face node (i, k)
    const double* Csrc = F + (k < NE ? 4 : 5) * N2 + N * j;   // x3 face node (i, j)
    const double* dz = a.dinv ? a.dinv + (long long)rhs * a.dinv_rhs_stride + (m.uniform ? 0 : e * (long long)(N2 * R)) +
                                    R * (j + N * k)
                              : nullptr;
    const double dzb = dz ? 0.0 : fma(d3, a.tab.lam[k], fma(d2, a.tab.lam[j], a.lam[rhs] * d0));
#pragma unroll
    for (int i = 0; i < N; ++i) {
      double FE = a.tab.c[i] * (i < NE ? Ap : Am);
      FE = fma(cjd2, Bsrc[i], FE);
      FE = fma(ckd3, Csrc[i], FE);
      const double u = FE * (dz ? dz[i] : 1.0 / fma(d1, a.tab.lam[i], dzb));
      U[i + N * line] = u;
      if (i < NE) Pp = fma(a.tab.c[i], u, Pp);
      else Pm = fma(a.tab.c[i], u, Pm);
    }
  }
  __syncthreads();

  // contractions onto the x2 face node (i, k) and the x3 face node (i, j),
  // (i, .) = (lo, hi), and the opposing-face term: r-hat of the six faces
  if (act) {
    const int i = lo, mm = hi;
    double Qp = 0.0, Qm = 0.0, Rp = 0.0, Rm = 0.0;
#pragma unroll
    for (int mo = 0; mo < N; ++mo) {
      const double uq = U[i + N * (mo + N * mm)];   // (i, j = mo, k = mm)
      const double ur = U[i + N * (mm + N * mo)];   // (i, j = mm, k = mo)
      if (mo < NE) { Qp = fma(a.tab.c[mo], uq, Qp); Rp = fma(a.tab.c[mo], ur, Rp); }
      else         { Qm = fma(a.tab.c[mo], uq, Qm); Rm = fma(a.tab.c[mo], ur, Rm); }
    }
    const double hs = a.tab.h0 + a.tab.h1, hd = a.tab.h0 - a.tab.h1;
    auto sides = [&](int d, double dd, double Sv, double Dv, double Pe, double Po) {
      const double sum = dd * (hs * Sv - 2.0 * Pe), dif = dd * (hd * Dv - 2.0 * Po);
      W[2 * d * N2 + line] = 0.5 * (sum + dif);
      W[(2 * d + 1) * N2 + line] = 0.5 * (sum - dif);
    };
    sides(0, d1, S1, D1, Pp, Pm);
    sides(1, d2, F[2 * N2 + line], F[3 * N2 + line], Qp, Qm);
    sides(2, d3, F[4 * N2 + line], F[5 * N2 + line], Rp, Rm);
  }
  __syncthreads();

  // transform out, first face axis: F[f][a + N be] = sum_al (M S)[a][al] W[f][al + N be]
  if (act) {
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      double v = 0.0;
#pragma unroll
      for (int c = 0; c < N; ++c) v = fma(Bs[lo * N + c], W[f * N2 + c + N * hi], v);
      F[f * N2 + line] = v;
    }
  }
  __syncthreads();
  // second face axis, added onto the shared faces
  if (act) {
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      double v = 0.0;
#pragma unroll
      for (int c = 0; c < N; ++c) v = fma(Bs[hi * N + c], F[f * N2 + lo + N * c], v);
      if (off[f] >= 0) red_add(yout + off[f], v);
    }
  }
}

template <int N>
cudaError_t nodal_launch(const NodalArgs& a0, int nrhs, cudaStream_t s) {
  NodalArgs a = a0;
  const long long nelem = (long long)a.mesh.ne[0] * a.mesh.ne[1] * a.mesh.ne[2];
  if (nelem <= 0) return cudaSuccess;
  constexpr int N2 = N * N;
  a.epb = std::max(1, kNodalMaxThreads / N2);
  const int threads = (a.epb * N2 + 31) / 32 * 32;
  const size_t smem = (size_t)(2 * N2 + a.epb * nodal_slot_smem<N>()) * sizeof(double);
  if (smem > kSmemOptIn) {
    const cudaError_t e =
        cudaFuncSetAttribute(tp_nodal_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const long long blocks = (nelem + a.epb - 1) / a.epb;
  tp_nodal_kernel<N><<<dim3((unsigned)blocks, (unsigned)nrhs), threads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_tp_nodal(int n, const NodalArgs& a, int nrhs, cudaStream_t s) {
  switch (n) {
    case 2: return nodal_launch<2>(a, nrhs, s);
    case 3: return nodal_launch<3>(a, nrhs, s);
    case 4: return nodal_launch<4>(a, nrhs, s);
    case 5: return nodal_launch<5>(a, nrhs, s);
    case 6: return nodal_launch<6>(a, nrhs, s);
    case 7: return nodal_launch<7>(a, nrhs, s);
    case 8: return nodal_launch<8>(a, nrhs, s);
    case 9: return nodal_launch<9>(a, nrhs, s);
    case 10: return nodal_launch<10>(a, nrhs, s);
    case 11: return nodal_launch<11>(a, nrhs, s);
    case 12: return nodal_launch<12>(a, nrhs, s);
    case 13: return nodal_launch<13>(a, nrhs, s);
    case 14: return nodal_launch<14>(a, nrhs, s);
    case 15: return nodal_launch<15>(a, nrhs, s);
    case 16: return nodal_launch<16>(a, nrhs, s);
    case 17: return nodal_launch<17>(a, nrhs, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace hdg
