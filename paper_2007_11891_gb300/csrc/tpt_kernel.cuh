// Condensed HDG operator in the transformed face basis, one CTA slot per
// x1-pencil of elements (arXiv:2007.11891, Alg. (hdg_op_3d_transformed)).
//
// Per element e (metric factors d0..d3 of Sec. 3.2, eigenvalues Lambda of
// Eq. (generalized_eigenvalue_decomposition)):
//   F_E(i,j,k) = sum_s B_S[i][s] d1 x1_s(j,k) + B_S[j][s] d2 x2_s(i,k)
//              + B_S[k][s] d3 x3_s(i,j)                          (expand)
//   u_E = F_E / (lambda d0 + d1 Lambda_i + d2 Lambda_j + d3 Lambda_k)
//   r_{d,s} = d_d (H x_d)_s - d_d sum_m B_S[m][s] u_E              (contract)
// with H = G + C^T M^-1 C.  The eigenbasis is ordered [even | odd] modes so
// that B_S[m][1] = sigma_m B_S[m][0] =: sigma_m c_m; in the face sums
// S = x_lo + x_hi, D = x_lo - x_hi each expansion term is one FMA
// (c_m d S or c_m d D by the parity of m) and each contraction is one FMA
// into Q+ (even modes) or Q- (odd modes):
//   r_lo + r_hi = d ((h0 + h1) S - 2 Q+),  r_lo - r_hi = d ((h0 - h1) D - 2 Q-).
// That is 7 n^3 multiply-adds per element instead of the 25 n^3 flops
// (12 + 1 + 12 n^3) of the direct evaluation.
//
// Work split: a CTA slot marches over a segment of `seg` consecutive
// elements of one x1-pencil (n^2 threads, one per x1-line).  An x1-face
// inside a segment is shared by consecutive elements of the slot; the thread
// of a face node keeps its running sum in a register and stores it once.
// x1-faces on segment ends and all x2/x3 faces are shared with other slots:
// both contributions are added with red.global.add into an output zeroed
// before the launch (two adds onto zero commute exactly, so the result is
// deterministic).
//
// Modes:
//   TPT_APPLY   y = K-hat x (homogeneous Dirichlet data); optional fused
//               x^T y partial sums for CG.
//   TPT_RHS     y = -K-hat_{I,B} g-hat - (contraction of f-hat / D_Z): the
//               transformed right-hand side of Alg. (hdg_cg) / (hdg_transformed_cg)
//               with the Dirichlet lift (inputs: Dirichlet faces only).
//   TPT_RECOVER w = (f-hat - F_E(x, g-hat)) / D_Z, the eigenspace volume
//               solution of the recovery step of Alg. (hdg_cg).
#pragma once

#include "common.cuh"

namespace hdg {

enum TptMode { TPT_APPLY = 0, TPT_RHS = 1, TPT_RECOVER = 2 };

// CG hook: fused dot partials and the "last block finishes" reduction.
struct CgHook {
  double* partials;        // [nrhs][gridDim.x]
  unsigned int* counter;   // [nrhs], zero between launches
  double* pq;              // [nrhs] result: x^T K x
};

template <typename T, typename ST>
struct TptArgs {
  MeshDev mesh;
  Tables<T> tab;
  const T* metric;              // (d0, d1, d2, d3) per element, or one entry if uniform
  const T* dinv;                // D_Z^-1: n^3 per element (or one table if uniform)
  long long dinv_rhs_stride;    // per right-hand side
  const ST* x;                  // unknown-face inputs (APPLY, RECOVER)
  ST* y;                        // unknown-face outputs (APPLY, RHS)
  long long trace_stride;
  const T* gbd;                 // transformed Dirichlet data, boundary layout (RHS, RECOVER)
  long long bdry_stride;
  const T* src;                 // f-hat volume source (RHS, RECOVER)
  T* vout;                      // w volume output (RECOVER)
  long long vol_stride;
  int ppb;                      // pencil segments per block
  long long npencils;           // ne[1] * ne[2]
  int seg;                      // elements per pencil segment (x1 direction)
  int nseg;                     // segments per pencil = ceil(ne[0] / seg)
  const int* skip;              // per rhs: nonzero -> do nothing (converged), or null
  CgHook hook;                  // partials == null: no dot
};

template <int N>
__host__ __device__ constexpr int tpt_smem_per_pencil() {
  return 4 * N * N + N * N * N;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T, typename ST, int N, int MODE>
__global__ void __launch_bounds__(512) tpt_kernel(const TptArgs<T, ST> a) {
  constexpr int N2 = N * N, N3 = N2 * N, NE = (N + 1) / 2;
  constexpr int PER = tpt_smem_per_pencil<N>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);

  const int rhs = blockIdx.y;
  if (a.skip && a.skip[rhs]) return;   // uniform per block: no barrier is skipped partially

  const int tid = threadIdx.x;
  const int slot = tid / N2;
  const int line = tid - slot * N2;
  const long long slot_id = (long long)blockIdx.x * a.ppb + slot;
  const long long pencil = slot_id / a.nseg;
  const int sg = (int)(slot_id - pencil * a.nseg);
  const bool act = slot < a.ppb && pencil < a.npencils;
  const MeshDev& m = a.mesh;
  const int N1e = m.ne[0], N2e = m.ne[1], N3e = m.ne[2];
  const int e2 = act ? (int)(pencil % N2e) : 0;
  const int e3 = act ? (int)(pencil / N2e) : 0;
  const int e1s = act ? sg * a.seg : 0;
  const int e1e = act ? min(e1s + a.seg, N1e) : 0;

  T* S2p = sm + (act ? slot : 0) * PER;
  T* S2m = S2p + N2;
  T* S3p = S2m + N2;
  T* S3m = S3p + N2;
  T* U = S3m + N2;

  const long long toff = (long long)rhs * a.trace_stride;
  const ST* xin = (MODE == TPT_RHS) ? nullptr : a.x + toff;
  ST* yout = (MODE == TPT_RECOVER) ? nullptr : a.y + toff;
  const T* gin = (MODE == TPT_APPLY || a.gbd == nullptr) ? nullptr : a.gbd + (long long)rhs * a.bdry_stride;
  const T* dinv_r = a.dinv + (long long)rhs * a.dinv_rhs_stride;

  // face-plane strides per direction (faces per plane) and in-plane face index
  const long long pl0 = (long long)N2e * N3e, pl1 = (long long)N1e * N3e, pl2 = (long long)N1e * N2e;
  const long long f0 = e2 + (long long)N2e * e3;

  // read one face node: unknown plane -> x, Dirichlet boundary plane -> g-hat
  auto face_in = [&](int d, int plane, long long fab, long long pl) -> T {
    if (plane >= m.lo[d] && plane <= m.hi[d]) {
      if (MODE == TPT_RHS) return T(0);
      return load_as<ST, T>(xin + (m.blk[d] + (long long)(plane - m.lo[d]) * pl + fab) * N2 + line);
    }
    if (gin == nullptr) return T(0);
    const int side = 2 * d + (plane == 0 ? 0 : 1);
    return gin[(m.side[side] + fab) * N2 + line];
  };
  auto unknown = [&](int d, int plane) -> bool { return plane >= m.lo[d] && plane <= m.hi[d]; };

  T carry = T(0);
  T dot = T(0);
  T xlo1 = act ? face_in(0, e1s, f0, pl0) : T(0);

  // same trip count in every slot of the CTA (the loop holds barriers)
  for (int t = 0; t < a.seg; ++t) {
    const int e1 = e1s + t;
    const bool live = act && e1 < e1e;
    const long long elem = live ? e1 + (long long)N1e * (e2 + (long long)N2e * e3) : 0;
    const T* mt = a.metric + (m.uniform ? 0 : 4 * elem);
    const T d1 = mt[1], d2 = mt[2], d3 = mt[3];
    const long long f1 = e1 + (long long)N1e * e3;  // x2-face index in its plane
    const long long f2 = e1 + (long long)N1e * e2;  // x3-face index in its plane
    T xhi1 = T(0);
    if (live) {
      xhi1 = face_in(0, e1 + 1, f0, pl0);
      const T x2l = face_in(1, e2, f1, pl1), x2h = face_in(1, e2 + 1, f1, pl1);
      const T x3l = face_in(2, e3, f2, pl2), x3h = face_in(2, e3 + 1, f2, pl2);
      S2p[line] = x2l + x2h;
      S2m[line] = x2l - x2h;
      S3p[line] = x3l + x3h;
      S3m[line] = x3l - x3h;
    }
    __syncthreads();

    // expansion along the x1-line (j, k) = (line % N, line / N), x1 contraction
    const T S1 = xlo1 + xhi1, D1 = xlo1 - xhi1;
    T Pp = T(0), Pm = T(0);
    if (live) {
      const int j = line % N, k = line / N;
      const T Ap = d1 * S1, Am = d1 * D1;
      const T cjd2 = a.tab.c[j] * d2, ckd3 = a.tab.c[k] * d3;
      const T* Bs = (j < NE ? S2p : S2m) + N * k;
      const T* Cs = (k < NE ? S3p : S3m) + N * j;
      const T* dz = dinv_r + (m.uniform ? 0 : elem * N3) + N * j + N2 * k;
      const T* sr = (MODE == TPT_APPLY) ? nullptr
                                         : a.src + (long long)rhs * a.vol_stride + elem * N3 + N * j + N2 * k;
      T* Ur = U + N * j + N2 * k;
#pragma unroll
      for (int i = 0; i < N; ++i) {
        T F = a.tab.c[i] * (i < NE ? Ap : Am);
        F = fma(cjd2, Bs[i], F);
        F = fma(ckd3, Cs[i], F);
        if (MODE != TPT_APPLY) F -= sr[i];
        const T u = F * dz[i];
        Ur[i] = u;
        if (i < NE) Pp = fma(a.tab.c[i], u, Pp);
        else Pm = fma(a.tab.c[i], u, Pm);
      }
    }
    __syncthreads();

    if (live) {
      const int i = line % N, mm = line / N;
      if (MODE == TPT_RECOVER) {
        // w = (f-hat - F_E) / D_Z = -u ; thread (i, mm) writes points (i, mm, k)
        T* w = a.vout + (long long)rhs * a.vol_stride + elem * N3;
#pragma unroll
        for (int k = 0; k < N; ++k) w[i + N * mm + N2 * k] = -U[i + N * mm + N2 * k];
      } else {
        T Qp = T(0), Qm = T(0), Rp = T(0), Rm = T(0);
#pragma unroll
        for (int mo = 0; mo < N; ++mo) {
          const T uq = U[i + N * mo + N2 * mm];   // (i, j = mo, k = mm)
          const T ur = U[i + N * mm + N2 * mo];   // (i, j = mm, k = mo)
          if (mo < NE) { Qp = fma(a.tab.c[mo], uq, Qp); Rp = fma(a.tab.c[mo], ur, Rp); }
          else         { Qm = fma(a.tab.c[mo], uq, Qm); Rm = fma(a.tab.c[mo], ur, Rm); }
        }
        const T hs = a.tab.h0 + a.tab.h1, hd = a.tab.h0 - a.tab.h1;
        const T sgn = (MODE == TPT_RHS) ? T(-1) : T(1);
        const T two = T(2), half = T(0.5);
        // x2 faces (node (i, k = mm)) on planes e2, e2 + 1
        {
          const T S = S2p[line], D = S2m[line];
          const T sum = d2 * (hs * S - two * Qp), dif = d2 * (hd * D - two * Qm);
          if (unknown(1, e2))
            red_add(yout + (m.blk[1] + (long long)(e2 - m.lo[1]) * pl1 + f1) * N2 + line, sgn * half * (sum + dif));
          if (unknown(1, e2 + 1))
            red_add(yout + (m.blk[1] + (long long)(e2 + 1 - m.lo[1]) * pl1 + f1) * N2 + line, sgn * half * (sum - dif));
          if (MODE == TPT_APPLY) dot = fma(S, sum, fma(D, dif, dot));
        }
        // x3 faces (node (i, j = mm)) on planes e3, e3 + 1
        {
          const T S = S3p[line], D = S3m[line];
          const T sum = d3 * (hs * S - two * Rp), dif = d3 * (hd * D - two * Rm);
          if (unknown(2, e3))
            red_add(yout + (m.blk[2] + (long long)(e3 - m.lo[2]) * pl2 + f2) * N2 + line, sgn * half * (sum + dif));
          if (unknown(2, e3 + 1))
            red_add(yout + (m.blk[2] + (long long)(e3 + 1 - m.lo[2]) * pl2 + f2) * N2 + line, sgn * half * (sum - dif));
          if (MODE == TPT_APPLY) dot = fma(S, sum, fma(D, dif, dot));
        }
        // x1 faces (node (j, k) = line): running sum over the pencil
        {
          const T sum = d1 * (hs * S1 - two * Pp), dif = d1 * (hd * D1 - two * Pm);
          const T rlo = sgn * half * (sum + dif), rhi = sgn * half * (sum - dif);
          if (MODE == TPT_APPLY) dot = fma(S1, sum, fma(D1, dif, dot));
          // plane e1: inside the segment -> complete sum, store; segment start
          // -> shared with the previous segment (add), unless physical boundary
          if (unknown(0, e1)) {
            ST* dst = yout + (m.blk[0] + (long long)(e1 - m.lo[0]) * pl0 + f0) * N2 + line;
            if (t > 0) store_from<ST, T>(dst, carry + rlo);
            else if (e1 == 0) store_from<ST, T>(dst, rlo);
            else red_add(dst, rlo);
          }
          carry = rhi;
          if (e1 == e1e - 1 && unknown(0, e1e)) {
            ST* dst = yout + (m.blk[0] + (long long)(e1e - m.lo[0]) * pl0 + f0) * N2 + line;
            if (e1e == N1e) store_from<ST, T>(dst, carry);
            else red_add(dst, carry);
          }
        }
      }
    }
    xlo1 = xhi1;
    __syncthreads();
  }

  if (MODE == TPT_APPLY && a.hook.partials != nullptr) {
    // x^T y = sum over element faces of x . r = 1/2 sum (S sum + D dif)
    __shared__ double wsum[16];
    __shared__ bool last;
    T v = warp_sum(act ? dot : T(0));
    if ((tid & 31) == 0) wsum[tid >> 5] = (double)v;
    __syncthreads();
    if (tid == 0) {
      double s = 0.0;
      for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) s += wsum[w];
      a.hook.partials[(long long)rhs * gridDim.x + blockIdx.x] = 0.5 * s;
      __threadfence();
      const unsigned int done = atomicAdd(a.hook.counter + rhs, 1u);
      last = (done == gridDim.x - 1);
    }
    __syncthreads();
    if (last) {
      // the last block sums all partials: fixed strided split + fixed tree
      __threadfence();
      const volatile double* pp = a.hook.partials + (long long)rhs * gridDim.x;
      double s = 0.0;
      for (unsigned int b = tid; b < gridDim.x; b += blockDim.x) s += pp[b];
      s = warp_sum(s);
      __syncthreads();
      if ((tid & 31) == 0) wsum[tid >> 5] = s;
      __syncthreads();
      if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) t += wsum[w];
        a.hook.pq[rhs] = t;
        a.hook.counter[rhs] = 0u;
      }
    }
  }
}

}  // namespace hdg
