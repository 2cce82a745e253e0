// FP32 operator application y = K-hat x (Alg. (hdg_op_3d_transformed)) with
// one thread per x2-plane of an element: n threads per element, thread j
// owning the points (i, j, k) for all i, k.
//
// Per element e and thread j (notation of tpt_kernel.cuh; S/D are face sums
// and differences of the lo and hi faces, c the parity-split B_S column):
//   for k:  F(i) = c_i d1 (S1 | D1)(j, k) + c_j d2 (S2 | D2)(i, k)
//                + c_k d3 (S3 | D3)(i, j)            (| by the parity of the
//                                                      mode index in front)
//           u(i) = F(i) / D_Z(i, j, k)
//           P(j, k) = sum_i c_i u(i)        -> x1-face node (j, k), here
//           U[k][j][i] = u(i)               -> shared memory
//   then    R(i, j) = sum_k c_k U[k][j][i]      -> x3-face nodes (i, j)
//           Q(i, k = j) = sum_jj c_jj U[j][jj][i] -> x2-face nodes (i, j)
// The x1 contraction runs along the thread's own points; the other two read
// the element's U back with 16-byte shared-memory loads.  The element's data are read once: the thread's x1 column
// (j, .), x3 row (., j) and x2 row (., k = j) of both faces of each
// direction; x2 rows are shared through shared memory.  All face outputs are
// red.global.add onto a zeroed output (two adds per face, which commute
// exactly: deterministic).  x^T y partial sums as in tpt_fast.cuh.
//
// Elements per CTA: `ppb` (n threads each); the grid strides over elements.
#pragma once

#include "tpt_kernel.cuh"

namespace hdg {

// shared memory per element: S2+ and S2- rows (2 n rows of R) and U (n^2 rows of R)
template <int N>
__host__ __device__ constexpr int plane_smem_per_elem() {
  return (2 * N + N * N) * dz_row(N, sizeof(float));
}

// At most 128 threads per CTA and three resident CTAs per SM: up to 168
// registers per thread, so that a thread's row data, its next D_Z^-1 rows
// and the unrolled point loop stay in registers.
template <int N, bool DZC>
__global__ void __launch_bounds__(128, 3) tpt_plane_kernel(const TptArgs<float, float> a) {
  constexpr int N2 = N * N, NE = (N + 1) / 2;
  constexpr int R = dz_row(N, sizeof(float));
  constexpr int NQ = R / 4;
  constexpr int PER = plane_smem_per_elem<N>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sm = reinterpret_cast<float*>(smem_raw);

  const int rhs = blockIdx.y;
  grid_dep_wait();   // everything below reads what the previous kernel wrote
  if (a.skip && a.skip[rhs]) return;
  __shared__ CgScalars s_cg;
  const HookPre hpre = hook_prefetch(a.hook, rhs, &s_cg);

  const int tid = threadIdx.x;
  const int slot = tid / N;
  const int j = tid - slot * N;
  const bool in_slot = slot < a.ppb;
  float* S2 = sm + (in_slot ? slot : 0) * PER;   // S2[s][k][i]: s = 0 sum, 1 difference
  float* U = S2 + 2 * N * R;                      // U[k][jj][i]

  const MeshDev& m = a.mesh;
  const int N1e = m.ne[0], N2e = m.ne[1], N3e = m.ne[2];
  const int pl0 = N2e * N3e, pl1 = N1e * N3e, pl2 = N1e * N2e;
  const int nelem = N1e * pl0;
  const long long toff = (long long)rhs * a.trace_stride;
  const float* __restrict__ xin = a.x + toff;
  float* __restrict__ yout = a.y + toff;
  const float* __restrict__ dinv_r = DZC ? nullptr : a.dinv + (long long)rhs * a.dinv_rhs_stride;
  const float lam_r = DZC ? static_cast<float>(a.lam[rhs]) : 0.f;
  const float hs = a.tab.h0 + a.tab.h1, hd = a.tab.h0 - a.tab.h1;
  const float cj = a.tab.c[j];
  const bool jeven = j < NE;
  float dot = 0.f;

  const int per_grid = gridDim.x * a.ppb;
  const int trips = (nelem + per_grid - 1) / per_grid;   // same in every thread (barriers)
  for (int t = 0; t < trips; ++t) {
    const int e = (t * gridDim.x + blockIdx.x) * a.ppb + slot;
    const bool live = in_slot && e < nelem;
    int e1 = 0, e2 = 0, e3 = 0;
    if (live) {
      e1 = e % N1e;
      const int rest = e / N1e;
      e2 = rest % N2e;
      e3 = rest / N2e;
    }
    // face bases (first node of the face) or -1 on a Dirichlet plane
    auto fb = [&](int d, int plane, int fab) -> int {
      return (live && plane >= m.lo[d] && plane <= m.hi[d]) ? ((int)m.blk[d] + (plane - m.lo[d]) * (d == 0 ? pl0 : d == 1 ? pl1 : pl2) + fab) * N2 : -1;
    };
    const int b1l = fb(0, e1, e2 + N2e * e3), b1h = fb(0, e1 + 1, e2 + N2e * e3);
    const int b2l = fb(1, e2, e1 + N1e * e3), b2h = fb(1, e2 + 1, e1 + N1e * e3);
    const int b3l = fb(2, e3, e1 + N1e * e2), b3h = fb(2, e3 + 1, e1 + N1e * e2);
    auto ld = [&](int base, int node) -> float { return base >= 0 ? xin[base + node] : 0.f; };

    // x1 column (j, k): sums and differences; x3 row (i, j); own x2 row (i, k = j)
    float S1[N], D1[N], C3s[N], C3d[N];
    static_for<0, N>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      const float lo = ld(b1l, j + N * k), hi = ld(b1h, j + N * k);
      S1[k] = lo + hi;
      D1[k] = lo - hi;
    });
    static_for<0, N>([&](auto ic) {
      constexpr int i = decltype(ic)::value;
      const float lo = ld(b3l, i + N * j), hi = ld(b3h, i + N * j);
      C3s[i] = lo + hi;
      C3d[i] = lo - hi;
    });
    if (live) {
      static_for<0, N>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        const float lo = ld(b2l, i + N * j), hi = ld(b2h, i + N * j);
        S2[R * j + i] = lo + hi;
        S2[N * R + R * j + i] = lo - hi;
      });
    }
    const float4 mt = *reinterpret_cast<const float4*>(a.metric + (m.uniform ? 0 : 4 * (live ? e : 0)));
    const float d0 = mt.x, d1 = mt.y, d2 = mt.z, d3 = mt.w;
    __syncthreads();

    if (live) {
      const float cjd2 = cj * d2;
      const float* Brow = S2 + (jeven ? 0 : N * R);   // (S2 | D2)(., k) rows
      const float* dz = DZC ? nullptr : dinv_r + (m.uniform ? 0 : (long long)e * (N2 * R)) + R * j;
      // D_Z^-1 rows of the next k are in flight while k is computed
      float4 dcur[NQ], dnext[NQ];
      if constexpr (!DZC) {
        static_for<0, NQ>([&](auto qc) {
          constexpr int q = decltype(qc)::value;
          dcur[q] = *reinterpret_cast<const float4*>(dz + 4 * q);
        });
      }
      static_for<0, N>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        constexpr bool keven = k < NE;
        if constexpr (!DZC && k + 1 < N) {
          static_for<0, NQ>([&](auto qc) {
            constexpr int q = decltype(qc)::value;
            dnext[q] = *reinterpret_cast<const float4*>(dz + R * N * (k + 1) + 4 * q);
          });
        }
        const float ckd3 = a.tab.c[k] * d3;
        const float Ap = d1 * S1[k], Am = d1 * D1[k];
        const float dzb = DZC ? fmaf(d3, a.tab.lam[k], fmaf(d2, a.tab.lam[j], lam_r * d0)) : 0.f;
        (void)dzb;
        float Pp = 0.f, Pm = 0.f;
        float* Uk = U + R * (j + N * k);
        static_for<0, NQ>([&](auto qc) {
          constexpr int q = decltype(qc)::value;
          const float4 bv = *reinterpret_cast<const float4*>(Brow + R * k + 4 * q);
          float4 dv = make_float4(0.f, 0.f, 0.f, 0.f);
          if constexpr (!DZC) dv = dcur[q];
          const float b[4] = {bv.x, bv.y, bv.z, bv.w};
          const float ev[4] = {dv.x, dv.y, dv.z, dv.w};
          (void)ev;
          float u[4] = {0.f, 0.f, 0.f, 0.f};
          static_for<0, 4>([&](auto lc) {
            constexpr int l = decltype(lc)::value;
            constexpr int i = 4 * q + l;
            if constexpr (i < N) {
              float F = a.tab.c[i] * (i < NE ? Ap : Am);
              F = fmaf(cjd2, b[l], F);
              F = fmaf(ckd3, keven ? C3s[i] : C3d[i], F);
              float inv;
              if constexpr (DZC) inv = __fdividef(1.0f, fmaf(d1, a.tab.lam[i], dzb));
              else inv = ev[l];
              u[l] = F * inv;
              if constexpr (i < NE) Pp = fmaf(a.tab.c[i], u[l], Pp);
              else Pm = fmaf(a.tab.c[i], u[l], Pm);
            }
          });
          *reinterpret_cast<float4*>(Uk + 4 * q) = make_float4(u[0], u[1], u[2], u[3]);
        });
        if constexpr (!DZC && k + 1 < N) {
          static_for<0, NQ>([&](auto qc) { dcur[decltype(qc)::value] = dnext[decltype(qc)::value]; });
        }
        // x1-face node (j, k)
        const float sum = d1 * (hs * S1[k] - 2.f * Pp), dif = d1 * (hd * D1[k] - 2.f * Pm);
        if (b1l >= 0) red_add(yout + b1l + j + N * k, 0.5f * (sum + dif));
        if (b1h >= 0) red_add(yout + b1h + j + N * k, 0.5f * (sum - dif));
        dot = fmaf(S1[k], sum, fmaf(D1[k], dif, dot));
      });
    }
    __syncthreads();   // U complete

    if (live) {
      // U rows of a contraction: sum_m c_m rows[m * stride] by the parity of m
      auto contract = [&](const float* rows, int stride, float (&Xp)[R], float (&Xm)[R]) {
        static_for<0, R>([&](auto ic) {
          Xp[decltype(ic)::value] = 0.f;
          Xm[decltype(ic)::value] = 0.f;
        });
        static_for<0, N>([&](auto mc) {
          constexpr int mo = decltype(mc)::value;
          const float cm = a.tab.c[mo];
          static_for<0, NQ>([&](auto qc) {
            constexpr int q = decltype(qc)::value;
            const float4 uv = *reinterpret_cast<const float4*>(rows + stride * mo + 4 * q);
            const float uu[4] = {uv.x, uv.y, uv.z, uv.w};
            static_for<0, 4>([&](auto lc) {
              constexpr int l = decltype(lc)::value;
              if constexpr (mo < NE) Xp[4 * q + l] = fmaf(cm, uu[l], Xp[4 * q + l]);
              else Xm[4 * q + l] = fmaf(cm, uu[l], Xm[4 * q + l]);
            });
          });
        });
      };
      float Xp[R], Xm[R];
      // x3-face nodes (i, j): R(i, j) = sum_k c_k U[k][j][i]
      contract(U + R * j, R * N, Xp, Xm);
      static_for<0, N>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        const float sum = d3 * (hs * C3s[i] - 2.f * Xp[i]), dif = d3 * (hd * C3d[i] - 2.f * Xm[i]);
        if (b3l >= 0) red_add(yout + b3l + i + N * j, 0.5f * (sum + dif));
        if (b3h >= 0) red_add(yout + b3h + i + N * j, 0.5f * (sum - dif));
        dot = fmaf(C3s[i], sum, fmaf(C3d[i], dif, dot));
      });
      // x2-face nodes (i, k = j): Q(i, j) = sum_jj c_jj U[j][jj][i]
      contract(U + R * N * j, R, Xp, Xm);
      static_for<0, N>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        const float Sv = S2[R * j + i], Dv = S2[N * R + R * j + i];
        const float sum = d2 * (hs * Sv - 2.f * Xp[i]), dif = d2 * (hd * Dv - 2.f * Xm[i]);
        if (b2l >= 0) red_add(yout + b2l + i + N * j, 0.5f * (sum + dif));
        if (b2h >= 0) red_add(yout + b2h + i + N * j, 0.5f * (sum - dif));
        dot = fmaf(Sv, sum, fmaf(Dv, dif, dot));
      });
    }
    __syncthreads();   // the next element restages S2 and U
  }

  grid_dep_launch();
  if (a.hook.partials != nullptr) hook_finish(a.hook, rhs, dot, hpre, &s_cg);
}

}  // namespace hdg
