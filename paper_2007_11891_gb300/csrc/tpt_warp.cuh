// FP32 operator application y = K-hat x (Alg. (hdg_op_3d_transformed)) with
// one warp per element slot.
//
// The per-element arithmetic is that of tpt_fast.cuh (parity-split
// expansion and contraction, D_Z^-1 from the table or computed, the
// x1-face between consecutive elements of a run summed in registers,
// exactly two additions onto a zeroed output elsewhere), and so is the work
// split into contiguous element runs.  What differs: a slot is one warp,
// and lane t owns the x1-lines (and face nodes) line = t + 32 q for
// q < L = ceil(n^2 / 32).  The exchange of an element's staged faces and of
// its eigenspace solution then stays inside the warp (__syncwarp instead of
// a block barrier), and the per-element index work is shared by L lines.
// FP32 storage only.
#pragma once

#include "internal.h"
#include "tpt_kernel.cuh"

namespace hdg {

template <int N>
__host__ __device__ constexpr int warp_lines() {
  return (N * N + 31) / 32;
}

template <int N, bool DZC>
__global__ void __launch_bounds__(kWarpSlotsPerCta * 32) tpt_warp_kernel(const TptArgs<float, float> a) {
  constexpr int N2 = N * N, NE = (N + 1) / 2;
  constexpr int L = warp_lines<N>();
  constexpr int R = dz_row(N, sizeof(float));
  constexpr int NQ = R / 4;
  constexpr int SF = N * R;
  constexpr int PER = tpt_smem_per_pencil<float, N>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sm = reinterpret_cast<float*>(smem_raw);

  const int rhs = blockIdx.y;
  grid_dep_wait();   // everything below reads what the previous kernel wrote
  if (a.skip && a.skip[rhs]) return;
  __shared__ CgScalars s_cg;
  const HookPre hpre = hook_prefetch(a.hook, rhs, &s_cg);

  const int lane = threadIdx.x & 31;
  const int slot = threadIdx.x >> 5;
  const bool in_slot = slot < a.ppb;
  float* base = sm + (in_slot ? slot : 0) * PER;
  float* U = base + 8 * SF;
  int lo_i[L], hi_i[L], qpad[L];
  bool lv[L];
#pragma unroll
  for (int q = 0; q < L; ++q) {
    const int line = lane + 32 * q;
    lv[q] = line < N2;
    lo_i[q] = line % N;
    hi_i[q] = line / N;
    qpad[q] = lo_i[q] + R * hi_i[q];
  }

  const MeshDev& m = a.mesh;
  const int N1e = m.ne[0], N2e = m.ne[1], N3e = m.ne[2];
  const int pl0 = N2e * N3e, pl1 = N1e * N3e, pl2 = N1e * N2e;
  const int lo0 = m.lo[0], hi0 = m.hi[0], lo1 = m.lo[1], hi1 = m.hi[1], lo2 = m.lo[2], hi2 = m.hi[2];
  const int blk0 = (int)m.blk[0], blk1 = (int)m.blk[1], blk2 = (int)m.blk[2];
  const long long toff = (long long)rhs * a.trace_stride;
  const float* __restrict__ xin = a.x + toff;
  float* __restrict__ yout = a.y + toff;
  const float* __restrict__ dinv_r = DZC ? nullptr : a.dinv + (long long)rhs * a.dinv_rhs_stride;
  const float lam_r = DZC ? static_cast<float>(a.lam[rhs]) : 0.f;
  const float hs = a.tab.h0 + a.tab.h1, hd = a.tab.h0 - a.tab.h1;

  const int nelem = N1e * pl0;
  const int chunk = a.chunk;
  const long long first = (long long)(blockIdx.x * a.ppb + slot) * chunk;
  int e = (in_slot && first < nelem) ? (int)first : nelem;
  const int eend = min(e + chunk, nelem);
  int c1 = 0, c2 = 0, c3 = 0;
  if (e < nelem) {
    c1 = e % N1e;
    const int rest = e / N1e;
    c2 = rest % N2e;
    c3 = rest / N2e;
  }
  // face offsets of line q = the lane's (line = lane) + 32 q; -1 on a Dirichlet plane
  struct Off {
    int x1l, x1h, x2l, x2h, x3l, x3h;
  };
  auto offsets = [&](int e1, int e2, int e3) -> Off {
    Off o;
    const int b1 = (blk0 + (e1 - lo0) * pl0 + e2 + N2e * e3) * N2 + lane;
    o.x1l = (e1 >= lo0 && e1 <= hi0) ? b1 : -1;
    o.x1h = (e1 + 1 >= lo0 && e1 + 1 <= hi0) ? b1 + pl0 * N2 : -1;
    const int b2 = (blk1 + (e2 - lo1) * pl1 + e1 + N1e * e3) * N2 + lane;
    o.x2l = (e2 >= lo1 && e2 <= hi1) ? b2 : -1;
    o.x2h = (e2 + 1 >= lo1 && e2 + 1 <= hi1) ? b2 + pl1 * N2 : -1;
    const int b3 = (blk2 + (e3 - lo2) * pl2 + e1 + N1e * e2) * N2 + lane;
    o.x3l = (e3 >= lo2 && e3 <= hi2) ? b3 : -1;
    o.x3h = (e3 + 1 >= lo2 && e3 + 1 <= hi2) ? b3 + pl2 * N2 : -1;
    return o;
  };
  auto ld = [&](int off, int q) -> float { return (off >= 0 && lv[q]) ? xin[off + 32 * q] : 0.f; };

  Off o = offsets(c1, c2, c3);
  float xlo1[L], xhi1[L], x2l[L], x2h[L], x3l[L], x3h[L], carry[L];
#pragma unroll
  for (int q = 0; q < L; ++q) {
    const bool g = e < eend;
    xlo1[q] = g ? ld(o.x1l, q) : 0.f;
    xhi1[q] = g ? ld(o.x1h, q) : 0.f;
    x2l[q] = g ? ld(o.x2l, q) : 0.f;
    x2h[q] = g ? ld(o.x2h, q) : 0.f;
    x3l[q] = g ? ld(o.x3l, q) : 0.f;
    x3h[q] = g ? ld(o.x3h, q) : 0.f;
    carry[q] = 0.f;
  }
  bool have_carry = false;
  float dot = 0.f;

  for (int t = 0; t < chunk; ++t) {
    const bool live = e < eend;
    float* S = base + (t & 1) * 4 * SF;
    float S1[L], D1[L];
#pragma unroll
    for (int q = 0; q < L; ++q) {
      if (live && lv[q]) {
        S[qpad[q]] = x2l[q] + x2h[q];
        S[SF + qpad[q]] = x2l[q] - x2h[q];
        S[2 * SF + qpad[q]] = x3l[q] + x3h[q];
        S[3 * SF + qpad[q]] = x3l[q] - x3h[q];
      }
      S1[q] = xlo1[q] + xhi1[q];
      D1[q] = xlo1[q] - xhi1[q];
    }
    int n1 = c1 + 1, n2 = c2, n3 = c3;
    const bool wrap = n1 == N1e;
    if (wrap) {
      n1 = 0;
      if (++n2 == N2e) { n2 = 0; ++n3; }
    }
    const bool nlive = live && e + 1 < eend;
    const bool same = nlive && !wrap;
    Off no;
    if (!wrap) {
      no.x1l = o.x1h;
      no.x1h = (n1 + 1 <= hi0) ? o.x1h + pl0 * N2 : -1;
      no.x2l = o.x2l >= 0 ? o.x2l + N2 : -1;
      no.x2h = o.x2h >= 0 ? o.x2h + N2 : -1;
      no.x3l = o.x3l >= 0 ? o.x3l + N2 : -1;
      no.x3h = o.x3h >= 0 ? o.x3h + N2 : -1;
    } else {
      no = offsets(n1, n2, n3);
    }
    if constexpr (!DZC)
      if (nlive && !m.uniform) {
#pragma unroll
        for (int q = 0; q < L; ++q)
          if (lv[q]) prefetch_l1(dinv_r + (long long)(e + 1) * (N2 * R) + R * (lane + 32 * q));
      }
    float nlo1[L], nhi1[L], n2l[L], n2h[L], n3l[L], n3h[L];
#pragma unroll
    for (int q = 0; q < L; ++q) {
      nlo1[q] = nlive ? (same ? xhi1[q] : ld(no.x1l, q)) : 0.f;
      nhi1[q] = nlive ? ld(no.x1h, q) : 0.f;
      n2l[q] = nlive ? ld(no.x2l, q) : 0.f;
      n2h[q] = nlive ? ld(no.x2h, q) : 0.f;
      n3l[q] = nlive ? ld(no.x3l, q) : 0.f;
      n3h[q] = nlive ? ld(no.x3h, q) : 0.f;
    }
    const float4 mt = *reinterpret_cast<const float4*>(a.metric + (m.uniform ? 0 : 4 * (live ? e : 0)));
    const float d0 = mt.x, d1 = mt.y, d2 = mt.z, d3 = mt.w;
    __syncwarp();

    // expansion along x1-line (j, k) = (lo_i[q], hi_i[q]) and x1 contraction
    float Pp[L], Pm[L];
#pragma unroll
    for (int q = 0; q < L; ++q) {
      Pp[q] = 0.f;
      Pm[q] = 0.f;
      if (live && lv[q]) {
        const int j = lo_i[q], k = hi_i[q];
        const float Ap = d1 * S1[q], Am = d1 * D1[q];
        const float cjd2 = a.tab.c[j] * d2, ckd3 = a.tab.c[k] * d3;
        const float* Bs = S + (j < NE ? 0 : SF) + R * k;
        const float* Cs = S + (k < NE ? 2 * SF : 3 * SF) + R * j;
        const float* dz = DZC ? nullptr : dinv_r + (m.uniform ? 0 : e * (N2 * R)) + R * (j + N * k);
        const float dzb = DZC ? fmaf(d3, a.tab.lam[k], fmaf(d2, a.tab.lam[j], lam_r * d0)) : 0.f;
        float* Ur = U + R * (j + N * k);
        float pp = 0.f, pm = 0.f;
        static_for<0, NQ>([&](auto qc) {
          constexpr int qq = decltype(qc)::value;
          const float4 bv = *reinterpret_cast<const float4*>(Bs + 4 * qq);
          const float4 cv = *reinterpret_cast<const float4*>(Cs + 4 * qq);
          float4 dv = make_float4(0.f, 0.f, 0.f, 0.f);
          if constexpr (!DZC) dv = *reinterpret_cast<const float4*>(dz + 4 * qq);
          const float b[4] = {bv.x, bv.y, bv.z, bv.w};
          const float c[4] = {cv.x, cv.y, cv.z, cv.w};
          const float ev[4] = {dv.x, dv.y, dv.z, dv.w};
          (void)ev;
          float u[4] = {0.f, 0.f, 0.f, 0.f};
          static_for<0, 4>([&](auto lc) {
            constexpr int l = decltype(lc)::value;
            constexpr int i = 4 * qq + l;
            if constexpr (i < N) {
              float F = a.tab.c[i] * (i < NE ? Ap : Am);
              F = fmaf(cjd2, b[l], F);
              F = fmaf(ckd3, c[l], F);
              float inv;
              if constexpr (DZC) inv = __fdividef(1.0f, fmaf(d1, a.tab.lam[i], dzb));
              else inv = ev[l];
              u[l] = F * inv;
              if constexpr (i < NE) pp = fmaf(a.tab.c[i], u[l], pp);
              else pm = fmaf(a.tab.c[i], u[l], pm);
            }
          });
          *reinterpret_cast<float4*>(Ur + 4 * qq) = make_float4(u[0], u[1], u[2], u[3]);
        });
        Pp[q] = pp;
        Pm[q] = pm;
      }
    }
    __syncwarp();

#pragma unroll
    for (int q = 0; q < L; ++q) {
      if (live && lv[q]) {
        const int i = lo_i[q], mm = hi_i[q];
        float Qp = 0.f, Qm = 0.f, Rp = 0.f, Rm = 0.f;
        const float* Uq = U + i + R * N * mm;   // (i, j = mo, k = mm): stride R
        const float* Ur2 = U + i + R * mm;       // (i, j = mm, k = mo): stride R N
        static_for<0, N>([&](auto mc) {
          constexpr int mo = decltype(mc)::value;
          const float uq = Uq[R * mo];
          const float ur = Ur2[R * N * mo];
          if constexpr (mo < NE) { Qp = fmaf(a.tab.c[mo], uq, Qp); Rp = fmaf(a.tab.c[mo], ur, Rp); }
          else                   { Qm = fmaf(a.tab.c[mo], uq, Qm); Rm = fmaf(a.tab.c[mo], ur, Rm); }
        });
        const int sh = 32 * q;
        {  // x2 faces, node (i, k = mm)
          const float Sv = S[qpad[q]], Dv = S[SF + qpad[q]];
          const float sum = d2 * (hs * Sv - 2.f * Qp), dif = d2 * (hd * Dv - 2.f * Qm);
          if (o.x2l >= 0) red_add(yout + o.x2l + sh, 0.5f * (sum + dif));
          if (o.x2h >= 0) red_add(yout + o.x2h + sh, 0.5f * (sum - dif));
          dot = fmaf(Sv, sum, fmaf(Dv, dif, dot));
        }
        {  // x3 faces, node (i, j = mm)
          const float Sv = S[2 * SF + qpad[q]], Dv = S[3 * SF + qpad[q]];
          const float sum = d3 * (hs * Sv - 2.f * Rp), dif = d3 * (hd * Dv - 2.f * Rm);
          if (o.x3l >= 0) red_add(yout + o.x3l + sh, 0.5f * (sum + dif));
          if (o.x3h >= 0) red_add(yout + o.x3h + sh, 0.5f * (sum - dif));
          dot = fmaf(Sv, sum, fmaf(Dv, dif, dot));
        }
        {  // x1 faces, node (j, k) = line
          const float sum = d1 * (hs * S1[q] - 2.f * Pp[q]), dif = d1 * (hd * D1[q] - 2.f * Pm[q]);
          const float rlo = 0.5f * (sum + dif), rhi = 0.5f * (sum - dif);
          dot = fmaf(S1[q], sum, fmaf(D1[q], dif, dot));
          if (o.x1l >= 0) {
            if (have_carry) yout[o.x1l + sh] = carry[q] + rlo;
            else if (c1 == 0) yout[o.x1l + sh] = rlo;
            else red_add(yout + o.x1l + sh, rlo);
          }
          if (o.x1h >= 0 && !same) {
            if (c1 + 1 == N1e) yout[o.x1h + sh] = rhi;
            else red_add(yout + o.x1h + sh, rhi);
          }
          carry[q] = rhi;
        }
      }
    }
    have_carry = same;
    o = no;
    c1 = n1; c2 = n2; c3 = n3;
    ++e;
#pragma unroll
    for (int q = 0; q < L; ++q) {
      xlo1[q] = nlo1[q]; xhi1[q] = nhi1[q];
      x2l[q] = n2l[q]; x2h[q] = n2h[q]; x3l[q] = n3l[q]; x3h[q] = n3h[q];
    }
  }

  grid_dep_launch();
  if (a.hook.partials != nullptr) hook_finish(a.hook, rhs, dot, hpre, &s_cg);
}

}  // namespace hdg
