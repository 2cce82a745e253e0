// FP32 operator application y = K-hat x (Alg. (hdg_op_3d_transformed)), the
// inner-loop kernel of the mixed-precision solve.
//
// Same algorithm, data layout and face ownership as tpt_kernel (see
// tpt_kernel.cuh): parity-split expansion/contraction, one CTA slot per
// x1-pencil segment with one thread per x1-line, x1-faces inside a segment
// summed in registers, all other shared faces combined with exactly two
// red.global.add onto zero.  This version is specialised for the hot
// path: FP32 storage and arithmetic, homogeneous Dirichlet data, the D_Z^-1
// source fixed at compile time (DZC: computed in the kernel; else a table),
// 32-bit index arithmetic with one integer division per slot group, and no
// per-element branches beyond the face-ownership predicates.
//
// FUSEP: the CG search-direction update is fused into the input loads: each
// face value is p_new = W r + beta p_old (p_old = x), the operator acts on
// p_new, and the owner slot of each face -- the element above it, or below
// it on the top boundary plane -- writes p_new to pout (p_old and pout are
// different buffers, swapped by the caller every iteration).
#pragma once

#include "tpt_kernel.cuh"

namespace hdg {

#ifndef HDG_FAST_MIN_CTAS
#define HDG_FAST_MIN_CTAS 2
#endif
#ifndef HDG_FUSED_MIN_CTAS
#define HDG_FUSED_MIN_CTAS 3
#endif

// Resident CTAs guaranteed per SM.  Plain apply: two (up to 96 registers);
// a cap of 64 made the compiler rematerialise values (29% more
// instructions, measured).  Fused search-direction update: three, whose
// three input streams per face need the extra warps to cover their latency
// (two CTAs: 34% slower inside the CG loop, measured).
template <int N, bool DZC, bool FUSEP>
__global__ void __launch_bounds__(320, FUSEP ? HDG_FUSED_MIN_CTAS : HDG_FAST_MIN_CTAS)
    tpt_fast_kernel(const TptArgs<float, float> a) {
  constexpr int N2 = N * N, NE = (N + 1) / 2;
  constexpr int R = dz_row(N, sizeof(float));
  constexpr int NQ = R / 4;
  constexpr int SF = N * R;
  constexpr int PER = tpt_smem_per_pencil<float, N>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sm = reinterpret_cast<float*>(smem_raw);

  const int rhs = blockIdx.y;
  if (a.skip && a.skip[rhs]) return;   // uniform per block

  const int tid = threadIdx.x;
  const int slot = tid / N2;
  const int line = tid - slot * N2;
  const int lo_i = line % N, hi_i = line / N;
  const int qpad = lo_i + R * hi_i;
  const bool in_slot = slot < a.ppb;
  float* base = sm + (in_slot ? slot : 0) * PER;
  float* U = base + 8 * SF;

  const MeshDev& m = a.mesh;
  const int N1e = m.ne[0], N2e = m.ne[1], N3e = m.ne[2];
  const int pl0 = N2e * N3e, pl1 = N1e * N3e, pl2 = N1e * N2e;
  const int lo0 = m.lo[0], hi0 = m.hi[0], lo1 = m.lo[1], hi1 = m.hi[1], lo2 = m.lo[2], hi2 = m.hi[2];
  const int blk0 = (int)m.blk[0], blk1 = (int)m.blk[1], blk2 = (int)m.blk[2];
  const int seg = a.seg, nseg = a.nseg;
  const long long toff = (long long)rhs * a.trace_stride;
  const float* __restrict__ xin = a.x + toff;
  float* __restrict__ yout = a.y + toff;
  const float* __restrict__ dinv_r = DZC ? nullptr : a.dinv + (long long)rhs * a.dinv_rhs_stride;
  const float lam_r = DZC ? static_cast<float>(a.lam[rhs]) : 0.f;
  const float hs = a.tab.h0 + a.tab.h1, hd = a.tab.h0 - a.tab.h1;
  const float* __restrict__ rin = FUSEP ? a.pr + toff : nullptr;
  const float* __restrict__ win = (FUSEP && a.pw) ? a.pw + toff : nullptr;
  float* __restrict__ pout = FUSEP ? a.pout + toff : nullptr;
  const float beta = FUSEP ? static_cast<float>(a.cg[rhs].beta) : 0.f;
  // operator input at offset o: x, or the updated search direction
  auto ld = [&](int o) -> float {
    if constexpr (FUSEP) {
      const float z = win ? win[o] * rin[o] : rin[o];
      return fmaf(beta, xin[o], z);
    } else {
      return xin[o];
    }
  };
  const int nslots = (int)(a.npencils * nseg);
  const int ngroups = (nslots + a.ppb - 1) / a.ppb;
  float dot = 0.f;

  for (int grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
    const int slot_id = grp * a.ppb + slot;
    const bool act = in_slot && slot_id < nslots;
    const int pencil = act ? slot_id / nseg : 0;
    const int sg = slot_id - pencil * nseg;
    const int e2 = pencil % N2e, e3 = pencil / N2e;
    const int e1s = act ? sg * seg : 0;
    const int e1e = act ? min(e1s + seg, N1e) : 0;
    const int f0 = e2 + N2e * e3;
    // unknown-face offsets (-1: Dirichlet plane, contributes nothing)
    int o2l = (act && e2 >= lo1 && e2 <= hi1) ? (blk1 + (e2 - lo1) * pl1 + N1e * e3 + e1s) * N2 + line : -1;
    int o2h = (act && e2 + 1 >= lo1 && e2 + 1 <= hi1) ? (blk1 + (e2 + 1 - lo1) * pl1 + N1e * e3 + e1s) * N2 + line : -1;
    int o3l = (act && e3 >= lo2 && e3 <= hi2) ? (blk2 + (e3 - lo2) * pl2 + N1e * e2 + e1s) * N2 + line : -1;
    int o3h = (act && e3 + 1 >= lo2 && e3 + 1 <= hi2) ? (blk2 + (e3 + 1 - lo2) * pl2 + N1e * e2 + e1s) * N2 + line : -1;
    // x1 face of plane p: b1 + p * p1 (valid for lo0 <= p <= hi0)
    const int p1 = pl0 * N2;
    const int b1 = (blk0 - lo0 * pl0 + f0) * N2 + line;
    auto x1 = [&](int p) -> float { return (act && p >= lo0 && p <= hi0) ? ld(b1 + p * p1) : 0.f; };

    float xlo1 = x1(e1s);
    float xhi1 = (e1s < e1e) ? x1(e1s + 1) : 0.f;
    float x2l = o2l >= 0 ? ld(o2l) : 0.f, x2h = o2h >= 0 ? ld(o2h) : 0.f;
    float x3l = o3l >= 0 ? ld(o3l) : 0.f, x3h = o3h >= 0 ? ld(o3h) : 0.f;
    // owner of the hi faces in x2/x3: only on the top boundary plane
    const bool own2h = (e2 + 1 == N2e), own3h = (e3 + 1 == N3e);
    float carry = 0.f;
    const int elem0 = e1s + N1e * f0;

    for (int t = 0; t < seg; ++t) {
      const int e1 = e1s + t;
      const bool live = act && e1 < e1e;
      float* S = base + (t & 1) * 4 * SF;
      if (live) {
        S[qpad] = x2l + x2h;
        S[SF + qpad] = x2l - x2h;
        S[2 * SF + qpad] = x3l + x3h;
        S[3 * SF + qpad] = x3l - x3h;
        if constexpr (FUSEP) {
          // this element owns its lo faces, and hi faces on the top boundary
          if (o2l >= 0) pout[o2l] = x2l;
          if (o2h >= 0 && own2h) pout[o2h] = x2h;
          if (o3l >= 0) pout[o3l] = x3l;
          if (o3h >= 0 && own3h) pout[o3h] = x3h;
          if (e1 >= lo0 && e1 <= hi0) pout[b1 + e1 * p1] = xlo1;
          if (e1 + 1 == N1e && e1 + 1 <= hi0) pout[b1 + (e1 + 1) * p1] = xhi1;
        }
      }
      const float S1 = xlo1 + xhi1, D1 = xlo1 - xhi1;
      // prefetch the next element's faces
      float nx1 = 0.f, n2l = 0.f, n2h = 0.f, n3l = 0.f, n3h = 0.f;
      if (live && e1 + 1 < e1e) {
        nx1 = x1(e1 + 2);
        if (o2l >= 0) n2l = ld(o2l + N2);
        if (o2h >= 0) n2h = ld(o2h + N2);
        if (o3l >= 0) n3l = ld(o3l + N2);
        if (o3h >= 0) n3h = ld(o3h + N2);
      }
      const int elem = elem0 + t;
      const float* mt = a.metric + (m.uniform ? 0 : 4 * elem);
      const float d0 = mt[0], d1 = mt[1], d2 = mt[2], d3 = mt[3];
      __syncthreads();

      float Pp = 0.f, Pm = 0.f;
      if (live) {
        const int j = lo_i, k = hi_i;
        const float Ap = d1 * S1, Am = d1 * D1;
        const float cjd2 = a.tab.c[j] * d2, ckd3 = a.tab.c[k] * d3;
        const float* Bs = S + (j < NE ? 0 : SF) + R * k;
        const float* Cs = S + (k < NE ? 2 * SF : 3 * SF) + R * j;
        const float* dz = DZC ? nullptr : dinv_r + (m.uniform ? 0 : elem * (N2 * R)) + R * (j + N * k);
        const float dzb = DZC ? fmaf(d3, a.tab.lam[k], fmaf(d2, a.tab.lam[j], lam_r * d0)) : 0.f;
        float* Ur = U + R * (j + N * k);
        static_for<0, NQ>([&](auto qc) {
          constexpr int q = decltype(qc)::value;
          const float4 bv = *reinterpret_cast<const float4*>(Bs + 4 * q);
          const float4 cv = *reinterpret_cast<const float4*>(Cs + 4 * q);
          float4 dv = make_float4(0.f, 0.f, 0.f, 0.f);
          if constexpr (!DZC) dv = *reinterpret_cast<const float4*>(dz + 4 * q);
          const float b[4] = {bv.x, bv.y, bv.z, bv.w};
          const float c[4] = {cv.x, cv.y, cv.z, cv.w};
          const float e[4] = {dv.x, dv.y, dv.z, dv.w};
          (void)e;
          float u[4] = {0.f, 0.f, 0.f, 0.f};
          static_for<0, 4>([&](auto lc) {
            constexpr int l = decltype(lc)::value;
            constexpr int i = 4 * q + l;
            if constexpr (i < N) {
              float F = a.tab.c[i] * (i < NE ? Ap : Am);
              F = fmaf(cjd2, b[l], F);
              F = fmaf(ckd3, c[l], F);
              float inv;
              if constexpr (DZC) inv = __fdividef(1.0f, fmaf(d1, a.tab.lam[i], dzb));
              else inv = e[l];
              u[l] = F * inv;
              if constexpr (i < NE) Pp = fmaf(a.tab.c[i], u[l], Pp);
              else Pm = fmaf(a.tab.c[i], u[l], Pm);
            }
          });
          *reinterpret_cast<float4*>(Ur + 4 * q) = make_float4(u[0], u[1], u[2], u[3]);
        });
      }
      __syncthreads();

      if (live) {
        const int i = lo_i, mm = hi_i;
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
        {  // x2 faces, node (i, k = mm)
          const float Sv = S[qpad], Dv = S[SF + qpad];
          const float sum = d2 * (hs * Sv - 2.f * Qp), dif = d2 * (hd * Dv - 2.f * Qm);
          if (o2l >= 0) red_add(yout + o2l, 0.5f * (sum + dif));
          if (o2h >= 0) red_add(yout + o2h, 0.5f * (sum - dif));
          dot = fmaf(Sv, sum, fmaf(Dv, dif, dot));
        }
        {  // x3 faces, node (i, j = mm)
          const float Sv = S[2 * SF + qpad], Dv = S[3 * SF + qpad];
          const float sum = d3 * (hs * Sv - 2.f * Rp), dif = d3 * (hd * Dv - 2.f * Rm);
          if (o3l >= 0) red_add(yout + o3l, 0.5f * (sum + dif));
          if (o3h >= 0) red_add(yout + o3h, 0.5f * (sum - dif));
          dot = fmaf(Sv, sum, fmaf(Dv, dif, dot));
        }
        {  // x1 faces, node (j, k) = line
          const float sum = d1 * (hs * S1 - 2.f * Pp), dif = d1 * (hd * D1 - 2.f * Pm);
          const float rlo = 0.5f * (sum + dif), rhi = 0.5f * (sum - dif);
          dot = fmaf(S1, sum, fmaf(D1, dif, dot));
          if (e1 >= lo0 && e1 <= hi0) {
            float* dst = yout + b1 + e1 * p1;
            if (t > 0) *dst = carry + rlo;
            else if (e1 == 0) *dst = rlo;
            else red_add(dst, rlo);
          }
          carry = rhi;
          if (e1 == e1e - 1 && e1e >= lo0 && e1e <= hi0) {
            float* dst = yout + b1 + e1e * p1;
            if (e1e == N1e) *dst = carry;
            else red_add(dst, carry);
          }
        }
      }
      if (o2l >= 0) o2l += N2;
      if (o2h >= 0) o2h += N2;
      if (o3l >= 0) o3l += N2;
      if (o3h >= 0) o3h += N2;
      xlo1 = xhi1;
      xhi1 = nx1;
      x2l = n2l; x2h = n2h; x3l = n3l; x3h = n3h;
    }
    __syncthreads();   // the next group restages the face buffers
  }

  if (a.hook.partials != nullptr) {
    // x^T y = 1/2 sum over element faces of (S sum + D dif); last block sums
    __shared__ double wsum[16];
    __shared__ bool last;
    const float v = warp_sum(dot);
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
      __threadfence();
      const volatile double* pp = a.hook.partials + (long long)rhs * gridDim.x;
      double s = 0.0;
      for (unsigned int b = tid; b < gridDim.x; b += blockDim.x) s += pp[b];
      s = warp_sum(s);
      __syncthreads();
      if ((tid & 31) == 0) wsum[tid >> 5] = s;
      __syncthreads();
      if (tid == 0) {
        double tt = 0.0;
        for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) tt += wsum[w];
        a.hook.pq[rhs] = tt;
        a.hook.counter[rhs] = 0u;
      }
    }
  }
}

}  // namespace hdg
