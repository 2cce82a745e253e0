// FP32 operator application y = K-hat x (Alg. (hdg_op_3d_transformed)), the
// inner-loop kernel of the mixed-precision solve.
//
// Same per-element algorithm as tpt_kernel (see tpt_kernel.cuh): parity-split
// expansion/contraction with n^2 threads per element (one per x1-line), and
// shared faces combined with exactly two additions onto a zeroed output.
// The work split differs: each CTA slot owns a contiguous run of `chunk`
// elements in the element order (x1 fastest), which may continue from one
// x1-pencil into the next.  Every slot of the grid gets the same number of
// elements (no wave quantisation over pencils), the faces of the next
// element are always in flight while the current one is computed, and the
// face offsets advance incrementally (recomputed only when the run enters a
// new pencil).  The x1-face between two consecutive elements of one run is
// summed in registers and stored once; every other shared face receives
// red.global.add contributions (two adds onto zero commute exactly, so the
// result does not depend on how the elements are split into runs).
//
// Specialised for the hot path: FP32 arithmetic, homogeneous Dirichlet data,
// D_Z^-1 source fixed at compile time (DZC: computed in the kernel; else a
// table), 32-bit offsets (trace size < 2^31 per right-hand side, checked on
// the host).  Trace storage ST: float, or bfloat16 (inputs widened to FP32;
// every output contribution rounded to BF16 and added with a BF16 atomic, so
// that, here too, each face value is the same two-term sum whatever the runs).
#pragma once

#include "tpt_kernel.cuh"

namespace hdg {


// Unknown-face offsets of one element's six faces (-1 on a Dirichlet plane).
struct FaceOffsets {
  int x1l, x1h, x2l, x2h, x3l, x3h;
};

template <int N, bool DZC, typename ST = float>
__global__ void __launch_bounds__(fast_max_threads(N), fast_min_ctas(N))
    tpt_fast_kernel(const TptArgs<float, ST> a) {
  // FP32 storage sums the x1-face between consecutive elements of a run in
  // registers; BF16 storage adds both contributions atomically (a register
  // sum would round once where the atomics round twice)
  constexpr bool kCarry = std::is_same<ST, float>::value;
  constexpr int N2 = N * N, NE = (N + 1) / 2;
  constexpr int R = dz_row(N, sizeof(float));
  constexpr int NQ = R / 4;
  constexpr int SF = N * R;
  constexpr int PER = tpt_smem_per_pencil<float, N>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sm = reinterpret_cast<float*>(smem_raw);

  const int rhs = blockIdx.y;
  // everything below reads what the previous kernel in the stream wrote
  grid_dep_wait();
  if (a.skip && a.skip[rhs]) return;   // uniform per block
  __shared__ CgScalars s_cg;
  const HookPre hpre = hook_prefetch(a.hook, rhs, &s_cg);

  constexpr bool AL = fast_aligned(N);
  constexpr int SLOT_T = fast_slot_threads(N);
  const int tid = threadIdx.x;
  const int slot = tid / SLOT_T;
  const int line = tid - slot * SLOT_T;   // >= N2 on the padding lanes of a whole-warp slot
  const int lo_i = line % N, hi_i = line / N;
  const int qpad = lo_i + R * hi_i;
  const bool in_slot = slot < a.ppb && line < N2;
  // barrier of this slot's threads (whole warps: a named barrier), else the CTA's
  auto slot_sync = [&]() {
    if constexpr (AL) asm volatile("bar.sync %0, %1;" ::"r"(1 + slot), "r"(SLOT_T) : "memory");
    else __syncthreads();
  };
  float* base = sm + (in_slot ? slot : 0) * PER;
  float* U = base + 8 * SF;

  const MeshDev& m = a.mesh;
  const int N1e = m.ne[0], N2e = m.ne[1], N3e = m.ne[2];
  const int pl0 = N2e * N3e, pl1 = N1e * N3e, pl2 = N1e * N2e;
  const int lo0 = m.lo[0], hi0 = m.hi[0], lo1 = m.lo[1], hi1 = m.hi[1], lo2 = m.lo[2], hi2 = m.hi[2];
  const int blk0 = (int)m.blk[0], blk1 = (int)m.blk[1], blk2 = (int)m.blk[2];
  const long long toff = (long long)rhs * a.trace_stride;
  const ST* __restrict__ xin = a.x + toff;
  ST* __restrict__ yout = a.y + toff;
  const float* __restrict__ dinv_r = DZC ? nullptr : a.dinv + (long long)rhs * a.dinv_rhs_stride;
  const float lam_r = DZC ? static_cast<float>(a.lam[rhs]) : 0.f;
  const float hs = a.tab.h0 + a.tab.h1, hd = a.tab.h0 - a.tab.h1;

  // this slot's run of elements [e, eend)
  const int nelem = N1e * pl0;
  const int chunk = a.chunk;
  const long long first = (long long)(blockIdx.x * a.ppb + slot) * chunk;
  int e = (in_slot && first < nelem) ? (int)first : nelem;
  const int eend = min(e + chunk, nelem);
  int c1 = 0, c2 = 0, c3 = 0;   // coordinates of element e
  if (e < nelem) {
    c1 = e % N1e;
    const int rest = e / N1e;
    c2 = rest % N2e;
    c3 = rest / N2e;
  }

  auto offsets = [&](int e1, int e2, int e3) -> FaceOffsets {
    FaceOffsets o;
    const int b1 = (blk0 + (e1 - lo0) * pl0 + e2 + N2e * e3) * N2 + line;
    o.x1l = (e1 >= lo0 && e1 <= hi0) ? b1 : -1;
    o.x1h = (e1 + 1 >= lo0 && e1 + 1 <= hi0) ? b1 + pl0 * N2 : -1;
    const int b2 = (blk1 + (e2 - lo1) * pl1 + e1 + N1e * e3) * N2 + line;
    o.x2l = (e2 >= lo1 && e2 <= hi1) ? b2 : -1;
    o.x2h = (e2 + 1 >= lo1 && e2 + 1 <= hi1) ? b2 + pl1 * N2 : -1;
    const int b3 = (blk2 + (e3 - lo2) * pl2 + e1 + N1e * e2) * N2 + line;
    o.x3l = (e3 >= lo2 && e3 <= hi2) ? b3 : -1;
    o.x3h = (e3 + 1 >= lo2 && e3 + 1 <= hi2) ? b3 + pl2 * N2 : -1;
    return o;
  };
  auto ld = [&](int off) -> float { return off >= 0 ? load_as<ST, float>(xin + off) : 0.f; };

  FaceOffsets o = offsets(c1, c2, c3);
  float xlo1 = 0.f, xhi1 = 0.f, x2l = 0.f, x2h = 0.f, x3l = 0.f, x3h = 0.f;
  if (e < eend) {
    xlo1 = ld(o.x1l); xhi1 = ld(o.x1h);
    x2l = ld(o.x2l); x2h = ld(o.x2h); x3l = ld(o.x3l); x3h = ld(o.x3h);
  }
  float carry = 0.f;
  bool have_carry = false;
  float dot = 0.f;

  // same trip count in every slot (the loop holds barriers)
  for (int t = 0; t < chunk; ++t) {
    const bool live = e < eend;
    float* S = base + (t & 1) * 4 * SF;
    if (live) {
      S[qpad] = x2l + x2h;
      S[SF + qpad] = x2l - x2h;
      S[2 * SF + qpad] = x3l + x3h;
      S[3 * SF + qpad] = x3l - x3h;
    }
    const float S1 = xlo1 + xhi1, D1 = xlo1 - xhi1;
    // the next element of the run and its faces (in flight during this one)
    int n1 = c1 + 1, n2 = c2, n3 = c3;
    const bool wrap = n1 == N1e;
    if (wrap) {
      n1 = 0;
      if (++n2 == N2e) { n2 = 0; ++n3; }
    }
    const bool nlive = live && e + 1 < eend;
    const bool same = nlive && !wrap;   // the next element continues this x1-pencil
    FaceOffsets no;
    if (!wrap) {
      // planes n1 and n1 + 1 >= 1 >= lo0; plane n1 + 1 <= hi0 implies plane n1 is unknown
      no.x1l = o.x1h;
      no.x1h = (n1 + 1 <= hi0) ? o.x1h + pl0 * N2 : -1;
      no.x2l = o.x2l >= 0 ? o.x2l + N2 : -1;
      no.x2h = o.x2h >= 0 ? o.x2h + N2 : -1;
      no.x3l = o.x3l >= 0 ? o.x3l + N2 : -1;
      no.x3h = o.x3h >= 0 ? o.x3h + N2 : -1;
    } else {
      no = offsets(n1, n2, n3);
    }
    float nlo1 = 0.f, nhi1 = 0.f, n2l = 0.f, n2h = 0.f, n3l = 0.f, n3h = 0.f;
    // the next element's D_Z^-1 row (a table in L2) moves to L1 meanwhile
    if constexpr (!DZC)
      if (nlive && !m.uniform) prefetch_l1(dinv_r + (long long)(e + 1) * (N2 * R) + R * line);
    if (nlive) {
      nlo1 = same ? xhi1 : ld(no.x1l);
      nhi1 = ld(no.x1h);
      n2l = ld(no.x2l); n2h = ld(no.x2h); n3l = ld(no.x3l); n3h = ld(no.x3h);
    }
    const float4 mt = *reinterpret_cast<const float4*>(a.metric + (m.uniform ? 0 : 4 * (live ? e : 0)));
    const float d0 = mt.x, d1 = mt.y, d2 = mt.z, d3 = mt.w;
    slot_sync();

    float Pp = 0.f, Pm = 0.f;
    if (live) {
      const int j = lo_i, k = hi_i;
      const float Ap = d1 * S1, Am = d1 * D1;
      const float cjd2 = a.tab.c[j] * d2, ckd3 = a.tab.c[k] * d3;
      const float* Bs = S + (j < NE ? 0 : SF) + R * k;
      const float* Cs = S + (k < NE ? 2 * SF : 3 * SF) + R * j;
      const float* dz = DZC ? nullptr : dinv_r + (m.uniform ? 0 : e * (N2 * R)) + R * (j + N * k);
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
        const float ev[4] = {dv.x, dv.y, dv.z, dv.w};
        (void)ev;
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
            else inv = ev[l];
            u[l] = F * inv;
            if constexpr (i < NE) Pp = fmaf(a.tab.c[i], u[l], Pp);
            else Pm = fmaf(a.tab.c[i], u[l], Pm);
          }
        });
        *reinterpret_cast<float4*>(Ur + 4 * q) = make_float4(u[0], u[1], u[2], u[3]);
      });
    }
    slot_sync();

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
        if (o.x2l >= 0) red_add(yout + o.x2l, 0.5f * (sum + dif));
        if (o.x2h >= 0) red_add(yout + o.x2h, 0.5f * (sum - dif));
        dot = fmaf(Sv, sum, fmaf(Dv, dif, dot));
      }
      {  // x3 faces, node (i, j = mm)
        const float Sv = S[2 * SF + qpad], Dv = S[3 * SF + qpad];
        const float sum = d3 * (hs * Sv - 2.f * Rp), dif = d3 * (hd * Dv - 2.f * Rm);
        if (o.x3l >= 0) red_add(yout + o.x3l, 0.5f * (sum + dif));
        if (o.x3h >= 0) red_add(yout + o.x3h, 0.5f * (sum - dif));
        dot = fmaf(Sv, sum, fmaf(Dv, dif, dot));
      }
      {  // x1 faces, node (j, k) = line
        const float sum = d1 * (hs * S1 - 2.f * Pp), dif = d1 * (hd * D1 - 2.f * Pm);
        const float rlo = 0.5f * (sum + dif), rhi = 0.5f * (sum - dif);
        dot = fmaf(S1, sum, fmaf(D1, dif, dot));
        // lo plane: the previous element of the run left its share in
        // `carry`; plane 0 has no other contributor; else another run adds
        if (o.x1l >= 0) {
          if (have_carry) store_from<ST, float>(yout + o.x1l, carry + rlo);
          else if (c1 == 0) store_from<ST, float>(yout + o.x1l, rlo);
          else red_add(yout + o.x1l, rlo);
        }
        // hi plane: kept for the next element of the run; the top plane has
        // no other contributor; else another run adds
        if (o.x1h >= 0 && !(kCarry && same)) {
          if (c1 + 1 == N1e) store_from<ST, float>(yout + o.x1h, rhi);
          else red_add(yout + o.x1h, rhi);
        }
        carry = rhi;
        have_carry = kCarry && same;
      }
    }
    o = no;
    c1 = n1; c2 = n2; c3 = n3;
    ++e;
    xlo1 = nlo1; xhi1 = nhi1;
    x2l = n2l; x2h = n2h; x3l = n3l; x3h = n3h;
  }

  grid_dep_launch();   // the next kernel's blocks may take this block's place
  if (a.hook.partials != nullptr) hook_finish(a.hook, rhs, dot, hpre, &s_cg);
}

}  // namespace hdg
