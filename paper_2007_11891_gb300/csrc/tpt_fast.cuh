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

#include "cg_fused.cuh"

namespace hdg {


// Unknown-face offsets of one element's six faces (-1 on a Dirichlet plane).
struct FaceOffsets {
  int x1l, x1h, x2l, x2h, x3l, x3h;
};

// Fused CG step (CGM = 1, FP32 storage only): the launch of iteration
// i + 1 stages, for every face value it reads, r, w = K u, s = K p and W of
// iteration i (and p, x at the face's owner: the element below it, or its
// only element) with asynchronous copies into this thread's part of shared
// memory while the previous element computes; it then forms
//   s' = w + beta s,  r' = r - alpha s',  u' = W r'
// and applies the operator to u'.  The owner also stores p' = W r + beta p,
// x' = x + alpha p', s', r', a zero into the w buffer of the launch after
// next, and adds r' . u' to gamma (CgVecs; alpha, beta from the previous
// launch's last block).  Each face value is updated by exactly the same
// arithmetic wherever it is read, so both readers see the same u'.
template <int N, bool DZC, typename ST = float, int CGM = 0>
__global__ void __launch_bounds__(fast_max_threads(N), fast_min_ctas(N))
    tpt_fast_kernel(const TptArgs<float, ST> a) {
  constexpr bool CG = CGM != 0;
  static_assert(!CG || std::is_same<ST, float>::value, "the fused CG step runs on FP32 storage");
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
  // Under programmatic dependent launch this grid may start while the
  // previous kernel (the CG update) still runs.  The set-up below (indices,
  // the first element's face offsets) reads nothing that kernel writes; the
  // skip flags come from the operator launch before it, which completed
  // before that kernel could let this one start.  Everything the previous
  // kernel writes is read after grid_dep_wait().
  if (a.skip && a.skip[rhs]) return;   // uniform per block
  __shared__ CgScalars s_cg;
  float al = 0.f, be = 0.f, gam = 0.f;

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

  // fused CG step: this thread's staging area (face k, value v at
  // (6 k + v) SLOT_T + line: r, w, s, W, and p, x at owned faces)
  float* stg = sm + a.ppb * PER + (in_slot ? slot : 0) * (36 * SLOT_T) + line;
  const float* __restrict__ vr = CG ? a.cgv.r_in + toff : nullptr;
  const float* __restrict__ vw = CG ? a.cgv.w_in + toff : nullptr;
  const float* __restrict__ vs = CG ? a.cgv.s_in + toff : nullptr;
  const float* __restrict__ vW = (CG && a.cgv.W) ? a.cgv.W + toff : nullptr;
  float* __restrict__ vp = CG ? a.cgv.p + toff : nullptr;
  float* __restrict__ vx = CG ? a.cgv.x + toff : nullptr;
  // asynchronous loads of the state at the faces of element (f1, f2, f3);
  // x1 lo is skipped when it was the previous element's x1 hi
  auto fetch = [&](const FaceOffsets& fo, int f1, int f2, int f3, bool skip_lo1) {
    const int off[6] = {fo.x1l, fo.x1h, fo.x2l, fo.x2h, fo.x3l, fo.x3h};
    const bool own[6] = {f1 == 0, true, f2 == 0, true, f3 == 0, true};
    static_for<0, 6>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      if (k == 0 && skip_lo1) return;
      const bool on = off[k] >= 0;
      const int oo = on ? off[k] : 0;
      cp_async4(stg + (6 * k + 0) * SLOT_T, vr + oo, on);
      cp_async4(stg + (6 * k + 1) * SLOT_T, vw + oo, on);
      cp_async4(stg + (6 * k + 2) * SLOT_T, vs + oo, on);
      if (vW) cp_async4(stg + (6 * k + 3) * SLOT_T, vW + oo, on);
      if (own[k]) {
        cp_async4(stg + (6 * k + 4) * SLOT_T, vp + oo, on);
        cp_async4(stg + (6 * k + 5) * SLOT_T, vx + oo, on);
      }
    });
    cp_async_commit();
  };
  // the update of the previous iteration at those faces: u' into v[k]
  auto consume = [&](const FaceOffsets& fo, int f1, int f2, int f3, bool skip_lo1, float* v) {
    cp_async_wait_all();
    const int off[6] = {fo.x1l, fo.x1h, fo.x2l, fo.x2h, fo.x3l, fo.x3h};
    const bool own[6] = {f1 == 0, true, f2 == 0, true, f3 == 0, true};
    float* __restrict__ vro = a.cgv.r_out + toff;
    float* __restrict__ vso = a.cgv.s_out + toff;
    float* __restrict__ vwz = a.cgv.w_zero + toff;
    static_for<0, 6>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      if (k == 0 && skip_lo1) return;
      v[k] = 0.f;
      if (off[k] < 0) return;
      const float r = stg[(6 * k + 0) * SLOT_T], w = stg[(6 * k + 1) * SLOT_T], sv = stg[(6 * k + 2) * SLOT_T];
      const float Wv = vW ? stg[(6 * k + 3) * SLOT_T] : 1.f;
      const float sn = fmaf(be, sv, w);
      const float rn = fmaf(-al, sn, r);
      const float un = Wv * rn;
      v[k] = un;
      if (own[k]) {
        const int oo = off[k];
        const float pn = fmaf(be, stg[(6 * k + 4) * SLOT_T], Wv * r);
        vx[oo] = fmaf(al, pn, stg[(6 * k + 5) * SLOT_T]);
        vp[oo] = pn;
        vso[oo] = sn;
        vro[oo] = rn;
        vwz[oo] = 0.f;
        gam = fmaf(un, rn, gam);
      }
    });
  };

  FaceOffsets o = offsets(c1, c2, c3);
  float xlo1 = 0.f, xhi1 = 0.f, x2l = 0.f, x2h = 0.f, x3l = 0.f, x3h = 0.f;
  bool carried = false;   // fused step: x1 lo is the previous element's x1 hi

  grid_dep_wait();   // from here on: data the previous kernel in the stream wrote
  const HookPre hpre = hook_prefetch(a.hook, rhs, &s_cg);
  if constexpr (CG) {
    __syncthreads();   // s_cg (hook_prefetch) visible to every thread
    al = static_cast<float>(s_cg.alpha);
    be = static_cast<float>(s_cg.beta);
  }
  if (e < eend) {
    if constexpr (CG) {
      fetch(o, c1, c2, c3, false);
    } else {
      xlo1 = ld(o.x1l); xhi1 = ld(o.x1h);
      x2l = ld(o.x2l); x2h = ld(o.x2h); x3l = ld(o.x3l); x3h = ld(o.x3h);
    }
  }
  float carry = 0.f;
  bool have_carry = false;
  float dot = 0.f;

  // same trip count in every slot (the loop holds barriers)
  for (int t = 0; t < chunk; ++t) {
    const bool live = e < eend;
    float* S = base + (t & 1) * 4 * SF;
    if constexpr (CG) {
      if (live) {
        float v[6];
        consume(o, c1, c2, c3, carried, v);
        if (!carried) xlo1 = v[0];
        xhi1 = v[1]; x2l = v[2]; x2h = v[3]; x3l = v[4]; x3h = v[5];
      }
    }
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
      if constexpr (CG) {
        fetch(no, n1, n2, n3, same);
      } else {
        nlo1 = same ? xhi1 : ld(no.x1l);
        nhi1 = ld(no.x1h);
        n2l = ld(no.x2l); n2h = ld(no.x2h); n3l = ld(no.x3l); n3h = ld(no.x3h);
      }
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
      // pairs of points (i, i + 1) in packed two-lane FP32 arithmetic (one
      // FMUL2/FFMA2 per pair); the x1 contraction keeps one two-lane
      // accumulator per parity combination of a pair
      float2 pEE = make_float2(0.f, 0.f), pOO = pEE, pEO = pEE;
      const float2 cjd2v = make_float2(cjd2, cjd2), ckd3v = make_float2(ckd3, ckd3);
      static_for<0, NQ>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        const float4 bv = *reinterpret_cast<const float4*>(Bs + 4 * q);
        const float4 cv = *reinterpret_cast<const float4*>(Cs + 4 * q);
        float4 dv = make_float4(0.f, 0.f, 0.f, 0.f);
        if constexpr (!DZC) dv = *reinterpret_cast<const float4*>(dz + 4 * q);
        (void)dv;
        float2 uh[2];
        static_for<0, 2>([&](auto hc) {
          constexpr int hh = decltype(hc)::value;
          constexpr int i0 = 4 * q + 2 * hh, i1 = i0 + 1;
          if constexpr (i0 < N) {
            constexpr bool e0 = i0 < NE, e1 = i1 < NE, v1 = i1 < N;
            const float c0 = a.tab.c[i0], c1v = v1 ? a.tab.c[i1] : 0.f;
            // the second lane of the last pair of an odd row lies in the row
            // padding, which no thread writes: it takes zeros
            const float b0 = hh == 0 ? bv.x : bv.z, b1 = v1 ? (hh == 0 ? bv.y : bv.w) : 0.f;
            const float k0 = hh == 0 ? cv.x : cv.z, k1 = v1 ? (hh == 0 ? cv.y : cv.w) : 0.f;
            float2 F = __fmul2_rn(make_float2(c0, c1v), make_float2(e0 ? Ap : Am, e1 ? Ap : Am));
            F = __ffma2_rn(cjd2v, make_float2(b0, b1), F);
            F = __ffma2_rn(ckd3v, make_float2(k0, k1), F);
            float2 inv;
            if constexpr (DZC) {
              const float2 den = __ffma2_rn(make_float2(d1, d1),
                                            make_float2(a.tab.lam[i0], v1 ? a.tab.lam[i1] : 0.f),
                                            make_float2(dzb, dzb));
              inv = make_float2(dz_recip(den.x), v1 ? dz_recip(den.y) : 0.f);
            } else {
              inv = make_float2(hh == 0 ? dv.x : dv.z, v1 ? (hh == 0 ? dv.y : dv.w) : 0.f);
            }
            const float2 u = __fmul2_rn(F, inv);
            uh[hh] = u;
            const float2 cc = make_float2(c0, c1v);
            if constexpr (e0 && e1) pEE = __ffma2_rn(cc, u, pEE);
            else if constexpr (!e0 && !e1) pOO = __ffma2_rn(cc, u, pOO);
            else pEO = __ffma2_rn(cc, u, pEO);
          } else {
            uh[hh] = make_float2(0.f, 0.f);
          }
        });
        *reinterpret_cast<float4*>(Ur + 4 * q) = make_float4(uh[0].x, uh[0].y, uh[1].x, uh[1].y);
      });
      Pp = (pEE.x + pEE.y) + pEO.x;
      Pm = (pOO.x + pOO.y) + pEO.y;
    }
    slot_sync();

    if (live) {
      const int i = lo_i, mm = hi_i;
      const float* Uq = U + i + R * N * mm;   // (i, j = mo, k = mm): stride R
      const float* Ur2 = U + i + R * mm;       // (i, j = mm, k = mo): stride R N
      // the x2 and x3 contractions as one two-lane accumulator per parity
      float2 QRp = make_float2(0.f, 0.f), QRm = QRp;
      static_for<0, N>([&](auto mc) {
        constexpr int mo = decltype(mc)::value;
        const float2 uu = make_float2(Uq[R * mo], Ur2[R * N * mo]);
        const float2 cm = make_float2(a.tab.c[mo], a.tab.c[mo]);
        if constexpr (mo < NE) QRp = __ffma2_rn(cm, uu, QRp);
        else QRm = __ffma2_rn(cm, uu, QRm);
      });
      {  // x2 faces, node (i, k = mm)
        const float Sv = S[qpad], Dv = S[SF + qpad];
        const float sum = d2 * (hs * Sv - 2.f * QRp.x), dif = d2 * (hd * Dv - 2.f * QRm.x);
        red_add_if(o.x2l >= 0, yout + max(o.x2l, 0), 0.5f * (sum + dif));
        red_add_if(o.x2h >= 0, yout + max(o.x2h, 0), 0.5f * (sum - dif));
        dot = fmaf(Sv, sum, fmaf(Dv, dif, dot));
      }
      {  // x3 faces, node (i, j = mm)
        const float Sv = S[2 * SF + qpad], Dv = S[3 * SF + qpad];
        const float sum = d3 * (hs * Sv - 2.f * QRp.y), dif = d3 * (hd * Dv - 2.f * QRm.y);
        red_add_if(o.x3l >= 0, yout + max(o.x3l, 0), 0.5f * (sum + dif));
        red_add_if(o.x3h >= 0, yout + max(o.x3h, 0), 0.5f * (sum - dif));
        dot = fmaf(Sv, sum, fmaf(Dv, dif, dot));
      }
      {  // x1 faces, node (j, k) = line
        const float sum = d1 * (hs * S1 - 2.f * Pp), dif = d1 * (hd * D1 - 2.f * Pm);
        const float rlo = 0.5f * (sum + dif), rhi = 0.5f * (sum - dif);
        dot = fmaf(S1, sum, fmaf(D1, dif, dot));
        // lo plane: the previous element of the run left its share in
        // `carry`; plane 0 has no other contributor (stored); else another
        // run adds
        {
          const bool on = o.x1l >= 0, st = on && (have_carry || c1 == 0);
          ST* dst = yout + max(o.x1l, 0);
          st_if(st, dst, have_carry ? carry + rlo : rlo);
          red_add_if(on && !st, dst, rlo);
        }
        // hi plane: kept for the next element of the run; the top plane has
        // no other contributor (stored); else another run adds
        {
          const bool on = o.x1h >= 0 && !(kCarry && same), st = on && c1 + 1 == N1e;
          ST* dst = yout + max(o.x1h, 0);
          st_if(st, dst, rhi);
          red_add_if(on && !st, dst, rhi);
        }
        carry = rhi;
        have_carry = kCarry && same;
      }
    }
    o = no;
    c1 = n1; c2 = n2; c3 = n3;
    ++e;
    if constexpr (CG) {
      carried = same;
      if (same) xlo1 = xhi1;
    } else {
      xlo1 = nlo1; xhi1 = nhi1;
      x2l = n2l; x2h = n2h; x3l = n3l; x3h = n3h;
    }
  }

  grid_dep_launch();   // the next kernel's blocks may take this block's place
  if constexpr (CG) hook_finish_cg(a.hook, a.cgv.gpartials, rhs, dot, gam, &s_cg);
  else if (a.hook.partials != nullptr) hook_finish(a.hook, rhs, dot, hpre, &s_cg);
}

}  // namespace hdg
