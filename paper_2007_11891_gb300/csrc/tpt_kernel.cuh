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
  // inside the CG loop: the scalars of the single-reduction CG (cg_scalars),
  // with the per-block partial sums of gamma left by the previous update step
  CgScalars* cg;
  int* flags;
  const double* step_partials;   // [nrhs][step_blocks]
  int step_blocks;
};

// Scalars of the single-reduction CG (Chronopoulos-Gear) at the end of the
// operator launch of iteration i, once delta_i = u_i^T K u_i is known.
// For i > 0 the previous update step left gamma_i = r_i . u_i as per-block
// partial sums (summed by the caller, so that the update kernel needs no
// reduction of its own): beta_i = gamma_i / gamma_{i-1}, and the convergence
// test gamma_i <= rr_stop or the iteration cap may stop this right-hand side
// here.  Then alpha_i = gamma_i / (delta_i - beta_i gamma_i / alpha_{i-1})
// (delta_0 alone for i = 0).  A non-positive or non-finite denominator is a
// breakdown (status 6).  flags[r] mirrors done.
__device__ __forceinline__ void cg_scalars(CgScalars* cgp, const CgScalars& c0, int* flag, double delta,
                                           double gamma_new) {
  CgScalars c = c0;
  if (c.done) return;
  if (c.ops > 0) {
    c.it = c.ops;
    if (!(gamma_new == gamma_new)) {
      c.status = 6;
      c.done = 1;
    } else {
      c.beta = gamma_new / c.rr;
      c.rr_old = c.rr;
      c.rr = gamma_new;
      if (gamma_new <= c.rr_stop) c.done = 1;
      else if (c.it >= c.max_it) { c.done = 1; c.status = 5; }
    }
  }
  if (!c.done) {
    const double den = c.ops == 0 ? delta : delta - c.beta * c.rr / c.alpha;
    if (!(den > 0.0) || !(den <= 1.79e308) || !(c.rr == c.rr)) {
      c.status = 6;
      c.done = 1;
    } else {
      c.alpha = c.rr / den;
      c.ops += 1;
    }
  }
  *cgp = c;
  *flag = c.done;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Start of an operator launch inside the CG loop: what the last block will
// need from before this launch (the scalar state, and this thread's share of
// the previous update's gamma partials, which are complete by now) is loaded
// while the block still has its elements to compute, so that the reduction
// at the end has one dependent global round trip instead of three.
struct HookPre {
  double g;   // this thread's share of the gamma partials
};
__device__ __forceinline__ HookPre hook_prefetch(const CgHook& hook, int rhs, CgScalars* s_cg) {
  HookPre pre{0.0};
  if (hook.partials == nullptr || hook.cg == nullptr) return pre;
  if (threadIdx.x == 0) *s_cg = hook.cg[rhs];
  if (threadIdx.x < 32) {   // the warp that would finish the reduction
    const double* gp = hook.step_partials + (long long)rhs * hook.step_blocks;
    for (int b = threadIdx.x; b < hook.step_blocks; b += 32) pre.g += __ldcg(gp + b);
  }
  return pre;
}

// End of an operator launch with a hook.  The per-thread x^T y contributions
// (1/2 sum over element faces of (S sum + D dif)) are summed per warp in the
// kernel's own precision T, per block and across blocks in FP64, all in a
// fixed order.  FP64 arithmetic runs at a small fraction of the FP32 rate on
// this part, so the cross-block reduction in the last block is done by one
// warp (about 15 partials per lane) rather than by the whole block.  The last
// block to arrive stores the result (and the CG step scalars when hook.cg is
// set); the summation order is fixed, so the result is deterministic.
template <typename T>
__device__ __forceinline__ void hook_finish(const CgHook& hook, int rhs, T dot, const HookPre& pre,
                                            const CgScalars* s_cg) {
  __shared__ double wsum[32];
  __shared__ bool last;
  const int tid = threadIdx.x;
  const T v = warp_sum(dot);
  if ((tid & 31) == 0) wsum[tid >> 5] = static_cast<double>(v);
  __syncthreads();
  if (tid == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) s += wsum[w];
    hook.partials[(long long)rhs * gridDim.x + blockIdx.x] = 0.5 * s;
    __threadfence();
    const unsigned int done = atomicAdd(hook.counter + rhs, 1u);
    last = (done == gridDim.x - 1);
    // acquire side of the arrival, in the one thread that observed it (the
    // other threads of the block have outstanding reductions of their own to
    // the output, which a fence of theirs would wait for); the reads below
    // go to L2 (__ldcg) after the barrier
    if (last) __threadfence();
  }
  __syncthreads();
  if (last && tid < 32) {
    const double* pp = hook.partials + (long long)rhs * gridDim.x;
    constexpr int K = 16;   // partials per lane per batch
    double s = 0.0;
    for (int b0 = 0; b0 < (int)gridDim.x; b0 += K * 32) {
      double sv[K];
#pragma unroll
      for (int q = 0; q < K; ++q) {
        const int b = b0 + q * 32 + tid;
        sv[q] = b < (int)gridDim.x ? __ldcg(pp + b) : 0.0;
      }
#pragma unroll
      for (int q = 0; q < K; ++q) s += sv[q];
    }
    s = warp_sum(s);
    const double g = warp_sum(pre.g);
    if (tid == 0) {
      if (hook.cg) cg_scalars(hook.cg + rhs, *s_cg, hook.flags + rhs, s, g);
      hook.pq[rhs] = s;
      hook.counter[rhs] = 0u;
    }
  }
}

// Vectors of the fused CG step of the tile kernel (tpt_tile.cuh): the launch
// of iteration i + 1 applies the update of iteration i to each face value it
// stages.  x and p are updated in place by the one owner of each face value;
// r and s are read from one buffer and written to the other (a face value's
// second reader, in another CTA, still reads the old values); w (= K u of
// iteration i, complete) is read from one of three buffers, the operator
// accumulates K u_{i+1} into the second, and the owners zero the third for
// the launch after next.
template <typename T>
struct CgVecs {
  T* x;
  T* p;
  const T* r_in;
  T* r_out;
  const T* s_in;
  T* s_out;
  const T* w_in;
  T* w_zero;
  const T* W;              // preconditioner weights, or null (W = I)
  double* gpartials;       // per-block partial sums of gamma = r . u: [nrhs][gridDim.x]
                           // (persistent kernel: [2][nrhs][gridDim.x])
  unsigned int* bar;       // persistent kernel: [nrhs][2] grid-barrier words, zero at launch
  int* err;                // persistent kernel: set when a grid barrier gave up
};

template <typename T, typename ST>
struct TptArgs {
  MeshDev mesh;
  Tables<T> tab;
  const T* metric;              // (d0, d1, d2, d3) per element, or one entry if uniform
  const T* dinv;                // D_Z^-1: n^3 per element (or one table if uniform);
                                // null: computed in the kernel from lam and Lambda
  long long dinv_rhs_stride;    // per right-hand side
  const double* lam;            // per right-hand side lambda (when dinv is null)
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
  int chunk;                    // FP32 apply kernel: elements per slot (a contiguous run
                                // in element order, possibly spanning x1-pencils)
  int max_grid;                 // CTAs launched (grid-stride over slot groups); 0 = one per group
  const int* skip;              // per rhs: nonzero -> do nothing (converged), or null
  CgHook hook;                  // partials == null: no dot
  int pdl;                      // host: launch with programmatic stream serialization
  int variant;                  // apply kernel: 0 element runs (tpt_fast.cuh / tpt_kernel.cuh),
                                // 1 x2-planes (tpt_plane.cuh), 2 warp slots (tpt_warp.cuh),
                                // 3 element tiles (tpt_tile.cuh), 4 runtime degree (tpt_generic.cuh)
  int sms;                      // host: SMs of the device (tile kernel grid)
  int tile;                     // host: elements per tile of the tile kernel, 0 = automatic
  int cg;                       // tile kernel: 1 = fused CG step (cgv), 0 = plain apply
  CgVecs<T> cgv;
};

// Shared memory per pencil slot (elements of T): two buffers of the four
// staged face arrays (S2+, S2-, S3+, S3-; N rows of R padded entries) and
// the element's eigenspace solution U (N^2 rows of R).
template <typename T, int N>
__host__ __device__ constexpr int tpt_smem_per_pencil() {
  return 2 * 4 * N * dz_row(N, sizeof(T)) + N * N * dz_row(N, sizeof(T));
}

// FP32 apply kernel (tpt_fast.cuh): slot layout, CTA size limit and
// guaranteed resident CTAs per SM.  Where rounding a slot up to whole warps
// wastes few lanes (n = 8, 9 and n >= 11), every slot owns whole warps and
// synchronises on its own named barrier, so a slow warp holds back only its
// slot; otherwise (n <= 7, n = 10) slots are packed n^2 threads apart and
// share the CTA barrier.  Up to 256 threads (288 for n = 9: three slots of
// three warps) and three CTAs per SM (at most 80, for n = 9 72, registers)
// for n <= 16, which measured 16% faster than two CTAs with more
// registers; n = 17 needs 289 threads per slot.
__host__ __device__ constexpr bool fast_aligned(int n) { return n >= 8 && n != 10; }
__host__ __device__ constexpr int fast_slot_threads(int n) { return fast_aligned(n) ? (n * n + 31) / 32 * 32 : n * n; }
__host__ __device__ constexpr int fast_threads(int n, int ppb) { return (ppb * fast_slot_threads(n) + 31) / 32 * 32; }
__host__ __device__ constexpr int fast_max_threads(int n) { return n * n > 256 ? 320 : (n == 9 ? 288 : 256); }
__host__ __device__ constexpr int fast_min_ctas(int n) { return n * n > 256 ? 2 : 3; }


// At most 320 threads per CTA (n = 17: 289 threads rounded to warps).  FP32
// instantiations keep three resident CTAs per SM (64 registers); FP64 ones
// are bound by the FP64 pipe and get two (up to 96 registers) for ILP.
template <typename T, typename ST, int N, int MODE>
__global__ void __launch_bounds__(320, sizeof(T) == 4 ? 3 : 2) tpt_kernel(const TptArgs<T, ST> a) {
  constexpr int N2 = N * N, NE = (N + 1) / 2;
  constexpr int R = dz_row(N, sizeof(T));          // padded row
  constexpr int VL = Vec<T>::L, NQ = R / VL;
  constexpr int SF = N * R;                          // one staged face array
  constexpr int PER = tpt_smem_per_pencil<T, N>();
  using V = typename Vec<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);

  const int rhs = blockIdx.y;
  if (a.skip && a.skip[rhs]) return;   // uniform per block: no barrier is skipped partially
  __shared__ CgScalars s_cg;
  const HookPre hpre = (MODE == TPT_APPLY) ? hook_prefetch(a.hook, rhs, &s_cg) : HookPre{0.0};

  const int tid = threadIdx.x;
  const int slot = tid / N2;
  const int line = tid - slot * N2;
  const int lo_i = line % N, hi_i = line / N;     // face node (a, b); x1-line (j, k)
  const int qpad = lo_i + R * hi_i;                // padded index of the face node
  T dot = T(0);
  const long long ngroups = (a.npencils * a.nseg + a.ppb - 1) / a.ppb;
  // persistent grid: each CTA takes slot groups blockIdx.x, + gridDim.x, ...
  for (long long grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
  const long long slot_id = grp * a.ppb + slot;
  const long long pencil = slot_id / a.nseg;
  const int sg = (int)(slot_id - pencil * a.nseg);
  const bool act = slot < a.ppb && pencil < a.npencils;
  const MeshDev& m = a.mesh;
  const int N1e = m.ne[0], N2e = m.ne[1], N3e = m.ne[2];
  const int e2 = act ? (int)(pencil % N2e) : 0;
  const int e3 = act ? (int)(pencil / N2e) : 0;
  const int e1s = act ? sg * a.seg : 0;
  const int e1e = act ? min(e1s + a.seg, N1e) : 0;

  T* base = sm + (act ? slot : 0) * PER;
  T* U = base + 8 * SF;

  const long long toff = (long long)rhs * a.trace_stride;
  const ST* xin = (MODE == TPT_RHS) ? nullptr : a.x + toff;
  ST* yout = (MODE == TPT_RECOVER) ? nullptr : a.y + toff;
  const T* gin = (MODE == TPT_APPLY || a.gbd == nullptr) ? nullptr : a.gbd + (long long)rhs * a.bdry_stride;
  const T* dinv_r = a.dinv ? a.dinv + (long long)rhs * a.dinv_rhs_stride : nullptr;
  const T lam_r = a.dinv ? T(0) : static_cast<T>(a.lam[rhs]);

  // Face offsets are 32-bit (trace and boundary sizes per right-hand side
  // are below 2^31, checked on the host).  An unknown face node has the same
  // offset in the input x and the output y.
  const int pl0 = N2e * N3e, pl1 = N1e * N3e, pl2 = N1e * N2e;
  const int f0 = e2 + N2e * e3;        // x1 faces: (e2, e3)
  const int f1 = N1e * e3 + e1s;       // x2 faces: (e1, e3) at the segment start
  const int f2 = N1e * e2 + e1s;       // x3 faces: (e1, e2) at the segment start
  auto unknown = [&](int d, int plane) -> bool { return plane >= m.lo[d] && plane <= m.hi[d]; };
  // unknown-face offset of direction d on `plane`, or -1
  auto uoff = [&](int d, int plane, int fab, int pl) -> int {
    return (act && unknown(d, plane)) ? (int)((m.blk[d] + (long long)(plane - m.lo[d]) * pl + fab) * N2 + line) : -1;
  };
  // Dirichlet-face offset (boundary layout) of direction d on `plane`, or -1
  auto goff = [&](int d, int plane, int fab) -> int {
    if (MODE == TPT_APPLY || gin == nullptr || !act || unknown(d, plane)) return -1;
    return (int)((m.side[2 * d + (plane == 0 ? 0 : 1)] + fab) * N2 + line);
  };
  int o2l = uoff(1, e2, f1, pl1), o2h = uoff(1, e2 + 1, f1, pl1);
  int o3l = uoff(2, e3, f2, pl2), o3h = uoff(2, e3 + 1, f2, pl2);
  int g2l = goff(1, e2, f1), g2h = goff(1, e2 + 1, f1), g3l = goff(2, e3, f2), g3h = goff(2, e3 + 1, f2);
  auto rd = [&](int o, int g) -> T {
    if (MODE != TPT_RHS && o >= 0) return load_as<ST, T>(xin + o);
    if (MODE != TPT_APPLY && g >= 0) return gin[g];
    return T(0);
  };
  auto x1_at = [&](int plane) -> T { return rd(uoff(0, plane, f0, pl0), goff(0, plane, f0)); };
  auto y1_at = [&](int plane) -> ST* {
    return yout + (m.blk[0] + (long long)(plane - m.lo[0]) * pl0 + f0) * N2 + line;
  };

  // values of the first element; the loop prefetches element t+1 while it
  // computes element t
  T xlo1 = act ? x1_at(e1s) : T(0);
  T xhi1 = (act && e1s < e1e) ? x1_at(e1s + 1) : T(0);
  T x2l = rd(o2l, g2l), x2h = rd(o2h, g2h), x3l = rd(o3l, g3l), x3h = rd(o3h, g3h);

  T carry = T(0);

  // same trip count in every slot of the CTA (the loop holds barriers)
  for (int t = 0; t < a.seg; ++t) {
    const int e1 = e1s + t;
    const bool live = act && e1 < e1e;
    const long long elem = live ? e1 + (long long)N1e * (e2 + (long long)N2e * e3) : 0;
    T* S = base + (t & 1) * 4 * SF;   // S2+, S2-, S3+, S3- of this element
    if (live) {
      S[qpad] = x2l + x2h;
      S[SF + qpad] = x2l - x2h;
      S[2 * SF + qpad] = x3l + x3h;
      S[3 * SF + qpad] = x3l - x3h;
    }
    const T S1 = xlo1 + xhi1, D1 = xlo1 - xhi1;
    // prefetch element t+1 (in flight during this element's arithmetic)
    T nx1 = T(0), n2l = T(0), n2h = T(0), n3l = T(0), n3h = T(0);
    if (live && e1 + 1 < e1e) {
      auto adv = [](int o) { return o >= 0 ? o + N2 : o; };
      nx1 = x1_at(e1 + 2);
      n2l = rd(adv(o2l), adv(g2l)); n2h = rd(adv(o2h), adv(g2h));
      n3l = rd(adv(o3l), adv(g3l)); n3h = rd(adv(o3h), adv(g3h));
    }
    const T* mt = a.metric + (m.uniform ? 0 : 4 * elem);
    const T d1 = mt[1], d2 = mt[2], d3 = mt[3];
    __syncthreads();

    // expansion along the x1-line (j, k) = (lo_i, hi_i) and x1 contraction
    T Pp = T(0), Pm = T(0);
    if (live) {
      const int j = lo_i, k = hi_i;
      const T Ap = d1 * S1, Am = d1 * D1;
      const T cjd2 = a.tab.c[j] * d2, ckd3 = a.tab.c[k] * d3;
      const T* Bs = S + (j < NE ? 0 : SF) + R * k;
      const T* Cs = S + (k < NE ? 2 * SF : 3 * SF) + R * j;
      const T* dz = dinv_r ? dinv_r + (m.uniform ? 0 : elem * (long long)N2 * R) + R * (j + N * k) : nullptr;
      const T dzb = dz ? T(0) : fma(d3, a.tab.lam[k], fma(d2, a.tab.lam[j], lam_r * mt[0]));
      const T* sr = (MODE == TPT_APPLY) ? nullptr
                                         : a.src + (long long)rhs * a.vol_stride + elem * (long long)(N2 * N) + N * j + N2 * k;
      T* Ur = U + R * (j + N * k);
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const V bv = *reinterpret_cast<const V*>(Bs + q * VL);
        const V cv = *reinterpret_cast<const V*>(Cs + q * VL);
        V dv;
        if (dz) dv = *reinterpret_cast<const V*>(dz + q * VL);
        V uv;
#pragma unroll
        for (int l = 0; l < VL; ++l) {
          const int i = q * VL + l;
          if (i < N) {
            T F = a.tab.c[i] * (i < NE ? Ap : Am);
            F = fma(cjd2, vget(bv, l), F);
            F = fma(ckd3, vget(cv, l), F);
            if (MODE != TPT_APPLY) F -= sr[i];
            const T u = F * (dz ? vget(dv, l) : dz_recip(fma(d1, a.tab.lam[i], dzb)));
            vset(uv, l, u);
            if (i < NE) Pp = fma(a.tab.c[i], u, Pp);
            else Pm = fma(a.tab.c[i], u, Pm);
          } else {
            vset(uv, l, T(0));
          }
        }
        *reinterpret_cast<V*>(Ur + q * VL) = uv;
      }
    }
    __syncthreads();

    if (live) {
      const int i = lo_i, mm = hi_i;
      if (MODE == TPT_RECOVER) {
        // w = (f-hat - F_E) / D_Z = -u ; thread (i, mm) writes points (i, mm, k)
        T* w = a.vout + (long long)rhs * a.vol_stride + elem * (long long)(N2 * N);
#pragma unroll
        for (int k = 0; k < N; ++k) w[i + N * mm + N2 * k] = -U[i + R * (mm + N * k)];
      } else {
        T Qp = T(0), Qm = T(0), Rp = T(0), Rm = T(0);
#pragma unroll
        for (int mo = 0; mo < N; ++mo) {
          const T uq = U[i + R * (mo + N * mm)];   // (i, j = mo, k = mm)
          const T ur = U[i + R * (mm + N * mo)];   // (i, j = mm, k = mo)
          if (mo < NE) { Qp = fma(a.tab.c[mo], uq, Qp); Rp = fma(a.tab.c[mo], ur, Rp); }
          else         { Qm = fma(a.tab.c[mo], uq, Qm); Rm = fma(a.tab.c[mo], ur, Rm); }
        }
        const T hs = a.tab.h0 + a.tab.h1, hd = a.tab.h0 - a.tab.h1;
        const T sgn = (MODE == TPT_RHS) ? T(-1) : T(1);
        const T two = T(2), half = T(0.5);
        // x2 faces (node (i, k = mm)) on planes e2, e2 + 1
        {
          const T Sv = S[qpad], Dv = S[SF + qpad];
          const T sum = d2 * (hs * Sv - two * Qp), dif = d2 * (hd * Dv - two * Qm);
          if (o2l >= 0) red_add(yout + o2l, sgn * half * (sum + dif));
          if (o2h >= 0) red_add(yout + o2h, sgn * half * (sum - dif));
          if (MODE == TPT_APPLY) dot = fma(Sv, sum, fma(Dv, dif, dot));
        }
        // x3 faces (node (i, j = mm)) on planes e3, e3 + 1
        {
          const T Sv = S[2 * SF + qpad], Dv = S[3 * SF + qpad];
          const T sum = d3 * (hs * Sv - two * Rp), dif = d3 * (hd * Dv - two * Rm);
          if (o3l >= 0) red_add(yout + o3l, sgn * half * (sum + dif));
          if (o3h >= 0) red_add(yout + o3h, sgn * half * (sum - dif));
          if (MODE == TPT_APPLY) dot = fma(Sv, sum, fma(Dv, dif, dot));
        }
        // x1 faces (node (j, k) = line): running sum over the segment
        {
          const T sum = d1 * (hs * S1 - two * Pp), dif = d1 * (hd * D1 - two * Pm);
          const T rlo = sgn * half * (sum + dif), rhi = sgn * half * (sum - dif);
          if (MODE == TPT_APPLY) dot = fma(S1, sum, fma(D1, dif, dot));
          // plane e1: inside the segment -> complete sum, store; segment start
          // -> shared with the previous segment (add), unless physical boundary
          if (unknown(0, e1)) {
            ST* dst = y1_at(e1);
            if (t > 0) store_from<ST, T>(dst, carry + rlo);
            else if (e1 == 0) store_from<ST, T>(dst, rlo);
            else red_add(dst, rlo);
          }
          carry = rhi;
          if (e1 == e1e - 1 && unknown(0, e1e)) {
            ST* dst = y1_at(e1e);
            if (e1e == N1e) store_from<ST, T>(dst, carry);
            else red_add(dst, carry);
          }
        }
      }
    }
    // advance the x2/x3 streams by one face (one element along x1)
    if (o2l >= 0) o2l += N2;
    if (o2h >= 0) o2h += N2;
    if (o3l >= 0) o3l += N2;
    if (o3h >= 0) o3h += N2;
    if (g2l >= 0) g2l += N2;
    if (g2h >= 0) g2h += N2;
    if (g3l >= 0) g3l += N2;
    if (g3h >= 0) g3h += N2;
    xlo1 = xhi1;
    xhi1 = nx1;
    x2l = n2l; x2h = n2h; x3l = n3l; x3h = n3h;
  }
  __syncthreads();   // the next group restages the face buffers
  }  // slot groups

  if (MODE == TPT_APPLY && a.hook.partials != nullptr) hook_finish(a.hook, rhs, dot, hpre, &s_cg);
}

}  // namespace hdg
