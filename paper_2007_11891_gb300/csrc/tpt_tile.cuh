// Operator application y = K-hat x in the transformed face basis
// (arXiv:2007.11891, Alg. (hdg_op_3d_transformed)) with tiles of elements:
// the inner-loop kernel of the solve, in FP32 (also with BF16 trace storage)
// and FP64.
//
// Per element (notation of tpt_kernel.cuh): with face sums S = x_lo + x_hi and
// differences D = x_lo - x_hi per direction,
//   u(i,j,k) = [c_i d1 (S1|D1)(j,k) + c_j d2 (S2|D2)(i,k) + c_k d3 (S3|D3)(i,j)]
//              / (lambda d0 + d1 Lambda_i + d2 Lambda_j + d3 Lambda_k)
// ((S|D) by the parity of the mode index in front), and for each direction
//   r_lo + r_hi = d (hs S - 2 Q+),  r_lo - r_hi = d (hd D - 2 Q-)
// with Q+/- the even/odd-mode contractions sum_m c_m u along that direction.
//
// Work split.  A CTA of n^2 G threads takes tiles of E = G x rounds
// consecutive elements in element order (x1 fastest; a tile may continue from
// one x1-pencil into the next), so every CTA of the grid gets the same amount
// of work whatever the pencil length.  Thread (g, q) owns one face node /
// x1-line q = (a, b) of the elements g, g + G, ... of every tile, so its index
// arithmetic (and, on a uniform grid, its row of the D_Z^-1 table, held in
// registers) is computed once per launch, not per element.  Per tile:
//   0. face offsets of the tile's elements (computed for the next tile during
//      the current one's staging, into a second buffer);
//   1. staging: the x2/x3 faces of the tile are read with coalesced loads
//      (the E faces of one plane are contiguous in the trace layout; all of a
//      thread's loads are issued before any is used) and written as
//      sums/differences into padded shared-memory rows; the x1 faces are
//      staged as they are;
//   2. pass 1, per element the x1-line (j, k) = (a, b): expansion along the
//      line with 16-byte shared-memory reads of the x2/x3 rows, the D_Z^-1
//      scaling (DZM: 0 the uniform grid's table row in registers; 1 computed
//      in the kernel; 2 the element's table in global memory), the x1
//      contraction, and the line of u written to shared memory;
//   3. pass 2, per element the node (i, m) = (a, b): the x2 and x3
//      contractions of u and their face residuals; the x1 faces of the tile.
// Face ownership.  An x1-face between two elements of the same tile is
// summed in shared memory and stored once.  Every other face value is
// shared with another tile (or is a Neumann boundary face with one
// contributor): its contribution(s) are added with red.global.add into an
// output zeroed before the launch.  Exactly two additions reach a shared
// face value and they commute in IEEE arithmetic, so the result is bitwise
// independent of the tiling and of the order in which tiles run.
#pragma once

#include "cg_fused.cuh"

namespace hdg {

// Row length R of the tile kernel's shared-memory rows (SD2, SD3, U): the
// D_Z^-1 table row dz_row(N), padded for 16-byte reads, and for FP32 rows of
// more than 8 entries a multiple of 8 plus 4, so that the 16-byte row
// accesses of 8 consecutive threads (one shared-memory wavefront) fall in
// distinct banks (rows of 16 words put two of them on the same banks).
template <typename T, int N>
__host__ __device__ constexpr int tile_row() {
  return (sizeof(T) == 4 && N > 8 && dz_row(N, 4) % 8 == 0) ? dz_row(N, 4) + 4 : dz_row(N, sizeof(T));
}
template <typename T, int N>
__host__ __device__ constexpr int tile_smem_per_elem() {
  // SD2, SD3 (2 x N rows each), U (N^2 rows), X1, X1H, OX1 (lo, hi): N^2 each
  return 4 * N * tile_row<T, N>() + N * N * tile_row<T, N>() + 4 * N * N;
}
constexpr int kTileMaxE = 32;
constexpr int kTileMaxThreads = 384;
// elements per thread and phase (E = G x rounds): the six face values of each
// are loaded into registers before any is stored, 24 FP32 or 12 FP64
// registers' worth at most, which keeps the FP64 instantiations free of spills
template <typename T, int CGM = 0>
__host__ __device__ constexpr int tile_rounds() { return CGM ? 1 : (sizeof(T) == 8 ? 2 : 4); }
// face offsets of a tile element: x1 lo/hi, x2 lo/hi, x3 lo/hi (face base,
// -1 on a Dirichlet plane), element index, flags
struct __align__(16) TileOff {
  int f[6];
  int elem;
  int flags;   // 1: next element of the tile in the same x1-pencil; 2: previous
               // one; 4: low x1-plane is the domain boundary; 8: high one;
               // 16, 32: low x2-, x3-plane is the domain boundary
};

__device__ __forceinline__ void load_met(const float* p, float& d0, float& d1, float& d2, float& d3) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  d0 = v.x; d1 = v.y; d2 = v.z; d3 = v.w;
}
__device__ __forceinline__ void load_met(const double* p, double& d0, double& d1, double& d2, double& d3) {
  const double2 v = reinterpret_cast<const double2*>(p)[0], w = reinterpret_cast<const double2*>(p)[1];
  d0 = v.x; d1 = v.y; d2 = w.x; d3 = w.y;
}

__device__ __forceinline__ TileOff load_off(const TileOff* p) {
  const int4 a = reinterpret_cast<const int4*>(p)[0], b = reinterpret_cast<const int4*>(p)[1];
  TileOff o;
  o.f[0] = a.x; o.f[1] = a.y; o.f[2] = a.z; o.f[3] = a.w;
  o.f[4] = b.x; o.f[5] = b.y; o.elem = b.z; o.flags = b.w;
  return o;
}

// Sum of the two contributions to a face value formed inside a tile, as the
// two additions onto zero would form it: FP32/FP64 storage a + b; BF16
// storage rounds each contribution to BF16 first (as red_add does) and the
// sum once more, so that the stored value does not depend on whether the
// face's two elements fell into one tile.
template <typename ST, typename T>
__device__ __forceinline__ T pair_sum(T a, T b) {
  if constexpr (std::is_same<ST, __nv_bfloat16>::value)
    return __bfloat162float(__float2bfloat16_rn(a)) + __bfloat162float(__float2bfloat16_rn(b));
  else
    return a + b;
}

// Element groups G of a CTA (n^2 G threads, at most kTileMaxThreads, G <=
// kTileMaxE) for degree n, and the CTA size it gives.
__host__ __device__ constexpr int tile_groups(int n) {
  return kTileMaxThreads / (n * n) < 1 ? 1 : (kTileMaxThreads / (n * n) > kTileMaxE ? kTileMaxE : kTileMaxThreads / (n * n));
}
// CTA size: n^2 G working threads, rounded up to whole warps (the padding
// threads take part in barriers and warp reductions only)
__host__ __device__ constexpr int tile_cta_threads(int n) { return (n * n * tile_groups(n) + 31) / 32 * 32; }

// The exact CTA size in the launch bounds lets the compiler give each thread
// the registers of three (FP32) or two (FP64) resident CTAs.
// CGM: 0 operator application; 1 fused CG step (one iteration per launch);
// 2 persistent CG (every iteration of an inner solve in one cooperative
// launch, one grid barrier per iteration).
template <typename T, typename ST, int N, int DZM, int CGM = 0>
__global__ void __launch_bounds__(tile_cta_threads(N), sizeof(T) == 4 ? (CGM ? 2 : 3) : (CGM ? 1 : 2)) tpt_tile_kernel(const TptArgs<T, ST> a) {
  constexpr bool CG = CGM > 0;
  constexpr bool DZC = DZM == 1;
  constexpr int N2 = N * N, NE = (N + 1) / 2;
  constexpr int R = tile_row<T, N>();
  constexpr int VL = Vec<T>::L, NQ = (N + VL - 1) / VL;   // vectors covering a row (R may pad further)
  using V = typename Vec<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int E = a.seg;    // elements per tile (host: E <= kTileMaxE, E = G RR)
  const int G = a.ppb;    // element groups: blockDim.x = N^2 G
  const int RR = E / G;   // elements per thread and phase (host: <= tile_rounds)
  // carve: SD2 | SD3 | U | X1 | X1H | OX1lo | OX1hi
  T* SD2 = sm;
  T* SD3 = SD2 + E * 2 * N * R;
  T* U = SD3 + E * 2 * N * R;
  T* X1 = U + E * N2 * R;
  T* X1H = X1 + E * N2;
  T* OXL = X1H + E * N2;
  T* OXH = OXL + E * N2;
  __shared__ TileOff s_off[2][kTileMaxE];
  __shared__ __align__(16) T s_met[2][kTileMaxE][4];
  __shared__ CgScalars s_cg;

  const int rhs = blockIdx.y;
  grid_dep_wait();   // everything below reads what the previous kernel in the stream wrote
  if (a.skip && a.skip[rhs]) return;   // uniform per block
  const HookPre hpre = hook_prefetch(a.hook, rhs, &s_cg);

  const MeshDev& m = a.mesh;
  const int N1e = m.ne[0], N2e = m.ne[1], N3e = m.ne[2];
  const int pl0 = N2e * N3e, pl1 = N1e * N3e, pl2 = N1e * N2e;
  const int nelem = N1e * pl0;
  const int ntiles = (nelem + E - 1) / E;
  const int tid = threadIdx.x;
  const long long toff = (long long)rhs * a.trace_stride;
  const ST* __restrict__ xin = a.x + toff;
  ST* __restrict__ yout = a.y + toff;
  const T hs = a.tab.h0 + a.tab.h1, hd = a.tab.h0 - a.tab.h1;
  const T lam_r = DZC ? static_cast<T>(a.lam[rhs]) : T(0);
  T dot = T(0);

  // offsets and metric of the elements of `tile` into buffer b
  auto tile_offsets = [&](int tile, int b) {
    if (tid < E) {
      const int e = tile * E + tid;
      TileOff o;
      if (e < nelem) {
        const int e1 = e % N1e, rest = e / N1e, e2 = rest % N2e, e3 = rest / N2e;
        auto face = [&](int d, int plane, int fab, int pl) -> int {
          return (plane >= m.lo[d] && plane <= m.hi[d]) ? ((int)m.blk[d] + (plane - m.lo[d]) * pl + fab) * N2 : -1;
        };
        o.f[0] = face(0, e1, e2 + N2e * e3, pl0);
        o.f[1] = face(0, e1 + 1, e2 + N2e * e3, pl0);
        o.f[2] = face(1, e2, e1 + N1e * e3, pl1);
        o.f[3] = face(1, e2 + 1, e1 + N1e * e3, pl1);
        o.f[4] = face(2, e3, e1 + N1e * e2, pl2);
        o.f[5] = face(2, e3 + 1, e1 + N1e * e2, pl2);
        o.elem = e;
        o.flags = (e1 + 1 < N1e && tid + 1 < E && e + 1 < nelem ? 1 : 0) | (e1 > 0 && tid > 0 ? 2 : 0) |
                  (e1 == 0 ? 4 : 0) | (e1 + 1 == N1e ? 8 : 0) | (e2 == 0 ? 16 : 0) | (e3 == 0 ? 32 : 0);
        const T* mt = a.metric + (m.uniform ? 0 : 4 * (long long)e);
        s_met[b][tid][0] = mt[0];
        s_met[b][tid][1] = mt[1];
        s_met[b][tid][2] = mt[2];
        s_met[b][tid][3] = mt[3];
      } else {
        for (int k = 0; k < 6; ++k) o.f[k] = -1;
        o.elem = -1;
        o.flags = 0;
      }
      s_off[b][tid] = o;
    }
  };

  // this thread's face node q = (qa, qb) (lower axis qa) and element group g:
  // the x1-line (j, k) = (qa, qb) in pass 1 and the face node (i, m) = (qa, qb)
  // of the x2/x3 contractions in pass 2, for the elements g, g + G, ... of
  // every tile; all of its index arithmetic is done once here
  const bool active = tid < N2 * G;
  const int q = tid % N2, g = active ? tid / N2 : 0;
  const int qa = q % N, qb = q / N;
  const T cj = a.tab.c[qa], ck = a.tab.c[qb];
  const T lj = a.tab.lam[qa], lk = a.tab.lam[qb];
  const int rowB = (qa < NE ? 0 : N * R) + R * qb;   // (S2|D2)(., k) by the parity of j
  const int rowC = (qb < NE ? 0 : N * R) + R * qa;   // (S3|D3)(., j) by the parity of k
  constexpr int RT = dz_row(N, sizeof(T));          // D_Z^-1 table row
  const int line = R * (qa + N * qb);                // U row (j, k)
  const int dzline = RT * (qa + N * qb);             // D_Z^-1 row (j, k)
  const int node = R * qb + qa;                      // face node (a, b) in a row array
  // uniform grid: the thread's row of the D_Z^-1 table in registers
  T dzr[N];
  if constexpr (DZM == 0) {
    const T* dz = a.dinv + (long long)rhs * a.dinv_rhs_stride + dzline;
    static_for<0, N>([&](auto ic) { dzr[decltype(ic)::value] = dz[decltype(ic)::value]; });
  }

  __syncthreads();   // s_cg (hook_prefetch) visible to every thread
  // fused CG step: the step scalars of iteration i (from the previous
  // launch's last block, or in the persistent kernel from this CTA's own
  // reduction after the previous grid barrier)
  T al = T(0), be = T(0), gam = T(0);
  unsigned int bar_gen = 0;   // persistent kernel: grid barriers passed
  if constexpr (CG) {
    al = static_cast<T>(s_cg.alpha);
    be = static_cast<T>(s_cg.beta);
  }
  // The value of a face node the operator acts on: the stored input, or in
  // CG mode u_{i+1} = W r_{i+1} from the update of iteration i; the face's
  // owner (the element below it, or its only element) also stores the
  // updated x, p, r, s, zeroes the w buffer of the launch after next and
  // adds its r . u to gamma.  In CG mode every load of the thread's six face
  // values is issued before any of them is used or stored (the vectors are
  // distinct buffers, declared so through restrict-qualified copies).
  T* __restrict__ vx = a.cgv.x;
  T* __restrict__ vp = a.cgv.p;
  const T* __restrict__ vW = a.cgv.W;
  constexpr int kR = tile_rounds<T, CGM>();

  // the persistent kernel's iterations; one pass for the other modes
  for (int iter = 0;; ++iter) {
  // buffers of this iteration: r and s rotate with period 2, w with period 3
  // (the persistent kernel rotates them itself, launch by launch otherwise)
  const int i2 = CGM == 2 ? iter % 2 : 0, i3 = CGM == 2 ? iter % 3 : 0;
  const T* r_b[2] = {a.cgv.r_in, a.cgv.r_out};
  const T* s_b[2] = {a.cgv.s_in, a.cgv.s_out};
  const T* w_b[3] = {a.cgv.w_in, reinterpret_cast<const T*>(a.y), a.cgv.w_zero};
  const T* __restrict__ vr = r_b[i2];
  T* __restrict__ vro = const_cast<T*>(r_b[i2 ^ 1]);
  const T* __restrict__ vs = s_b[i2];
  T* __restrict__ vso = const_cast<T*>(s_b[i2 ^ 1]);
  const T* __restrict__ vw = w_b[i3];
  T* __restrict__ vwz = const_cast<T*>(w_b[(i3 + 2) % 3]);
  if constexpr (CGM == 2) yout = reinterpret_cast<ST*>(const_cast<T*>(w_b[(i3 + 1) % 3])) + toff;

  int tile = blockIdx.x;
  int buf = 0;
  tile_offsets(tile, buf);
  __syncthreads();
  for (; tile < ntiles; tile += gridDim.x, buf ^= 1) {
    const TileOff* off = s_off[buf];
    // ---- 1. staging: every load of the thread's elements first ---------------
    T v[kR][6];
    static_for<0, kR>([&](auto rc) {
      constexpr int r = decltype(rc)::value;
      T* w = v[r];
      w[0] = w[1] = w[2] = w[3] = w[4] = w[5] = T(0);
      if (active && r < RR) {
        const TileOff o = load_off(off + g + r * G);
        if constexpr (!CG) {
          if (o.f[2] >= 0) w[0] = load_as<ST, T>(xin + o.f[2] + q);
          if (o.f[3] >= 0) w[1] = load_as<ST, T>(xin + o.f[3] + q);
          if (o.f[4] >= 0) w[2] = load_as<ST, T>(xin + o.f[4] + q);
          if (o.f[5] >= 0) w[3] = load_as<ST, T>(xin + o.f[5] + q);
          if (o.f[0] >= 0) w[4] = load_as<ST, T>(xin + o.f[0] + q);
          if (!(o.flags & 1) && o.f[1] >= 0) w[5] = load_as<ST, T>(xin + o.f[1] + q);
        } else {
          // slots x2 lo/hi, x3 lo/hi, x1 lo, x1 hi: offset (or -1), owner
          const int fo[6] = {o.f[2], o.f[3], o.f[4], o.f[5], o.f[0], (o.flags & 1) ? -1 : o.f[1]};
          const bool own[6] = {(o.flags & 16) != 0, true, (o.flags & 32) != 0, true, (o.flags & 6) != 0, true};
          T lr[6], lw[6], ls[6], lW[6], lp[6], lx[6];
          static_for<0, 6>([&](auto kc) {
            constexpr int k = decltype(kc)::value;
            const long long oo = toff + (fo[k] >= 0 ? fo[k] + q : 0);
            const bool on = fo[k] >= 0, ow = on && own[k];
            // the persistent kernel reads vectors other CTAs wrote during
            // this launch: through L2 (ld.cg), never a stale L1 line
            lr[k] = on ? ld_state<CGM>(vr + oo) : T(0);
            lw[k] = on ? ld_state<CGM>(vw + oo) : T(0);
            ls[k] = on ? ld_state<CGM>(vs + oo) : T(0);
            lW[k] = (on && vW) ? vW[oo] : T(1);
            lp[k] = ow ? ld_state<CGM>(vp + oo) : T(0);
            lx[k] = ow ? ld_state<CGM>(vx + oo) : T(0);
          });
          static_for<0, 6>([&](auto kc) {
            constexpr int k = decltype(kc)::value;
            if (fo[k] >= 0) {
              const long long oo = toff + fo[k] + q;
              const T sn = fma(be, ls[k], lw[k]);
              const T rn = fma(-al, sn, lr[k]);
              const T un = lW[k] * rn;
              w[k] = un;
              if (own[k]) {
                const T pn = fma(be, lp[k], lW[k] * lr[k]);
                vx[oo] = fma(al, pn, lx[k]);
                vp[oo] = pn;
                vso[oo] = sn;
                vro[oo] = rn;
                vwz[oo] = T(0);
                gam = fma(un, rn, gam);
              }
            }
          });
        }
      }
    });
    static_for<0, kR>([&](auto rc) {
      constexpr int r = decltype(rc)::value;
      if (active && r < RR) {
        const int el = g + r * G;
        const T* w = v[r];
        // x2 face node (i, k) -> row k; x3 face node (i, j) -> row j
        T* s2 = SD2 + el * 2 * N * R + node;
        s2[0] = w[0] + w[1];
        s2[N * R] = w[0] - w[1];
        T* s3 = SD3 + el * 2 * N * R + node;
        s3[0] = w[2] + w[3];
        s3[N * R] = w[2] - w[3];
        X1[el * N2 + q] = w[4];
        X1H[el * N2 + q] = w[5];
      }
    });
    // offsets of the next tile (its buffer was last read by the previous tile)
    if (tile + (int)gridDim.x < ntiles) tile_offsets(tile + gridDim.x, buf ^ 1);
    __syncthreads();

    // ---- 2. pass 1: the x1-line (j, k) of each element --------------------------
    for (int r = 0; r < (active ? RR : 0); ++r) {
      const int el = g + r * G;
      const TileOff o = load_off(off + el);
      if (o.elem < 0) continue;
      T d0, d1, d2, d3;
      load_met(&s_met[buf][el][0], d0, d1, d2, d3);
      const int it = el * N2 + q;
      const T xl = X1[it];
      const T xh = (o.flags & 1) ? X1[it + N2] : X1H[it];
      const T S1 = xl + xh, D1 = xl - xh;
      const T Ap = d1 * S1, Am = d1 * D1;
      const T cjd2 = cj * d2, ckd3 = ck * d3;
      const T* Bs = SD2 + el * 2 * N * R + rowB;
      const T* Cs = SD3 + el * 2 * N * R + rowC;
      const T* dzg = nullptr;
      if constexpr (DZM == 2) dzg = a.dinv + (long long)rhs * a.dinv_rhs_stride + (long long)o.elem * (N2 * RT) + dzline;
      T dzb = T(0);
      if constexpr (DZC) dzb = fma(d3, lk, fma(d2, lj, lam_r * d0));
      T* Ur = U + el * N2 * R + line;
      T Pp = T(0), Pm = T(0);
      if constexpr (std::is_same<T, float>::value) {
        // FP32: pairs of points (i, i + 1) in packed two-lane FP32 arithmetic
        // (one FFMA2/FMUL2 per pair); the x1 contraction keeps one two-lane
        // accumulator per parity combination of a pair
        float2 pEE = make_float2(0.f, 0.f), pOO = pEE, pEO = pEE;
        const float2 cjd2v = make_float2(cjd2, cjd2), ckd3v = make_float2(ckd3, ckd3);
        static_for<0, NQ>([&](auto qc) {
          constexpr int qq = decltype(qc)::value;
          const float4 bv = *reinterpret_cast<const float4*>(Bs + 4 * qq);
          const float4 cv = *reinterpret_cast<const float4*>(Cs + 4 * qq);
          float4 dv = make_float4(0.f, 0.f, 0.f, 0.f);
          if constexpr (DZM == 2) dv = *reinterpret_cast<const float4*>(dzg + 4 * qq);
          (void)dv;
          float2 uh[2];
          static_for<0, 2>([&](auto hc) {
            constexpr int hh = decltype(hc)::value;
            constexpr int i0 = 4 * qq + 2 * hh, i1 = i0 + 1;
            if constexpr (i0 < N) {
              constexpr bool e0 = i0 < NE, e1 = i1 < NE, v1 = i1 < N;
              const float c0 = a.tab.c[i0], c1 = v1 ? a.tab.c[i1] : 0.f;
              // the second lane of the last pair of an odd row (i1 = N) lies in
              // the row padding, which no thread writes: it takes zeros, never
              // the padding (0 x a stale NaN or Inf there would be NaN)
              const float b0 = hh == 0 ? bv.x : bv.z, b1 = v1 ? (hh == 0 ? bv.y : bv.w) : 0.f;
              const float k0 = hh == 0 ? cv.x : cv.z, k1 = v1 ? (hh == 0 ? cv.y : cv.w) : 0.f;
              float2 F = __fmul2_rn(make_float2(c0, c1), make_float2(e0 ? Ap : Am, e1 ? Ap : Am));
              F = __ffma2_rn(cjd2v, make_float2(b0, b1), F);
              F = __ffma2_rn(ckd3v, make_float2(k0, k1), F);
              float2 inv;
              if constexpr (DZM == 0) {
                inv = make_float2(dzr[i0], v1 ? dzr[i1] : 0.f);
              } else if constexpr (DZC) {
                const float2 den = __ffma2_rn(make_float2(d1, d1),
                                              make_float2(a.tab.lam[i0], v1 ? a.tab.lam[i1] : 0.f),
                                              make_float2(dzb, dzb));
                inv = make_float2(dz_recip(den.x), v1 ? dz_recip(den.y) : 0.f);
              } else {
                inv = make_float2(hh == 0 ? dv.x : dv.z, v1 ? (hh == 0 ? dv.y : dv.w) : 0.f);
              }
              const float2 u = __fmul2_rn(F, inv);
              uh[hh] = u;
              const float2 cc = make_float2(c0, c1);
              if constexpr (e0 && e1) pEE = __ffma2_rn(cc, u, pEE);
              else if constexpr (!e0 && !e1) pOO = __ffma2_rn(cc, u, pOO);
              else pEO = __ffma2_rn(cc, u, pEO);
            } else {
              uh[hh] = make_float2(0.f, 0.f);
            }
          });
          *reinterpret_cast<float4*>(Ur + 4 * qq) = make_float4(uh[0].x, uh[0].y, uh[1].x, uh[1].y);
        });
        Pp = (pEE.x + pEE.y) + pEO.x;
        Pm = (pOO.x + pOO.y) + pEO.y;
      } else {
      static_for<0, NQ>([&](auto qc) {
        constexpr int qq = decltype(qc)::value;
        const V bv = *reinterpret_cast<const V*>(Bs + VL * qq);
        const V cv = *reinterpret_cast<const V*>(Cs + VL * qq);
        V dv{};
        if constexpr (DZM == 2) dv = *reinterpret_cast<const V*>(dzg + VL * qq);
        (void)dv;
        V uv;
        static_for<0, VL>([&](auto lc) {
          constexpr int l = decltype(lc)::value;
          constexpr int i = VL * qq + l;
          if constexpr (i < N) {
            T F = a.tab.c[i] * (i < NE ? Ap : Am);
            F = fma(cjd2, vget(bv, l), F);
            F = fma(ckd3, vget(cv, l), F);
            T inv;
            if constexpr (DZM == 0) inv = dzr[i];
            else if constexpr (DZC) inv = dz_recip(fma(d1, a.tab.lam[i], dzb));
            else inv = vget(dv, l);
            const T u = F * inv;
            vset(uv, l, u);
            if constexpr (i < NE) Pp = fma(a.tab.c[i], u, Pp);
            else Pm = fma(a.tab.c[i], u, Pm);
          } else {
            vset(uv, l, T(0));
          }
        });
        *reinterpret_cast<V*>(Ur + VL * qq) = uv;
      });
      }
      // x1 face residuals of this line (node (j, k) of the lo and hi faces)
      const T sum = d1 * (hs * S1 - T(2) * Pp), dif = d1 * (hd * D1 - T(2) * Pm);
      OXL[it] = T(0.5) * (sum + dif);
      OXH[it] = T(0.5) * (sum - dif);
      dot = fma(S1, sum, fma(D1, dif, dot));
    }
    __syncthreads();

    // ---- 3. pass 2: x2/x3 contractions at the node (i, m), x1 faces -------------
    for (int r = 0; r < (active ? RR : 0); ++r) {
      const int el = g + r * G;
      const TileOff o = load_off(off + el);
      if (o.elem < 0) continue;
      const T d2 = s_met[buf][el][2], d3 = s_met[buf][el][3];
      const T* Uq = U + el * N2 * R + R * N * qb + qa;   // (i, j = mo, k = m): + R mo
      const T* Uk = U + el * N2 * R + R * qb + qa;       // (i, j = m, k = mo): + R N mo
      T Qp = T(0), Qm = T(0), Rp = T(0), Rm = T(0);
      if constexpr (std::is_same<T, float>::value) {
        // FP32: the x2 and x3 contractions as one two-lane accumulator per parity
        float2 QRp = make_float2(0.f, 0.f), QRm = QRp;
        static_for<0, N>([&](auto mc) {
          constexpr int mo = decltype(mc)::value;
          const float2 uu = make_float2(Uq[R * mo], Uk[R * N * mo]);
          const float2 cm = make_float2(a.tab.c[mo], a.tab.c[mo]);
          if constexpr (mo < NE) QRp = __ffma2_rn(cm, uu, QRp);
          else QRm = __ffma2_rn(cm, uu, QRm);
        });
        Qp = QRp.x; Rp = QRp.y; Qm = QRm.x; Rm = QRm.y;
      } else {
        static_for<0, N>([&](auto mc) {
          constexpr int mo = decltype(mc)::value;
          const T uq = Uq[R * mo];
          const T ur = Uk[R * N * mo];
          if constexpr (mo < NE) { Qp = fma(a.tab.c[mo], uq, Qp); Rp = fma(a.tab.c[mo], ur, Rp); }
          else                   { Qm = fma(a.tab.c[mo], uq, Qm); Rm = fma(a.tab.c[mo], ur, Rm); }
        });
      }
      {  // x2 faces, node (i, k = m)
        const T* s2 = SD2 + el * 2 * N * R + node;
        const T Sv = s2[0], Dv = s2[N * R];
        const T sum = d2 * (hs * Sv - T(2) * Qp), dif = d2 * (hd * Dv - T(2) * Qm);
        red_add_if(o.f[2] >= 0, yout + (max(o.f[2], 0) + q), T(0.5) * (sum + dif));
        red_add_if(o.f[3] >= 0, yout + (max(o.f[3], 0) + q), T(0.5) * (sum - dif));
        dot = fma(Sv, sum, fma(Dv, dif, dot));
      }
      {  // x3 faces, node (i, j = m)
        const T* s3 = SD3 + el * 2 * N * R + node;
        const T Sv = s3[0], Dv = s3[N * R];
        const T sum = d3 * (hs * Sv - T(2) * Rp), dif = d3 * (hd * Dv - T(2) * Rm);
        red_add_if(o.f[4] >= 0, yout + (max(o.f[4], 0) + q), T(0.5) * (sum + dif));
        red_add_if(o.f[5] >= 0, yout + (max(o.f[5], 0) + q), T(0.5) * (sum - dif));
        dot = fma(Sv, sum, fma(Dv, dif, dot));
      }
      // x1 faces, node q: the lo face of this element (stored when the tile
      // holds both of its contributions or it is a boundary face, else added),
      // and its hi face where the next element of the tile does not own it
      const int it = el * N2 + q;
      {
        const bool on = o.f[0] >= 0, st = on && (o.flags & 6) != 0;
        // (it - N2 stays inside the shared buffers for el = 0: OXH follows OXL)
        const T lv = (o.flags & 2) ? pair_sum<ST>(OXL[it], OXH[it - N2]) : OXL[it];
        ST* dst = yout + (max(o.f[0], 0) + q);
        st_if(st, dst, lv);
        red_add_if(on && !st, dst, lv);
      }
      {
        const bool on = o.f[1] >= 0 && !(o.flags & 1), st = on && (o.flags & 8) != 0;
        ST* dst = yout + (max(o.f[1], 0) + q);
        st_if(st, dst, OXH[it]);
        red_add_if(on && !st, dst, OXH[it]);
      }
    }
    __syncthreads();   // the next tile restages every buffer
  }
  if constexpr (CGM != 2) break;
  else {
    // end of iteration `iter`: per-block partial sums of delta and gamma
    // (buffer by the parity of the iteration: a fast CTA may write the next
    // iteration's partials while a slow one still reads these), one grid
    // barrier, then every CTA forms the step scalars from all partials in the
    // same fixed order, so that every CTA takes the same decisions
    if (!persistent_step(a.hook, a.cgv, rhs, iter, dot, gam, &s_cg, &bar_gen)) break;
    if (s_cg.done) break;
    al = static_cast<T>(s_cg.alpha);
    be = static_cast<T>(s_cg.beta);
    dot = T(0);
    gam = T(0);
  }
  }   // iterations

  if constexpr (CGM == 2) {
    if (blockIdx.x == 0 && tid == 0) {
      a.hook.cg[rhs] = s_cg;
      a.hook.flags[rhs] = 1;
    }
    return;
  }
  grid_dep_launch();   // the next kernel's blocks may take this block's place
  if constexpr (CG) hook_finish_cg(a.hook, a.cgv.gpartials, rhs, dot, gam, &s_cg);
  else if (a.hook.partials != nullptr) hook_finish(a.hook, rhs, dot, hpre, &s_cg);
}

}  // namespace hdg
