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

#include "tpt_kernel.cuh"

namespace hdg {

// Shared-memory footprint of the tile kernel, in elements of T, for tile
// size E (rows of R = dz_row(N) entries, padded for 16-byte reads).
template <typename T, int N>
__host__ __device__ constexpr int tile_row() { return dz_row(N, sizeof(T)); }
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
template <typename T, bool CG = false>
__host__ __device__ constexpr int tile_rounds() { return CG ? (sizeof(T) == 8 ? 1 : 2) : (sizeof(T) == 8 ? 2 : 4); }
// face offsets of a tile element: x1 lo/hi, x2 lo/hi, x3 lo/hi (face base,
// -1 on a Dirichlet plane), element index, flags
struct TileOff {
  int f[6];
  int elem;
  int flags;   // 1: next element of the tile in the same x1-pencil; 2: previous
               // one; 4: low x1-plane is the domain boundary; 8: high one;
               // 16, 32: low x2-, x3-plane is the domain boundary
};

// End of a fused CG launch (launch i + 1): delta = u^T K u from the element
// contributions and gamma = r . u from the face owners, both of iteration
// i + 1, summed per warp in T, per block and across blocks in FP64 in a
// fixed order (deterministic); the last block to arrive forms the step
// scalars of iteration i + 1 (cg_scalars) for the next launch.
template <typename T>
__device__ __forceinline__ void hook_finish_cg(const CgHook& hook, double* gpartials, int rhs, T dot, T gam,
                                               const CgScalars* s_cg) {
  __shared__ double wsum[2][32];
  __shared__ bool last;
  const int tid = threadIdx.x;
  const T v = warp_sum(dot), gv = warp_sum(gam);
  if ((tid & 31) == 0) {
    wsum[0][tid >> 5] = static_cast<double>(v);
    wsum[1][tid >> 5] = static_cast<double>(gv);
  }
  __syncthreads();
  if (tid == 0) {
    double sd = 0.0, sg = 0.0;
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) {
      sd += wsum[0][w];
      sg += wsum[1][w];
    }
    hook.partials[(long long)rhs * gridDim.x + blockIdx.x] = 0.5 * sd;
    gpartials[(long long)rhs * gridDim.x + blockIdx.x] = sg;
    __threadfence();
    const unsigned int done = atomicAdd(hook.counter + rhs, 1u);
    last = (done == gridDim.x - 1);
    if (last) __threadfence();
  }
  __syncthreads();
  if (last && tid < 32) {
    const double* pp = hook.partials + (long long)rhs * gridDim.x;
    const double* gp = gpartials + (long long)rhs * gridDim.x;
    double sd = 0.0, sg = 0.0;
    for (int b = tid; b < (int)gridDim.x; b += 32) {
      sd += __ldcg(pp + b);
      sg += __ldcg(gp + b);
    }
    sd = warp_sum(sd);
    sg = warp_sum(sg);
    if (tid == 0) {
      cg_scalars(hook.cg + rhs, *s_cg, hook.flags + rhs, sd, sg);
      hook.pq[rhs] = sd;
      hook.counter[rhs] = 0u;
    }
  }
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

template <typename T, typename ST, int N, int DZM, bool CG = false>
__global__ void __launch_bounds__(kTileMaxThreads, sizeof(T) == 4 ? 3 : 2) tpt_tile_kernel(const TptArgs<T, ST> a) {
  constexpr bool DZC = DZM == 1;
  constexpr int N2 = N * N, NE = (N + 1) / 2;
  constexpr int R = tile_row<T, N>();
  constexpr int VL = Vec<T>::L, NQ = R / VL;
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
  __shared__ T s_met[2][kTileMaxE][4];
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
  const int q = tid % N2, g = tid / N2;
  const int qa = q % N, qb = q / N;
  const T cj = a.tab.c[qa], ck = a.tab.c[qb];
  const T lj = a.tab.lam[qa], lk = a.tab.lam[qb];
  const int rowB = (qa < NE ? 0 : N * R) + R * qb;   // (S2|D2)(., k) by the parity of j
  const int rowC = (qb < NE ? 0 : N * R) + R * qa;   // (S3|D3)(., j) by the parity of k
  const int line = R * (qa + N * qb);                // U row (j, k); D_Z^-1 row (j, k)
  const int node = R * qb + qa;                      // face node (a, b) in a row array
  // uniform grid: the thread's row of the D_Z^-1 table in registers
  T dzr[N];
  if constexpr (DZM == 0) {
    const T* dz = a.dinv + (long long)rhs * a.dinv_rhs_stride + line;
    static_for<0, N>([&](auto ic) { dzr[decltype(ic)::value] = dz[decltype(ic)::value]; });
  }

  int tile = blockIdx.x;
  int buf = 0;
  tile_offsets(tile, buf);
  __syncthreads();

  // fused CG step: the step scalars of iteration i (from the previous
  // launch's last block, read by hook_prefetch before the barrier above)
  T al = T(0), be = T(0), gam = T(0);
  if constexpr (CG) {
    al = static_cast<T>(s_cg.alpha);
    be = static_cast<T>(s_cg.beta);
  }
  // the value of a face node the operator acts on: the stored input, or in
  // CG mode u_{i+1} = W r_{i+1} from the update of iteration i; the face's
  // owner (the element below it, or its only element) also stores the
  // updated x, p, r, s, zeroes the w buffer of the launch after next and
  // adds its r . u to gamma
  auto face_value = [&](int off_, bool owner) -> T {
    if constexpr (!CG) {
      (void)owner;
      return load_as<ST, T>(xin + off_);
    } else {
      const CgVecs<T>& v = a.cgv;
      const long long o_ = toff + off_;
      const T r = v.r_in[o_], w = v.w_in[o_], sv = v.s_in[o_];
      const T wt = v.W ? v.W[o_] : T(1);
      const T sn = fma(be, sv, w);
      const T rn = fma(-al, sn, r);
      const T un = wt * rn;
      if (owner) {
        const T pn = fma(be, v.p[o_], wt * r);
        v.x[o_] = fma(al, pn, v.x[o_]);
        v.p[o_] = pn;
        v.s_out[o_] = sn;
        v.r_out[o_] = rn;
        v.w_zero[o_] = T(0);
        gam = fma(un, rn, gam);
      }
      return un;
    }
  };

  constexpr int kR = tile_rounds<T, CG>();
  for (; tile < ntiles; tile += gridDim.x, buf ^= 1) {
    const TileOff* off = s_off[buf];
    // ---- 1. staging: every load of the thread's elements first ---------------
    T v[kR][6];
    static_for<0, kR>([&](auto rc) {
      constexpr int r = decltype(rc)::value;
      T* w = v[r];
      w[0] = w[1] = w[2] = w[3] = w[4] = w[5] = T(0);
      if (r < RR) {
        const TileOff& o = off[g + r * G];
        if (o.f[2] >= 0) w[0] = face_value(o.f[2] + q, (o.flags & 16) != 0);
        if (o.f[3] >= 0) w[1] = face_value(o.f[3] + q, true);
        if (o.f[4] >= 0) w[2] = face_value(o.f[4] + q, (o.flags & 32) != 0);
        if (o.f[5] >= 0) w[3] = face_value(o.f[5] + q, true);
        if (o.f[0] >= 0) w[4] = face_value(o.f[0] + q, (o.flags & 6) != 0);
        if (!(o.flags & 1) && o.f[1] >= 0) w[5] = face_value(o.f[1] + q, true);
      }
    });
    static_for<0, kR>([&](auto rc) {
      constexpr int r = decltype(rc)::value;
      if (r < RR) {
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
    for (int r = 0; r < RR; ++r) {
      const int el = g + r * G;
      const TileOff& o = off[el];
      if (o.elem < 0) continue;
      const T d0 = s_met[buf][el][0], d1 = s_met[buf][el][1], d2 = s_met[buf][el][2], d3 = s_met[buf][el][3];
      const int it = el * N2 + q;
      const T xl = X1[it];
      const T xh = (o.flags & 1) ? X1[it + N2] : X1H[it];
      const T S1 = xl + xh, D1 = xl - xh;
      const T Ap = d1 * S1, Am = d1 * D1;
      const T cjd2 = cj * d2, ckd3 = ck * d3;
      const T* Bs = SD2 + el * 2 * N * R + rowB;
      const T* Cs = SD3 + el * 2 * N * R + rowC;
      const T* dzg = nullptr;
      if constexpr (DZM == 2) dzg = a.dinv + (long long)rhs * a.dinv_rhs_stride + (long long)o.elem * (N2 * R) + line;
      T dzb = T(0);
      if constexpr (DZC) dzb = fma(d3, lk, fma(d2, lj, lam_r * d0));
      T* Ur = U + el * N2 * R + line;
      T Pp = T(0), Pm = T(0);
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
      // x1 face residuals of this line (node (j, k) of the lo and hi faces)
      const T sum = d1 * (hs * S1 - T(2) * Pp), dif = d1 * (hd * D1 - T(2) * Pm);
      OXL[it] = T(0.5) * (sum + dif);
      OXH[it] = T(0.5) * (sum - dif);
      dot = fma(S1, sum, fma(D1, dif, dot));
    }
    __syncthreads();

    // ---- 3. pass 2: x2/x3 contractions at the node (i, m), x1 faces -------------
    for (int r = 0; r < RR; ++r) {
      const int el = g + r * G;
      const TileOff& o = off[el];
      if (o.elem < 0) continue;
      const T d2 = s_met[buf][el][2], d3 = s_met[buf][el][3];
      const T* Uq = U + el * N2 * R + R * N * qb + qa;   // (i, j = mo, k = m): + R mo
      const T* Uk = U + el * N2 * R + R * qb + qa;       // (i, j = m, k = mo): + R N mo
      T Qp = T(0), Qm = T(0), Rp = T(0), Rm = T(0);
      static_for<0, N>([&](auto mc) {
        constexpr int mo = decltype(mc)::value;
        const T uq = Uq[R * mo];
        const T ur = Uk[R * N * mo];
        if constexpr (mo < NE) { Qp = fma(a.tab.c[mo], uq, Qp); Rp = fma(a.tab.c[mo], ur, Rp); }
        else                   { Qm = fma(a.tab.c[mo], uq, Qm); Rm = fma(a.tab.c[mo], ur, Rm); }
      });
      {  // x2 faces, node (i, k = m)
        const T* s2 = SD2 + el * 2 * N * R + node;
        const T Sv = s2[0], Dv = s2[N * R];
        const T sum = d2 * (hs * Sv - T(2) * Qp), dif = d2 * (hd * Dv - T(2) * Qm);
        if (o.f[2] >= 0) red_add(yout + o.f[2] + q, T(0.5) * (sum + dif));
        if (o.f[3] >= 0) red_add(yout + o.f[3] + q, T(0.5) * (sum - dif));
        dot = fma(Sv, sum, fma(Dv, dif, dot));
      }
      {  // x3 faces, node (i, j = m)
        const T* s3 = SD3 + el * 2 * N * R + node;
        const T Sv = s3[0], Dv = s3[N * R];
        const T sum = d3 * (hs * Sv - T(2) * Rp), dif = d3 * (hd * Dv - T(2) * Rm);
        if (o.f[4] >= 0) red_add(yout + o.f[4] + q, T(0.5) * (sum + dif));
        if (o.f[5] >= 0) red_add(yout + o.f[5] + q, T(0.5) * (sum - dif));
        dot = fma(Sv, sum, fma(Dv, dif, dot));
      }
      // x1 faces, node q: the lo face of this element, and its hi face where
      // the next element of the tile does not own it
      const int it = el * N2 + q;
      if (o.f[0] >= 0) {
        if (o.flags & 2) store_from<ST, T>(yout + o.f[0] + q, pair_sum<ST>(OXL[it], OXH[it - N2]));
        else if (o.flags & 4) store_from<ST, T>(yout + o.f[0] + q, OXL[it]);
        else red_add(yout + o.f[0] + q, OXL[it]);
      }
      if (o.f[1] >= 0 && !(o.flags & 1)) {
        if (o.flags & 8) store_from<ST, T>(yout + o.f[1] + q, OXH[it]);
        else red_add(yout + o.f[1] + q, OXH[it]);
      }
    }
    __syncthreads();   // the next tile restages every buffer
  }

  grid_dep_launch();   // the next kernel's blocks may take this block's place
  if constexpr (CG) hook_finish_cg(a.hook, a.cgv.gpartials, rhs, dot, gam, &s_cg);
  else if (a.hook.partials != nullptr) hook_finish(a.hook, rhs, dot, hpre, &s_cg);
}

}  // namespace hdg
