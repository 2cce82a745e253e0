// Face and volume tensor-product transforms, D_Z^-1 tables, vector kernels
// and the CG scalar updates of the condensed HDG library.
#include <algorithm>
#include <cfloat>

#include "internal.h"

namespace hdg {
namespace {

constexpr int kVecThreads = 256;

inline unsigned int grid_for(long long count, int threads, long long cap = 152LL * 32) {
  long long b = (count + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (unsigned int)b;
}

// ---- 4-wide vector access (16-byte transactions) ---------------------------------
// Streaming kernels load every operand of a group of 4 consecutive entries
// before storing anything, so the loads of a group are all in flight at
// once; the group path needs 16-byte aligned rows (length % 4 == 0).
template <typename T>
__device__ __forceinline__ void ld4(const T* p, T v[4]);
template <>
__device__ __forceinline__ void ld4<float>(const float* p, float v[4]) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
}
template <>
__device__ __forceinline__ void ld4<double>(const double* p, double v[4]) {
  const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
template <typename T>
__device__ __forceinline__ void st4(T* p, const T v[4]);
template <>
__device__ __forceinline__ void st4<float>(float* p, const float v[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
template <>
__device__ __forceinline__ void st4<double>(double* p, const double v[4]) {
  reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
}

// ---- volume transforms: y_e = s_e (A (x) A (x) A) x_e -------------------------
// One 1D line transform out[a] = sum_i A[a][i] in[i] of n values.
// PAR = 0: dense, n^2 multiply-adds.  The basis-change matrices inherit the
// mirror symmetry of the GLL points, with the eigenmodes ordered [even | odd]
// (m < NE even, sigma_m = +1; else odd, sigma_m = -1):
// PAR = 1 (rows are modes: S^T, S^T M): A[m][n-1-i] = sigma_m A[m][i], so an
//   even mode only sees in[i] + in[n-1-i] and an odd one in[i] - in[n-1-i];
// PAR = 2 (columns are modes: S, M S): A[n-1-i][m] = sigma_m A[i][m], so
//   out[i] = E_i + O_i and out[n-1-i] = E_i - O_i with the even- and
//   odd-mode partial sums E_i, O_i.
// Either parity form takes about n^2 / 2 multiply-adds.
template <int N, int PAR, typename T>
__device__ __forceinline__ void line_transform(const Mat1D<T>& A, const T (&in)[N], T (&out)[N]) {
  constexpr int NE = (N + 1) / 2, H = N / 2;
  if constexpr (PAR == 1) {
    T sp[NE], dm[H > 0 ? H : 1];
#pragma unroll
    for (int i = 0; i < H; ++i) {
      sp[i] = in[i] + in[N - 1 - i];
      dm[i] = in[i] - in[N - 1 - i];
    }
    if constexpr (N % 2 == 1) sp[H] = in[H];
#pragma unroll
    for (int a = 0; a < N; ++a) {
      T v = T(0);
      if (a < NE) {
#pragma unroll
        for (int i = 0; i < NE; ++i) v = fma(A.a[a * N + i], sp[i], v);
      } else {
#pragma unroll
        for (int i = 0; i < H; ++i) v = fma(A.a[a * N + i], dm[i], v);
      }
      out[a] = v;
    }
  } else if constexpr (PAR == 2) {
#pragma unroll
    for (int i = 0; i < NE; ++i) {
      T ev = T(0), od = T(0);
#pragma unroll
      for (int m = 0; m < NE; ++m) ev = fma(A.a[i * N + m], in[m], ev);
#pragma unroll
      for (int m = NE; m < N; ++m) od = fma(A.a[i * N + m], in[m], od);
      out[i] = ev + od;
      if (N - 1 - i != i) out[N - 1 - i] = ev - od;
    }
  } else {
#pragma unroll
    for (int a = 0; a < N; ++a) {
      T v = T(0);
#pragma unroll
      for (int i = 0; i < N; ++i) v = fma(A.a[a * N + i], in[i], v);
      out[a] = v;
    }
  }
}

// ---- face transforms (Sec. 4.2 basis change), one thread per face row:
//      y_f = scale (W (x) W) x_f ------------------------------------------------
// Thread l of a face first transforms row l (T[l][.] = W x[l][.]), then,
// after a barrier, column l (y[.][l] = scale W T[.][l]); both with the
// line transform above, so the matrix entries are compile-time operands and
// mirror-symmetric matrices take the parity-split form.
template <typename TI, typename TO, int N, int PAR>
__global__ void face_rows_kernel(const TI* __restrict__ x, TO* __restrict__ y, long long nfaces, long long sx,
                                 long long sy, const Mat1D<TO> W, TO scale, int accumulate, int fpb) {
  constexpr int N2 = N * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TO* sm = reinterpret_cast<TO*>(smem_raw);
  const int slot = threadIdx.x / N;
  const int l = threadIdx.x - slot * N;
  const long long face = (long long)blockIdx.x * fpb + slot;
  const bool act = slot < fpb && face < nfaces;
  const int r = blockIdx.y;
  TO* Tm = sm + (act ? slot : 0) * N2;   // T[row][a1]
  if (act) {
    const TI* xf = x + r * sx + face * N2 + N * l;
    TO in[N], out[N];
#pragma unroll
    for (int c = 0; c < N; ++c) in[c] = load_as<TI, TO>(xf + c);
    line_transform<N, PAR>(W, in, out);
#pragma unroll
    for (int a = 0; a < N; ++a) Tm[N * l + a] = out[a];
  }
  __syncthreads();
  if (act) {
    TO in[N], out[N];
#pragma unroll
    for (int c = 0; c < N; ++c) in[c] = Tm[N * c + l];
    line_transform<N, PAR>(W, in, out);
    TO* yf = y + r * sy + face * N2 + l;
#pragma unroll
    for (int a = 0; a < N; ++a) {
      TO v = scale * out[a];
      if (accumulate) v += yf[N * a];
      yf[N * a] = v;
    }
  }
}

// Runtime-n forms of the two transforms, for degrees above the specialised
// instantiations: the same products, the matrix staged in shared memory.
// Face transform: one slot of n threads per face (row pass, then column
// pass through shared memory).
template <typename TI, typename TO>
__global__ void face_rows_generic_kernel(const TI* __restrict__ x, TO* __restrict__ y, long long nfaces,
                                         long long sx, long long sy, const Mat1D<TO> W, TO scale, int accumulate,
                                         int fpb, int n) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TO* Wm = reinterpret_cast<TO*>(smem_raw);   // W[row][col], n x n
  TO* sm = Wm + n * n;
  const int n2 = n * n;
  for (int t = threadIdx.x; t < n2; t += blockDim.x) Wm[t] = W.a[t];
  const int slot = threadIdx.x / n;
  const int l = threadIdx.x - slot * n;
  const long long face = (long long)blockIdx.x * fpb + slot;
  const bool act = slot < fpb && face < nfaces;
  const int r = blockIdx.y;
  TO* Tm = sm + (act ? slot : 0) * n2;
  __syncthreads();
  if (act) {
    const TI* xf = x + r * sx + face * n2 + n * l;
    for (int a = 0; a < n; ++a) {
      TO acc = TO(0);
      for (int c = 0; c < n; ++c) acc = fma(Wm[a * n + c], load_as<TI, TO>(xf + c), acc);
      Tm[n * l + a] = acc;
    }
  }
  __syncthreads();
  if (act) {
    TO* yf = y + r * sy + face * n2 + l;
    for (int a = 0; a < n; ++a) {
      TO acc = TO(0);
      for (int c = 0; c < n; ++c) acc = fma(Wm[a * n + c], Tm[n * c + l], acc);
      TO v = scale * acc;
      if (accumulate) v += yf[n * a];
      yf[n * a] = v;
    }
  }
}

// Volume transform y_e = s_e (A (x) A (x) A) x_e: one CTA per element, three
// passes of line transforms (x1 lines from x into y, then x2 and x3 lines of
// y in place: each line is read whole into registers by the one thread that
// writes it back), the scale applied in the last pass.
constexpr int kGenericLine = 33;
__global__ void __launch_bounds__(256) volume_transform_generic_kernel(const double* __restrict__ x, double* y,
                                                                       long long nelem, long long stride,
                                                                       const Mat1D<double> A,
                                                                       const double* __restrict__ metric,
                                                                       int uniform, int use_d0, int n) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* Am = reinterpret_cast<double*>(smem_raw);
  const int n2 = n * n;
  for (int t = threadIdx.x; t < n2; t += blockDim.x) Am[t] = A.a[t];
  __syncthreads();
  const int r = blockIdx.y;
  for (long long e = blockIdx.x; e < nelem; e += gridDim.x) {
    const double* xe = x + r * stride + e * (long long)(n2 * n);
    double* ye = y + r * stride + e * (long long)(n2 * n);
    const double sc = use_d0 ? metric[uniform ? 0 : 4 * e] : 1.0;
    for (int pass = 0; pass < 3; ++pass) {
      const int st = pass == 0 ? 1 : (pass == 1 ? n : n2);   // stride along the line
      for (int line = threadIdx.x; line < n2; line += blockDim.x) {
        const int la = line % n, lb = line / n;
        // first node of the line: the two other indices (la, lb)
        const long long b0 = pass == 0 ? (long long)n * la + (long long)n2 * lb
                                       : (pass == 1 ? la + (long long)n2 * lb : la + (long long)n * lb);
        const double* src = pass == 0 ? xe + b0 : ye + b0;
        double in[kGenericLine];
        for (int c = 0; c < n; ++c) in[c] = src[(long long)c * st];
        for (int a = 0; a < n; ++a) {
          double acc = 0.0;
          for (int c = 0; c < n; ++c) acc = fma(Am[a * n + c], in[c], acc);
          ye[b0 + (long long)a * st] = pass == 2 ? sc * acc : acc;
        }
      }
      __syncthreads();   // the next pass reads lines other threads wrote
    }
  }
}

template <int N, int PAR>
__global__ void volume_transform_kernel(const double* __restrict__ x, double* __restrict__ y,
                                        long long nelem, long long stride, const Mat1D<double> A,
                                        const double* __restrict__ metric, int uniform, int use_d0,
                                        int epb) {
  constexpr int N2 = N * N, N3 = N2 * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sm = reinterpret_cast<double*>(smem_raw);
  const int slot = threadIdx.x / N2;
  const int q = threadIdx.x - slot * N2;
  const long long e = (long long)blockIdx.x * epb + slot;
  const bool act = slot < epb && e < nelem;
  const int r = blockIdx.y;
  double* B0 = sm + (act ? slot : 0) * 2 * N3;
  double* B1 = B0 + N3;
  const double* xe = x + r * stride + e * N3;
  const int lo = q % N, hi = q / N;
  if (act) {
#pragma unroll
    for (int t = 0; t < N; ++t) B0[q + N2 * t] = xe[q + N2 * t];
  }
  __syncthreads();
  // pass 1 (x1): B1[k][j][a] = sum_i A[a][i] B0[k][j][i]; thread (j, k) = (lo, hi)
  if (act) {
    double in[N], out[N];
#pragma unroll
    for (int i = 0; i < N; ++i) in[i] = B0[i + N * lo + N2 * hi];
    line_transform<N, PAR>(A, in, out);
#pragma unroll
    for (int aa = 0; aa < N; ++aa) B1[aa + N * lo + N2 * hi] = out[aa];
  }
  __syncthreads();
  // pass 2 (x2): B0[k][b][i] = sum_j A[b][j] B1[k][j][i]; thread (i, k) = (lo, hi)
  if (act) {
    double in[N], out[N];
#pragma unroll
    for (int j = 0; j < N; ++j) in[j] = B1[lo + N * j + N2 * hi];
    line_transform<N, PAR>(A, in, out);
#pragma unroll
    for (int bb = 0; bb < N; ++bb) B0[lo + N * bb + N2 * hi] = out[bb];
  }
  __syncthreads();
  // pass 3 (x3): y[c][j][i] = s sum_k A[c][k] B0[k][j][i]; thread (i, j) = (lo, hi)
  if (act) {
    const double s = use_d0 ? metric[uniform ? 0 : 4 * e] : 1.0;
    double in[N], out[N];
#pragma unroll
    for (int k = 0; k < N; ++k) in[k] = B0[lo + N * hi + N2 * k];
    line_transform<N, PAR>(A, in, out);
    double* ye = y + r * stride + e * N3;
#pragma unroll
    for (int cc = 0; cc < N; ++cc) ye[lo + N * hi + N2 * cc] = s * out[cc];
  }
}

// ---- D_Z^-1 tables (Sec. 4.1, fast diagonalisation) -------------------------------
// Layout: [rhs][class][k][j][i], rows of dz_row(n) entries (padding = 0).
template <typename T>
__global__ void dinv_kernel(int n, const double* __restrict__ lam, int nrhs,
                            const double* __restrict__ metric, long long nclass,
                            const double* __restrict__ Lambda, T* __restrict__ out) {
  const int row = dz_row(n, sizeof(T));
  const long long per = (long long)n * n * row;
  const long long total = (long long)nrhs * nclass * per;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long pidx = t % per;
    const long long cls = (t / per) % nclass;
    const int r = (int)(t / (per * nclass));
    const int i = (int)(pidx % row), j = (int)((pidx / row) % n), k = (int)(pidx / ((long long)row * n));
    if (i >= n) {
      out[t] = T(0);
      continue;
    }
    const double* mt = metric + 4 * cls;
    const double dz = lam[r] * mt[0] + mt[1] * Lambda[i] + mt[2] * Lambda[j] + mt[3] * Lambda[k];
    out[t] = static_cast<T>(1.0 / dz);
  }
}

// ---- Neumann load in the transformed basis -------------------------------------
__global__ void neumann_add_kernel(MeshDev m, int n, const double* __restrict__ widths, int wstride,
                                   const double* __restrict__ ghat, double* __restrict__ F,
                                   long long bstride, long long tstride) {
  const int r = blockIdx.y;
  const long long n2 = (long long)n * n;
  const long long total = m.nbfaces * n2;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long bf = t / n2, node = t % n2;
    int side = 5;
    while (side > 0 && bf < m.side[side]) --side;
    const int d = side / 2, s = side % 2;
    const int plane = s == 0 ? 0 : m.ne[d];
    if (plane < m.lo[d] || plane > m.hi[d]) continue;   // Dirichlet side
    const int ax = d == 0 ? 1 : 0, bx = d == 2 ? 1 : 2;
    const long long ab = bf - m.side[side];
    const int Na = m.ne[ax];
    const int ea = (int)(ab % Na), eb = (int)(ab / Na);
    const double scale = widths[ax * wstride + ea] * widths[bx * wstride + eb] * 0.25;
    const long long Na_Nb = (long long)Na * m.ne[bx];
    const long long uf = m.blk[d] + (long long)(plane - m.lo[d]) * Na_Nb + ab;
    F[r * tstride + uf * n2 + node] += scale * ghat[r * bstride + t];
  }
}

// ---- face-block Jacobi preconditioner in the transformed basis (Sec. 5.1) ----
// The self-coupling of a face f in K-hat is the sum over its two elements of
// d (I (x) I (x) H) - d^2 (I (x) I (x) B_S^T) D_Z^-1 (I (x) I (x) B_S) restricted
// to f's side s; with B_S[m][s]^2 = c_m^2 it is diagonal in the face modes:
//   Y(a, b) = sum_e [ d h0 - d^2 sum_m c_m^2 D_Z^-1(m, a, b) ].
__global__ void pc_diag_kernel(MeshDev m, int n, Tables<double> tab, const double* __restrict__ metric,
                               const double* __restrict__ dinv, long long dinv_rhs_stride,
                               const double* __restrict__ lam, double* __restrict__ diag, long long tstride) {
  const int r = blockIdx.y;
  const int n2 = n * n;
  const long long nel = (long long)m.ne[0] * m.ne[1] * m.ne[2];
  const long long total = nel * n2;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long e = t / n2;
    const int q = (int)(t - e * n2);
    const int lo = q % n, hi = q / n;
    const int e1 = (int)(e % m.ne[0]), e2 = (int)((e / m.ne[0]) % m.ne[1]);
    const int e3 = (int)(e / ((long long)m.ne[0] * m.ne[1]));
    const double* mt = metric + (m.uniform ? 0 : 4 * e);
    const int row = dz_row(n, sizeof(double));
    const double* dz = dinv ? dinv + r * dinv_rhs_stride + (m.uniform ? 0 : e * (long long)n2 * row) : nullptr;
    // D_Z^-1(i, j, k) from the table, or computed (no table above the
    // specialised degrees)
    auto dzv = [&](int i, int j, int k) -> double {
      if (dz) return dz[i + row * (j + n * k)];
      return 1.0 / (lam[r] * mt[0] + mt[1] * tab.lam[i] + mt[2] * tab.lam[j] + mt[3] * tab.lam[k]);
    };
    double sd[3] = {0.0, 0.0, 0.0};
    for (int t2 = 0; t2 < n; ++t2) {
      const double c2 = tab.c[t2] * tab.c[t2];
      sd[0] += c2 * dzv(t2, lo, hi);   // x1 face node (j, k) = (lo, hi)
      sd[1] += c2 * dzv(lo, t2, hi);   // x2 face node (i, k) = (lo, hi)
      sd[2] += c2 * dzv(lo, hi, t2);   // x3 face node (i, j) = (lo, hi)
    }
    const int ed[3] = {e1, e2, e3};
    const long long fab[3] = {e2 + (long long)m.ne[1] * e3, e1 + (long long)m.ne[0] * e3,
                              e1 + (long long)m.ne[0] * e2};
    const long long pl[3] = {(long long)m.ne[1] * m.ne[2], (long long)m.ne[0] * m.ne[2],
                             (long long)m.ne[0] * m.ne[1]};
    for (int d = 0; d < 3; ++d) {
      const double dd = mt[1 + d];
      const double v = dd * tab.h0 - dd * dd * sd[d];
      for (int s = 0; s < 2; ++s) {
        const int plane = ed[d] + s;
        if (plane < m.lo[d] || plane > m.hi[d]) continue;
        red_add(diag + r * tstride + (m.blk[d] + (long long)(plane - m.lo[d]) * pl[d] + fab[d]) * n2 + q, v);
      }
    }
  }
}

__global__ void pc_invert_kernel(const double* __restrict__ diag, double* __restrict__ w64,
                                 float* __restrict__ w32, long long count) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < count;
       t += (long long)gridDim.x * blockDim.x) {
    const double w = 1.0 / diag[t];
    w64[t] = w;
    w32[t] = (float)w;
  }
}

// ---- element-wise helpers ----------------------------------------------------------
template <typename TI, typename TO>
__global__ void convert_kernel(const TI* __restrict__ x, TO* __restrict__ y, long long count) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < count;
       t += (long long)gridDim.x * blockDim.x)
    store_from<TO, TO>(y + t, static_cast<TO>(load_as<TI, double>(x + t)));
}
template <>
__global__ void convert_kernel<double, __nv_bfloat16>(const double* __restrict__ x,
                                                      __nv_bfloat16* __restrict__ y, long long count) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < count;
       t += (long long)gridDim.x * blockDim.x)
    y[t] = __double2bfloat16(x[t]);
}

__global__ void sub_kernel(const double* __restrict__ a, const double* __restrict__ b,
                           double* __restrict__ out, long long count) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < count;
       t += (long long)gridDim.x * blockDim.x)
    out[t] = a[t] - b[t];
}

template <typename T>
__global__ void add_to_kernel(double* __restrict__ x, const T* __restrict__ d, long long count) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < count;
       t += (long long)gridDim.x * blockDim.x)
    x[t] += static_cast<double>(d[t]);
}

// y[r] = scale[r] x[r] in FP32 (grid.y = rhs); scale[r] is a power of two,
// so the scaling itself is exact and only the conversion rounds
__global__ void scale_convert_kernel(const double* __restrict__ x, float* __restrict__ y, long long len,
                                     const double* __restrict__ scale) {
  const long long o = (long long)blockIdx.y * len;
  const double sc = scale[blockIdx.y];
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < len; t += (long long)gridDim.x * blockDim.x)
    y[o + t] = static_cast<float>(sc * x[o + t]);
}

// x[r] += inv_scale[r] d[r] (inv_scale a power of two: exact)
__global__ void add_unscaled_kernel(double* __restrict__ x, const float* __restrict__ d, long long len,
                                    const double* __restrict__ inv_scale) {
  const long long o = (long long)blockIdx.y * len;
  const double inv = inv_scale[blockIdx.y];
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < len; t += (long long)gridDim.x * blockDim.x)
    x[o + t] += inv * static_cast<double>(d[o + t]);
}

// block sum of a double, result valid in thread 0
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double ws[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) ws[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x + 31) / 32; ++i) s += ws[i];
  return s;
}

// Writes the block partial; returns true in every thread of the last block
// to finish (block-uniform), after which every partial of right-hand side r
// is visible.
__device__ __forceinline__ bool finish_partial(double s, double* partials, unsigned int* counter, int r) {
  __shared__ bool last;
  if (threadIdx.x == 0) {
    partials[(long long)r * gridDim.x + blockIdx.x] = s;
    __threadfence();
    const unsigned int done = atomicAdd(counter + r, 1u);
    last = (done == gridDim.x - 1);
  }
  __syncthreads();
  const bool l = last;
  if (l) __threadfence();
  return l;
}

// Sum of the gridDim.x partials of right-hand side r by the whole (last)
// block: fixed strided split and fixed tree, so the result is deterministic.
// Valid in thread 0.
__device__ __forceinline__ double sum_partials(const double* partials, int r) {
  const volatile double* pp = partials + (long long)r * gridDim.x;
  double v = 0.0;
  for (unsigned int b = threadIdx.x; b < gridDim.x; b += blockDim.x) v += pp[b];
  return block_sum(v);
}

template <typename T>
__global__ void dot_kernel(const T* __restrict__ a, const T* __restrict__ b, const T* __restrict__ w,
                           long long len, double* partials, unsigned int* counter, double* out) {
  const int r = blockIdx.y;
  const T* ar = a + r * len;
  const T* br = b + r * len;
  const T* wr = w ? w + r * len : nullptr;
  double acc = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < len;
       t += (long long)gridDim.x * blockDim.x) {
    const double ab = static_cast<double>(ar[t]) * static_cast<double>(br[t]);
    acc += wr ? ab * static_cast<double>(wr[t]) : ab;
  }
  const double s = block_sum(acc);
  if (finish_partial(s, partials, counter, r)) {
    const double tot = sum_partials(partials, r);
    if (threadIdx.x == 0) {
      out[r] = tot;
      counter[r] = 0u;
    }
  }
}

// FP32 dot: accumulate in FP32 per thread (no FP64 arithmetic in the loop)
template <>
__global__ void dot_kernel<float>(const float* __restrict__ a, const float* __restrict__ b,
                                  const float* __restrict__ w, long long len, double* partials,
                                  unsigned int* counter, double* out) {
  const int r = blockIdx.y;
  const float* ar = a + r * len;
  const float* br = b + r * len;
  const float* wr = w ? w + r * len : nullptr;
  float acc = 0.f;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < len;
       t += (long long)gridDim.x * blockDim.x)
    acc = fmaf(wr ? ar[t] * wr[t] : ar[t], br[t], acc);
  const double s = block_sum((double)acc);
  if (finish_partial(s, partials, counter, r)) {
    const double tot = sum_partials(partials, r);
    if (threadIdx.x == 0) {
      out[r] = tot;
      counter[r] = 0u;
    }
  }
}

// ---- CG scalars ----------------------------------------------------------------------
__global__ void cg_init_kernel(CgScalars* cg, int* flags, const double* rr, const double* tol, int max_it,
                               int nrhs) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrhs) return;
  CgScalars c;
  c.rr = rr[r];
  c.rr_stop = tol[r] * tol[r] * c.rr;
  c.rr_old = 0.0;
  c.alpha = 0.0;
  c.beta = 0.0;
  c.it = 0;
  c.ops = 0;
  c.max_it = max_it;
  c.status = 0;
  c.done = (flags[r] != 0) || !(c.rr > 0.0) || max_it <= 0;
  if (!(c.rr >= 0.0) || c.rr != c.rr) c.status = 6;
  cg[r] = c;
  flags[r] = c.done;
}

// One iteration of the single-reduction preconditioned CG of Chronopoulos
// and Gear, after the operator launch w_i = K u_i, whose last block already
// produced the step scalars alpha_i, beta_i (cg_scalars):
//   p_i = u_i + beta_i p_{i-1},  s_i = w_i + beta_i s_{i-1}   (s_i = K p_i)
//   x_{i+1} = x_i + alpha_i p_i,  r_{i+1} = r_i - alpha_i s_i
//   u_{i+1} = W r_{i+1},  gamma_{i+1} = r_{i+1} . u_{i+1}.
// In exact arithmetic these are the iterates of the standard preconditioned
// CG; the two inner products of an iteration meet in one reduction phase, so
// an iteration is two kernels (operator, this update).  gamma_{i+1} is left
// as one partial sum per block in `partials`: the next operator launch's
// last block adds them up (in a fixed order) with its own inner product, so
// this kernel has no grid-wide reduction tail.  w is zeroed for the next
// operator launch, which accumulates into it.  Every thread issues all loads
// of its entries before it reads the scalars; one resident wave of blocks
// covers the vectors.
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 2)
    cg_step_kernel(const CgScalars* cg, const int* flags, T* __restrict__ x, T* __restrict__ rvec,
                   T* __restrict__ u, T* __restrict__ wv, T* __restrict__ p, T* __restrict__ sv,
                   const T* __restrict__ W, long long len, double* partials) {
  const int r = blockIdx.y;
  const long long o = r * len;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nvec = (len % 4 == 0) ? len / 4 : 0;
  // u_i = W r_i is formed again from W and r (bitwise the stored product)
  // instead of being read: 6 streams read (w, p, s, x, r, W), 6 written.
  // The first group's p, s, x, r and W were written by the update launch
  // before the operator (complete before the operator's blocks passed their
  // own wait, hence before this launch began), and the operator does not
  // write them: they are loaded while the operator's last block is still
  // reducing.  w, the scalars and the flags are the operator's and are read
  // after the wait; every store comes after it.
  // Two groups of 4 entries per thread (v = tid and tid + stride): all of
  // their operator-independent loads are issued before the wait, and the w
  // loads of both after it, so that one resident wave covers the vectors
  // with a single dependent round trip; groups beyond are handled by the
  // loop after them.
  constexpr int KG = 2;
  T wq[KG][4], pv[KG][4], sq[KG][4], xv[KG][4], rv[KG][4], mv[KG][4];
#pragma unroll
  for (int g = 0; g < KG; ++g) {
    const long long v = tid + g * stride;
#pragma unroll
    for (int k = 0; k < 4; ++k) mv[g][k] = T(1);
    if (v < nvec) {
      const long long t = o + 4 * v;
      ld4(p + t, pv[g]);
      ld4(sv + t, sq[g]);
      ld4(x + t, xv[g]);
      ld4(rvec + t, rv[g]);
      if (W) ld4(W + t, mv[g]);
    }
  }
  grid_dep_wait();     // the operator launch before this one wrote w, the scalars and flags
  grid_dep_launch();   // the next operator launch may queue its blocks behind this wave
  if (flags[r]) return;
  const T zero[4] = {T(0), T(0), T(0), T(0)};
  T acc = T(0);
  const T al = static_cast<T>(cg[r].alpha), be = static_cast<T>(cg[r].beta);
#pragma unroll
  for (int g = 0; g < KG; ++g) {
    const long long v = tid + g * stride;
    if (v < nvec) ld4(wv + o + 4 * v, wq[g]);
  }
  auto step = [&](long long v, T (&pg)[4], T (&sg)[4], T (&xg)[4], T (&rg)[4], const T (&mg)[4], const T (&wg)[4]) {
    const long long t = o + 4 * v;
    T ug[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      pg[k] = fma(be, pg[k], mg[k] * rg[k]);   // u = W r of this iteration, bitwise as stored
      sg[k] = fma(be, sg[k], wg[k]);
      xg[k] = fma(al, pg[k], xg[k]);
      rg[k] = fma(-al, sg[k], rg[k]);
      ug[k] = mg[k] * rg[k];
      acc = fma(ug[k], rg[k], acc);
    }
    st4(p + t, pg);
    st4(sv + t, sg);
    st4(x + t, xg);
    st4(rvec + t, rg);
    st4(u + t, ug);
    st4(wv + t, zero);
  };
#pragma unroll
  for (int g = 0; g < KG; ++g) {
    const long long v = tid + g * stride;
    if (v < nvec) step(v, pv[g], sq[g], xv[g], rv[g], mv[g], wq[g]);
  }
  for (long long v = tid + KG * stride; v < nvec; v += stride) {
    const long long t = o + 4 * v;
    T p1[4], s1[4], x1[4], r1[4], m1[4] = {T(1), T(1), T(1), T(1)}, w1[4];
    ld4(p + t, p1);
    ld4(sv + t, s1);
    ld4(x + t, x1);
    ld4(rvec + t, r1);
    if (W) ld4(W + t, m1);
    ld4(wv + t, w1);
    step(v, p1, s1, x1, r1, m1, w1);
  }
  {
    const T al = static_cast<T>(cg[r].alpha), be = static_cast<T>(cg[r].beta);
    for (long long t = o + nvec * 4 + tid; t < o + len; t += stride) {
      const T pn = fma(be, p[t], (W ? W[t] : T(1)) * rvec[t]);
      const T sn = fma(be, sv[t], wv[t]);
      const T rn = fma(-al, sn, rvec[t]);
      const T un = (W ? W[t] : T(1)) * rn;
      x[t] = fma(al, pn, x[t]);
      p[t] = pn;
      sv[t] = sn;
      rvec[t] = rn;
      u[t] = un;
      wv[t] = T(0);
      acc = fma(un, rn, acc);
    }
  }
  // warp sums in T (FP64 arithmetic is slow on this part), then FP64 across warps
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, m);
  __shared__ double wsum[8];
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = static_cast<double>(acc);
  __syncthreads();
  if (threadIdx.x == 0) {
    double sblk = 0.0;
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) sblk += wsum[w];
    partials[(long long)r * gridDim.x + blockIdx.x] = sblk;
  }
}

template <typename T>
__global__ void cg_pupdate_kernel(const CgScalars* cg, T* __restrict__ p, const T* __restrict__ rvec,
                                  const T* __restrict__ w, long long len) {
  const int r = blockIdx.y;
  if (cg[r].done) return;
  __shared__ T s_beta;
  if (threadIdx.x == 0) s_beta = static_cast<T>(cg[r].beta);
  __syncthreads();
  const T beta = s_beta;
  T* __restrict__ pr = p + r * len;
  const T* __restrict__ rr = rvec + r * len;
  const T* __restrict__ wr = w ? w + r * len : nullptr;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nvec = (len % 4 == 0) ? len / 4 : 0;
  for (long long v = tid; v < nvec; v += stride) {
    const long long t = 4 * v;
    T pv[4], rv[4], wv[4] = {T(1), T(1), T(1), T(1)};
    ld4(pr + t, pv);
    ld4(rr + t, rv);
    if (wr) ld4(wr + t, wv);
#pragma unroll
    for (int k = 0; k < 4; ++k) pv[k] = fma(beta, pv[k], wv[k] * rv[k]);   // p = z + beta p
    st4(pr + t, pv);
  }
  for (long long t = nvec * 4 + tid; t < len; t += stride) {
    const T z = wr ? wr[t] * rr[t] : rr[t];
    pr[t] = fma(beta, pr[t], z);
  }
}

// Mirror-symmetry form of A (see line_transform): 1 rows, 2 columns, 0 none.
// Checked to a relative 1e-13 of the largest entry; the parity kernels then
// use only the first half of each row or column.
int matrix_parity(int n, const Mat1D<double>& A) {
  const int ne = (n + 1) / 2;
  double amax = 0.0;
  for (int i = 0; i < n * n; ++i) amax = fmax(amax, fabs(A.a[i]));
  const double tol = 1e-13 * amax;
  bool row = true, col = true;
  for (int a = 0; a < n; ++a)
    for (int i = 0; i < n; ++i) {
      const double sa = a < ne ? 1.0 : -1.0, si = i < ne ? 1.0 : -1.0;
      row = row && fabs(A.a[a * n + (n - 1 - i)] - sa * A.a[a * n + i]) <= tol;
      col = col && fabs(A.a[(n - 1 - a) * n + i] - si * A.a[a * n + i]) <= tol;
    }
  return row ? 1 : (col ? 2 : 0);
}

template <typename TI, typename TO, int N, int PAR>
cudaError_t ft_launch(const TI* x, TO* y, long long nfaces, int nrhs, long long sx, long long sy,
                      const Mat1D<TO>& W, TO scale, int accumulate, cudaStream_t s) {
  const int fpb = std::max(1, 256 / N);
  const int threads = (fpb * N + 31) / 32 * 32;
  const size_t smem = (size_t)fpb * N * N * sizeof(TO);
  if (smem > kSmemOptIn)
    cudaFuncSetAttribute(face_rows_kernel<TI, TO, N, PAR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  dim3 grid((unsigned)((nfaces + fpb - 1) / fpb), nrhs);
  if (nfaces <= 0) return cudaSuccess;
  face_rows_kernel<TI, TO, N, PAR><<<grid, threads, smem, s>>>(x, y, nfaces, sx, sy, W, scale, accumulate, fpb);
  return cudaGetLastError();
}

template <typename TI, typename TO, int N>
cudaError_t ft_one(const TI* x, TO* y, long long nfaces, int nrhs, long long sx, long long sy,
                   const Mat1D<double>& Wd, double scale, int accumulate, cudaStream_t s) {
  Mat1D<TO> W;
  for (int i = 0; i < N * N; ++i) W.a[i] = static_cast<TO>(Wd.a[i]);
  const TO sc = static_cast<TO>(scale);
  switch (matrix_parity(N, Wd)) {
    case 1: return ft_launch<TI, TO, N, 1>(x, y, nfaces, nrhs, sx, sy, W, sc, accumulate, s);
    case 2: return ft_launch<TI, TO, N, 2>(x, y, nfaces, nrhs, sx, sy, W, sc, accumulate, s);
    default: return ft_launch<TI, TO, N, 0>(x, y, nfaces, nrhs, sx, sy, W, sc, accumulate, s);
  }
}

template <int N, int PAR>
cudaError_t vt_launch(const double* x, double* y, long long nelem, int nrhs, long long stride,
                      const Mat1D<double>& A, const double* metric, int uniform, int use_d0,
                      cudaStream_t s) {
  const int epb = (256 / (N * N)) > 0 ? 256 / (N * N) : 1;
  const int threads = (epb * N * N + 31) / 32 * 32;
  const size_t smem = (size_t)epb * 2 * N * N * N * sizeof(double);
  if (smem > kSmemOptIn)
    cudaFuncSetAttribute(volume_transform_kernel<N, PAR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  dim3 grid((unsigned)((nelem + epb - 1) / epb), nrhs);
  if (nelem <= 0) return cudaSuccess;
  volume_transform_kernel<N, PAR><<<grid, threads, smem, s>>>(x, y, nelem, stride, A, metric, uniform,
                                                             use_d0, epb);
  return cudaGetLastError();
}

template <int N>
cudaError_t vt_one(const double* x, double* y, long long nelem, int nrhs, long long stride,
                   const Mat1D<double>& A, const double* metric, int uniform, int use_d0,
                   cudaStream_t s) {
  switch (matrix_parity(N, A)) {
    case 1: return vt_launch<N, 1>(x, y, nelem, nrhs, stride, A, metric, uniform, use_d0, s);
    case 2: return vt_launch<N, 2>(x, y, nelem, nrhs, stride, A, metric, uniform, use_d0, s);
    default: return vt_launch<N, 0>(x, y, nelem, nrhs, stride, A, metric, uniform, use_d0, s);
  }
}

}  // namespace

#define HDG_N_SWITCH(n, CALL, GENERIC)                                          \
  switch (n) {                                                                  \
    case 2: return CALL(2); case 3: return CALL(3); case 4: return CALL(4);     \
    case 5: return CALL(5); case 6: return CALL(6); case 7: return CALL(7);     \
    case 8: return CALL(8); case 9: return CALL(9); case 10: return CALL(10);   \
    case 11: return CALL(11); case 12: return CALL(12); case 13: return CALL(13); \
    case 14: return CALL(14); case 15: return CALL(15); case 16: return CALL(16); \
    case 17: return CALL(17);                                                   \
    default: return GENERIC;                                                    \
  }

template <typename TI, typename TO>
cudaError_t ft_generic(int n, const TI* x, TO* y, long long nfaces, int nrhs, long long sx, long long sy,
                       const Mat1D<double>& Wd, double scale, int accumulate, cudaStream_t s) {
  if (n < 2 || n > kMaxNDev) return cudaErrorInvalidValue;
  if (nfaces <= 0) return cudaSuccess;
  Mat1D<TO> W;
  for (int i = 0; i < n * n; ++i) W.a[i] = static_cast<TO>(Wd.a[i]);
  const int fpb = std::max(1, 256 / n);
  const int threads = (fpb * n + 31) / 32 * 32;
  const size_t smem = (size_t)(fpb + 1) * n * n * sizeof(TO);
  if (smem > kSmemOptIn)
    cudaFuncSetAttribute(face_rows_generic_kernel<TI, TO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  dim3 grid((unsigned)((nfaces + fpb - 1) / fpb), nrhs);
  face_rows_generic_kernel<TI, TO><<<grid, threads, smem, s>>>(x, y, nfaces, sx, sy, W, static_cast<TO>(scale),
                                                              accumulate, fpb, n);
  return cudaGetLastError();
}

cudaError_t vt_generic(int n, const double* x, double* y, long long nelem, int nrhs, long long stride,
                       const Mat1D<double>& A, const double* metric, int uniform, int use_d0, cudaStream_t s) {
  if (n < 2 || n > kGenericLine || n > kMaxNDev || x == y) return cudaErrorInvalidValue;
  if (nelem <= 0) return cudaSuccess;
  const size_t smem = (size_t)n * n * sizeof(double);
  const long long blocks = std::min<long long>(nelem, 65535LL * 4);
  dim3 grid((unsigned)blocks, nrhs);
  volume_transform_generic_kernel<<<grid, 256, smem, s>>>(x, y, nelem, stride, A, metric, uniform, use_d0, n);
  return cudaGetLastError();
}

template <typename TI, typename TO>
cudaError_t launch_face_transform(int n, const TI* x, TO* y, long long nfaces, int nrhs,
                                  long long stride_x, long long stride_y, const Mat1D<double>& W,
                                  double scale, int accumulate, cudaStream_t s) {
#define FT_CALL(N) ft_one<TI, TO, N>(x, y, nfaces, nrhs, stride_x, stride_y, W, scale, accumulate, s)
  HDG_N_SWITCH(n, FT_CALL, (ft_generic<TI, TO>(n, x, y, nfaces, nrhs, stride_x, stride_y, W, scale, accumulate, s)))
#undef FT_CALL
}
template cudaError_t launch_face_transform<double, double>(int, const double*, double*, long long, int,
                                                           long long, long long, const Mat1D<double>&,
                                                           double, int, cudaStream_t);
template cudaError_t launch_face_transform<float, float>(int, const float*, float*, long long, int,
                                                         long long, long long, const Mat1D<double>&,
                                                         double, int, cudaStream_t);

cudaError_t launch_volume_transform(int n, const double* x, double* y, long long nelem, int nrhs,
                                    long long stride, const Mat1D<double>& A, const double* metric,
                                    int uniform, int use_d0, cudaStream_t s) {
#define VT_CALL(N) vt_one<N>(x, y, nelem, nrhs, stride, A, metric, uniform, use_d0, s)
  HDG_N_SWITCH(n, VT_CALL, (vt_generic(n, x, y, nelem, nrhs, stride, A, metric, uniform, use_d0, s)))
#undef VT_CALL
}

template <typename T>
cudaError_t launch_dinv(int n, const double* lambda_dev, int nrhs, const double* metric,
                        long long nclass, const double* Lambda_dev, T* out, cudaStream_t s) {
  const long long total = (long long)nrhs * nclass * n * n * dz_row(n, sizeof(T));
  dinv_kernel<T><<<grid_for(total, kVecThreads), kVecThreads, 0, s>>>(n, lambda_dev, nrhs, metric,
                                                                      nclass, Lambda_dev, out);
  return cudaGetLastError();
}
template cudaError_t launch_dinv<double>(int, const double*, int, const double*, long long,
                                         const double*, double*, cudaStream_t);
template cudaError_t launch_dinv<float>(int, const double*, int, const double*, long long,
                                        const double*, float*, cudaStream_t);

cudaError_t launch_neumann_add(const MeshDev& m, int n, const double* widths_dev, int wstride,
                               const double* ghat, double* F, int nrhs, long long bstride,
                               long long tstride, cudaStream_t s) {
  const long long total = m.nbfaces * n * n;
  dim3 grid(grid_for(total, kVecThreads), nrhs);
  neumann_add_kernel<<<grid, kVecThreads, 0, s>>>(m, n, widths_dev, wstride, ghat, F, bstride, tstride);
  return cudaGetLastError();
}

template <typename TI, typename TO>
cudaError_t launch_convert(const TI* x, TO* y, long long count, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  convert_kernel<TI, TO><<<grid_for(count, kVecThreads), kVecThreads, 0, s>>>(x, y, count);
  return cudaGetLastError();
}
template cudaError_t launch_convert<double, float>(const double*, float*, long long, cudaStream_t);
template cudaError_t launch_convert<float, double>(const float*, double*, long long, cudaStream_t);
template cudaError_t launch_convert<double, double>(const double*, double*, long long, cudaStream_t);
template cudaError_t launch_convert<double, __nv_bfloat16>(const double*, __nv_bfloat16*, long long,
                                                          cudaStream_t);

cudaError_t launch_scale_convert(const double* x, float* y, long long len, int nrhs, const double* scale,
                                 cudaStream_t s) {
  if (len <= 0 || nrhs <= 0) return cudaSuccess;
  dim3 grid(grid_for(len, kVecThreads), nrhs);
  scale_convert_kernel<<<grid, kVecThreads, 0, s>>>(x, y, len, scale);
  return cudaGetLastError();
}

cudaError_t launch_add_unscaled(double* x, const float* d, long long len, int nrhs, const double* inv_scale,
                                cudaStream_t s) {
  if (len <= 0 || nrhs <= 0) return cudaSuccess;
  dim3 grid(grid_for(len, kVecThreads), nrhs);
  add_unscaled_kernel<<<grid, kVecThreads, 0, s>>>(x, d, len, inv_scale);
  return cudaGetLastError();
}

cudaError_t launch_sub(const double* a, const double* b, double* out, long long count, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  sub_kernel<<<grid_for(count, kVecThreads), kVecThreads, 0, s>>>(a, b, out, count);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_add_to(double* x, const T* d, long long count, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  add_to_kernel<T><<<grid_for(count, kVecThreads), kVecThreads, 0, s>>>(x, d, count);
  return cudaGetLastError();
}
template cudaError_t launch_add_to<double>(double*, const double*, long long, cudaStream_t);
template cudaError_t launch_add_to<float>(double*, const float*, long long, cudaStream_t);

template <typename T>
cudaError_t launch_dot(const T* a, const T* b, const T* w, long long len, int nrhs, double* partials,
                       unsigned int* counter, double* out, int blocks, cudaStream_t s) {
  dim3 grid(blocks, nrhs);
  dot_kernel<T><<<grid, kVecThreads, 0, s>>>(a, b, w, len, partials, counter, out);
  return cudaGetLastError();
}
template cudaError_t launch_dot<double>(const double*, const double*, const double*, long long, int,
                                        double*, unsigned int*, double*, int, cudaStream_t);
template cudaError_t launch_dot<float>(const float*, const float*, const float*, long long, int, double*,
                                       unsigned int*, double*, int, cudaStream_t);

cudaError_t launch_pc_diag(const MeshDev& m, int n, const Tables<double>& tab, const double* metric,
                           const double* dinv, long long dinv_rhs_stride, const double* lam, double* diag,
                           int nrhs, long long tstride, cudaStream_t s) {
  const long long total = (long long)m.ne[0] * m.ne[1] * m.ne[2] * n * n;
  dim3 grid(grid_for(total, kVecThreads), nrhs);
  pc_diag_kernel<<<grid, kVecThreads, 0, s>>>(m, n, tab, metric, dinv, dinv_rhs_stride, lam, diag, tstride);
  return cudaGetLastError();
}

cudaError_t launch_pc_invert(const double* diag, double* w64, float* w32, long long count, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  pc_invert_kernel<<<grid_for(count, kVecThreads), kVecThreads, 0, s>>>(diag, w64, w32, count);
  return cudaGetLastError();
}

cudaError_t launch_cg_init(CgScalars* cg, int* flags, const double* rr, const double* tol, int max_it,
                           int nrhs, cudaStream_t s) {
  cg_init_kernel<<<(nrhs + 127) / 128, 128, 0, s>>>(cg, flags, rr, tol, max_it, nrhs);
  return cudaGetLastError();
}

template <typename T>
int cg_step_blocks(long long len) {
  static int per_sm = 0;
  static int sms = 0;
  if (per_sm == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
      sms = 152;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cg_step_kernel<T>, kVecThreads, 0) != cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
    cudaGetLastError();
  }
  // two groups of 4 entries per thread (cg_step_kernel)
  const long long need = (len / 4 + 2 * kVecThreads - 1) / (2 * kVecThreads);
  return (int)std::max(1LL, std::min(need, (long long)sms * per_sm));
}

template <typename T>
cudaError_t launch_cg_step(const CgScalars* cg, const int* flags, T* x, T* r, T* u, T* w, T* p, T* sv,
                           const T* W, long long len, int nrhs, double* partials, int blocks, bool pdl,
                           cudaStream_t s) {
  dim3 grid(blocks, nrhs);
  if (pdl) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(kVecThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, cg_step_kernel<T>, cg, flags, x, r, u, w, p, sv, W, len, partials);
  }
  cg_step_kernel<T><<<grid, kVecThreads, 0, s>>>(cg, flags, x, r, u, w, p, sv, W, len, partials);
  return cudaGetLastError();
}
template int cg_step_blocks<double>(long long);
template int cg_step_blocks<float>(long long);
template cudaError_t launch_cg_step<double>(const CgScalars*, const int*, double*, double*, double*, double*,
                                            double*, double*, const double*, long long, int, double*, int, bool,
                                            cudaStream_t);
template cudaError_t launch_cg_step<float>(const CgScalars*, const int*, float*, float*, float*, float*, float*,
                                           float*, const float*, long long, int, double*, int, bool, cudaStream_t);

template <typename T>
cudaError_t launch_cg_pupdate(const CgScalars* cg, T* p, const T* r, const T* w, long long len, int nrhs,
                              cudaStream_t s) {
  dim3 grid(grid_for(len, kVecThreads), nrhs);
  cg_pupdate_kernel<T><<<grid, kVecThreads, 0, s>>>(cg, p, r, w, len);
  return cudaGetLastError();
}
template cudaError_t launch_cg_pupdate<double>(const CgScalars*, double*, const double*, const double*,
                                               long long, int, cudaStream_t);
template cudaError_t launch_cg_pupdate<float>(const CgScalars*, float*, const float*, const float*,
                                              long long, int, cudaStream_t);

}  // namespace hdg
