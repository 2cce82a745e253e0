// Shared device-side definitions of the condensed HDG library (sm_103a).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace hdg {

constexpr int kMaxNDev = 33;   // p <= 32

// Dynamic shared memory above which a kernel's limit is raised explicitly
// (cudaFuncAttributeMaxDynamicSharedMemorySize).  The default limit of 48 KB
// covers dynamic plus static shared memory, and the operator kernels hold a
// little static shared memory for their reductions, so the opt-in starts
// well below 48 KB.
constexpr size_t kSmemOptIn = 40 * 1024;

// Cartesian mesh in the library's face-wise layout (see include/hdg.h).
struct MeshDev {
  int ne[3];          // elements per direction
  int lo[3], hi[3];   // unknown planes per direction (hi < lo: none)
  long long blk[3];   // first face id of each direction block
  long long side[6];  // first face id of each boundary side (boundary buffer)
  long long nfaces;   // unknown faces
  long long nbfaces;  // boundary faces
  int uniform;        // all elements have the same widths
};

// Per right-hand-side scalars of the (preconditioned) CG, device resident.
struct CgScalars {
  double rr;        // gamma = r . u of the current iterate (u = W r)
  double rr_old;    // gamma of the previous iterate
  double rr_stop;   // stop when rr <= rr_stop
  double alpha, beta;   // step length and direction update of the current step
  int it, max_it;   // completed update steps, cap
  int ops;          // operator launches whose scalars are done
  int done;         // 1: stop (converged, iteration cap or breakdown)
  int status;       // 0 ok / converged, 5 not converged, 6 breakdown
};

// 1D tables of one degree in the transformed basis (Alg. hdg_op_3d_transformed):
// c[m] = B_S[m][0] (B_S[m][1] = sigma_m c[m], sigma = +1 for m < n_even),
// lam[m] = Lambda_m, and H = [[h0, h1], [h1, h0]] = G + C^T M^-1 C.
template <typename T>
struct Tables {
  T c[kMaxNDev];
  T lam[kMaxNDev];   // Lambda_m (used when D_Z^-1 is computed in the kernel)
  T h0, h1;
};

// Compile-time loop: f(std::integral_constant<int, I>) for I = B..E-1, so the
// body sees its index as a constant expression (constant-bank operands,
// register-resident arrays, no loop control).
template <int B, int E, typename F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    static_for<B + 1, E>(f);
  }
}

// 16-byte vector type per arithmetic type and the padded row length used by
// the operator's shared-memory arrays and by the D_Z^-1 tables: rows of n
// values are padded to a multiple of the vector width so that a row can be
// read with 16-byte accesses.
template <typename T>
struct Vec;
template <>
struct Vec<float> {
  using type = float4;
  static constexpr int L = 4;
};
template <>
struct Vec<double> {
  using type = double2;
  static constexpr int L = 2;
};
__host__ __device__ constexpr int dz_row(int n, int elem_bytes) {
  return elem_bytes == 4 ? (n + 3) / 4 * 4 : (n + 1) / 2 * 2;
}
__device__ __forceinline__ float vget(const float4& v, int l) { return l == 0 ? v.x : l == 1 ? v.y : l == 2 ? v.z : v.w; }
__device__ __forceinline__ double vget(const double2& v, int l) { return l == 0 ? v.x : v.y; }
__device__ __forceinline__ void vset(float4& v, int l, float x) {
  if (l == 0) v.x = x; else if (l == 1) v.y = x; else if (l == 2) v.z = x; else v.w = x;
}
__device__ __forceinline__ void vset(double2& v, int l, double x) {
  if (l == 0) v.x = x; else v.y = x;
}

// n x n matrix passed by value (row-major).
template <typename T>
struct Mat1D {
  T a[kMaxNDev * kMaxNDev];
};

// 1 / x for the in-kernel D_Z^-1: the hardware reciprocal approximation in
// FP32 (relative error ~2^-22, below the FP32 rounding of the operator
// itself); exact division in FP64.
__device__ __forceinline__ float dz_recip(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double dz_recip(double x) { return 1.0 / x; }

// ---- storage conversions --------------------------------------------------
template <typename ST, typename T>
__device__ __forceinline__ T load_as(const ST* p) { return static_cast<T>(*p); }
template <>
__device__ __forceinline__ float load_as<__nv_bfloat16, float>(const __nv_bfloat16* p) {
  return __bfloat162float(*p);
}
template <typename ST, typename T>
__device__ __forceinline__ void store_from(ST* p, T v) { *p = static_cast<ST>(v); }
template <>
__device__ __forceinline__ void store_from<__nv_bfloat16, float>(__nv_bfloat16* p, float v) {
  *p = __float2bfloat16_rn(v);
}

// Programmatic dependent launch (sm_90+): a kernel launched with
// programmatic stream serialization may start while the previous kernel in
// the stream is still finishing; grid_dep_wait() blocks until that kernel
// has completed and its memory operations are visible (a no-op without such
// a dependency), and grid_dep_launch() lets the next kernel's blocks be
// scheduled once every block of this grid has signalled or exited.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
// Cache hint: bring the line holding *p into L1 (p must be a valid global
// address); no register is written.
__device__ __forceinline__ void prefetch_l1(const void* p) { asm volatile("prefetch.global.L1 [%0];" ::"l"(p)); }

// y += v with a single global reduction (L2 atomic).  Exactly two adds reach
// an interior face value that starts at zero: 0 + a + b == 0 + b + a in IEEE
// arithmetic, so the result does not depend on their order.
__device__ __forceinline__ void red_add(double* p, double v) {
  asm volatile("red.global.add.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}
__device__ __forceinline__ void red_add(float* p, float v) {
  asm volatile("red.global.add.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}
__device__ __forceinline__ void red_add(__nv_bfloat16* p, float v) {
  atomicAdd(p, __float2bfloat16_rn(v));
}
// Stores under a predicate (no branch around them); p is not dereferenced
// when `on` is false.
__device__ __forceinline__ void st_if(bool on, double* p, double v) {
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %0, 0;\n\t@q st.global.f64 [%1], %2;\n\t}"
               ::"r"((int)on), "l"(p), "d"(v) : "memory");
}
__device__ __forceinline__ void st_if(bool on, float* p, float v) {
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %0, 0;\n\t@q st.global.f32 [%1], %2;\n\t}"
               ::"r"((int)on), "l"(p), "f"(v) : "memory");
}
__device__ __forceinline__ void st_if(bool on, __nv_bfloat16* p, float v) {
  const unsigned short b = __bfloat16_as_ushort(__float2bfloat16_rn(v));
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %0, 0;\n\t@q st.global.b16 [%1], %2;\n\t}"
               ::"r"((int)on), "l"(p), "h"(b) : "memory");
}
// The same reductions under a predicate (no branch around them): the add is
// issued only when `on`; p is not dereferenced otherwise.
__device__ __forceinline__ void red_add_if(bool on, double* p, double v) {
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %0, 0;\n\t@q red.global.add.f64 [%1], %2;\n\t}"
               ::"r"((int)on), "l"(p), "d"(v) : "memory");
}
__device__ __forceinline__ void red_add_if(bool on, float* p, float v) {
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %0, 0;\n\t@q red.global.add.f32 [%1], %2;\n\t}"
               ::"r"((int)on), "l"(p), "f"(v) : "memory");
}
__device__ __forceinline__ void red_add_if(bool on, __nv_bfloat16* p, float v) {
  const unsigned short b = __bfloat16_as_ushort(__float2bfloat16_rn(v));
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %0, 0;\n\t@q red.global.add.noftz.bf16 [%1], %2;\n\t}"
               ::"r"((int)on), "l"(p), "h"(b) : "memory");
}

}  // namespace hdg
