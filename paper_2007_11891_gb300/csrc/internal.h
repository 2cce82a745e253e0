// Host-side launchers shared between the translation units of the library.
#pragma once

#include <cuda_runtime.h>

#include "../../include/hdg.h"

#include "common.cuh"
#include "tpt_kernel.cuh"

namespace hdg {

// ---- condensed operator (tpt_*.cu) -----------------------------------------
// Launches tpt_kernel<T, ST, n, mode> over all x1-pencils for nrhs right-hand
// sides.  The caller zeroes the x2/x3 blocks of the output first (APPLY, RHS).
template <typename T, typename ST>
cudaError_t launch_tpt(int mode, int n, TptArgs<T, ST> a, int nrhs, cudaStream_t s);

// launch geometry for degree n: segments per block (ppb), threads per block,
// and the pencil split: `seg` elements per segment, `nseg` segments per
// x1-pencil, chosen so that nrhs x ne[1] x ne[2] x nseg slots fill the GPU
int tpt_ppb(int n);
int tpt_threads(int n, int ppb);
long long tpt_blocks(long long nslots, int ppb);
void tpt_split(int n, const int ne[3], int nrhs, int ctas, int ppb, int* seg, int* nseg);
// resident CTAs per SM of tpt_kernel<T, ST, n, mode> at ppb slots per CTA
template <typename T, typename ST>
int tpt_blocks_per_sm(int mode, int n, int ppb);
// CTAs per SM of the FP32 element-run kernel with the fused CG step
int fast_fused_blocks_per_sm(int n, int ppb);
// any mode for degrees above the specialised kernels (tpt_generic.cuh):
// D_Z^-1 computed in the kernel, a.dinv ignored
template <typename T>
cudaError_t launch_generic(int mode, int n, const TptArgs<T, T>& a, int nrhs, cudaStream_t s);
constexpr int kMaxSpecialisedN = 17;
// the apply with the tile kernel (tpt_tile.cuh), per storage precision
cudaError_t launch_tile_f32(int n, const TptArgs<float, float>& a, int nrhs, cudaStream_t s);
cudaError_t launch_tile_f64(int n, const TptArgs<double, double>& a, int nrhs, cudaStream_t s);
cudaError_t launch_tile_bf16(int n, const TptArgs<float, __nv_bfloat16>& a, int nrhs, cudaStream_t s);

// ---- tp_nodal.cu: nodal-basis operator in one kernel (Alg. hdg_op_3d) ------
struct NodalArgs {
  MeshDev mesh;
  Tables<double> tab;
  Mat1D<double> StM;            // S^T M, [mode][node]
  Mat1D<double> MS;             // M S, [node][mode]
  const double* metric;         // d0..d3 per element (one set when uniform)
  const double* dinv;           // D_Z^-1 table [rhs][class][k][j][i] (padded rows), or null
  long long dinv_rhs_stride;
  const double* lam;            // per right-hand side lambda (device; when dinv is null)
  const double* x;              // nodal unknown-face inputs
  double* y;                    // nodal unknown-face outputs, zeroed by the caller
  long long trace_stride;
  int epb;                      // elements per CTA (set by the launcher)
};
// y = K x in the nodal basis for nrhs right-hand sides, y zeroed beforehand
cudaError_t launch_tp_nodal(int n, const NodalArgs& a, int nrhs, cudaStream_t s);

// ---- lowdim.cu: 1D (Alg. hdg_op_1d) and 2D condensed operators ----------------
struct LowDimArgs {
  int dim;                      // 1 or 2
  int n;                        // p + 1
  int ne[2];                    // elements per direction (ne[1] = 1 when dim = 1)
  int lo[2], hi[2];             // unknown planes per direction
  long long blk[2];             // first face id of each direction block
  Tables<double> tab;
  Mat1D<double> StM, MS;        // face transforms (2D nodal basis)
  const double* metric;         // d0, d1, d2, 0 per element
  const double* lam;            // per right-hand side lambda (device)
  const double* x;              // unknown-face inputs
  double* y;                    // unknown-face outputs, zeroed by the caller
  long long trace_stride;
  int nodal;                    // 2D: inputs and outputs in the nodal basis
  int epb;                      // elements per CTA (set by the launcher)
};
cudaError_t launch_lowdim(const LowDimArgs& a, int nrhs, cudaStream_t s);

// ---- kernels.cu ---------------------------------------------------------------
// y_f = scale (W (x) W) x_f for every face f (n x n nodes, lower axis fastest),
// optionally y_f += ...;  nfaces faces per right-hand side, strides in values.
template <typename TI, typename TO>
cudaError_t launch_face_transform(int n, const TI* x, TO* y, long long nfaces, int nrhs,
                                  long long stride_x, long long stride_y, const Mat1D<double>& W,
                                  double scale, int accumulate, cudaStream_t s);

// y_e = scale_e (A (x) A (x) A) x_e per element (n^3 values, x1 fastest);
// scale_e = metric[4 e + 0] (d0) if use_d0, else 1.
cudaError_t launch_volume_transform(int n, const double* x, double* y, long long nelem, int nrhs,
                                    long long stride, const Mat1D<double>& A, const double* metric,
                                    int uniform, int use_d0, cudaStream_t s);

// D_Z^-1 tables: out[r][cls][i + n j + n^2 k] = 1 / (lam_r d0 + d1 L_i + d2 L_j + d3 L_k)
template <typename T>
cudaError_t launch_dinv(int n, const double* lambda_dev, int nrhs, const double* metric,
                        long long nclass, const double* Lambda_dev, T* out, cudaStream_t s);

// F-hat[unknown Neumann face] += (h_a h_b / 4) g-hat[boundary face]
cudaError_t launch_neumann_add(const MeshDev& m, int n, const double* widths_dev /*3 x maxN*/,
                               int wstride, const double* ghat, double* F, int nrhs,
                               long long bstride, long long tstride, cudaStream_t s);

// element-wise vector helpers over nrhs blocks of length len (stride = len)
template <typename TI, typename TO>
cudaError_t launch_convert(const TI* x, TO* y, long long count, cudaStream_t s);
cudaError_t launch_sub(const double* a, const double* b, double* out, long long count, cudaStream_t s);  // out = a - b
template <typename T>
cudaError_t launch_add_to(double* x, const T* d, long long count, cudaStream_t s);  // x += d
// per right-hand side r (vectors of length len): y[r] = (float)(scale[r] x[r]),
// and x[r] += inv_scale[r] d[r]; scale, inv_scale (device, nrhs) hold powers
// of two
cudaError_t launch_scale_convert(const double* x, float* y, long long len, int nrhs, const double* scale,
                                 cudaStream_t s);
cudaError_t launch_add_unscaled(double* x, const float* d, long long len, int nrhs, const double* inv_scale,
                                cudaStream_t s);

// deterministic dot products sum_i a_i b_i (w_i) per right-hand side into
// out[r]; w may be null (partials[nrhs * blocks], counter[nrhs] zero on
// entry and exit)
template <typename T>
cudaError_t launch_dot(const T* a, const T* b, const T* w, long long len, int nrhs, double* partials,
                       unsigned int* counter, double* out, int blocks, cudaStream_t s);

// face-block Jacobi preconditioner: diag (zeroed by the caller) += the face
// self-coupling of K-hat; then w = 1 / diag in FP64 and FP32
// (dinv null: D_Z^-1 computed from lam[r], the metric and tab.lam)
cudaError_t launch_pc_diag(const MeshDev& m, int n, const Tables<double>& tab, const double* metric,
                           const double* dinv, long long dinv_rhs_stride, const double* lam, double* diag,
                           int nrhs, long long tstride, cudaStream_t s);
cudaError_t launch_pc_invert(const double* diag, double* w64, float* w32, long long count, cudaStream_t s);

// ---- CG (cg_kernels in kernels.cu) ----------------------------------------------
// init: rr from dot result, rr_stop = tol[r]^2 rr, done if rr == 0 (or if
// the right-hand side is already masked in `flags`); flags[r] mirrors done.
cudaError_t launch_cg_init(CgScalars* cg, int* flags, const double* rr, const double* tol, int max_it,
                           int nrhs, cudaStream_t s);
// One step of the single-reduction CG (Chronopoulos-Gear) after the operator
// launch w = K u whose hook produced the step scalars (cg_scalars): updates
// p, s, x, r, u = W r (W = I if null), zeroes w, and leaves the per-block
// partial sums of gamma = r . u in partials[r][block] for the next operator
// launch.  Skips right-hand sides with flags[r] set.  `blocks` from
// cg_step_blocks (one resident wave).  pdl: programmatic dependent launch on
// the operator launch before it.
template <typename T>
int cg_step_blocks(long long len);
template <typename T>
cudaError_t launch_cg_step(const CgScalars* cg, const int* flags, T* x, T* r, T* u, T* w, T* p, T* sv,
                           const T* W, long long len, int nrhs, double* partials, int blocks, bool pdl,
                           cudaStream_t s);
// p = W r + beta p (skips finished right-hand sides)
template <typename T>
cudaError_t launch_cg_pupdate(const CgScalars* cg, T* p, const T* r, const T* w, long long len, int nrhs,
                              cudaStream_t s);

// ---- read-only view of a context's device tables (hdg_api.cu) ----------------
struct CtxView {
  int device = 0;
  int sms = 1;
  int n = 0;
  int uniform = 1;
  MeshDev mesh{};
  Tables<double> tab{};
  const double* metric64 = nullptr;
  const double* Lambda = nullptr;
  Mat1D<double> StM{}, MS{};
  long long nelem = 0, ntrace = 0, nclass = 0;
};

}  // namespace hdg

struct hdg_ctx;
namespace hdg {
bool ctx_view(const hdg_ctx* c, CtxView* out);
void set_last_error(const char* msg);
// entry-point prologue of every C ABI call: clears the previous message and
// takes a CUDA error left pending by earlier work out of the runtime's slot
// (quoted in this call's message if it fails)
void begin_entry();
// lambda_r finite and >= 0 for r < nrhs (INVALID_ARG and a message otherwise)
hdg_status check_lambdas(int nrhs, const double* lam);
}  // namespace hdg
