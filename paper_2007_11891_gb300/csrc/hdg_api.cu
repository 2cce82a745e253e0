// C ABI of the condensed HDG library: context set-up, operator application,
// solve (transformed CG inside FP64 iterative refinement), recovery, adjoint.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/hdg.h"
#include "internal.h"
#include "setup1d.h"

namespace {

thread_local std::string g_last_error;
// a (non-sticky) CUDA error that was already pending when the current entry
// point started: cleared at entry so that it is not blamed on this call's
// own launches, and quoted if this call fails
thread_local std::string g_pending;

hdg_status fail(hdg_status s, const std::string& msg) {
  g_last_error = g_pending.empty() ? msg : msg + " [CUDA error pending before this call: " + g_pending + "]";
  return s;
}

// Entry-point prologue: clear the message of the previous call and take any
// pending CUDA error out of the runtime's error slot.
void begin_call() {
  g_last_error.clear();
  g_pending.clear();
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) g_pending = cudaGetErrorString(e);
}

#define HDG_CUDA(...)                                                                   \
  do {                                                                                  \
    cudaError_t e_ = (__VA_ARGS__);                                                     \
    if (e_ != cudaSuccess)                                                              \
      return fail(e_ == cudaErrorMemoryAllocation ? HDG_ERR_OOM : HDG_ERR_CUDA,         \
                  std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(e_));           \
  } while (0)

#define HDG_TRY(...)                \
  do {                              \
    hdg_status s_ = (__VA_ARGS__);  \
    if (s_ != HDG_OK) return s_;    \
  } while (0)

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

}  // namespace

struct hdg_ctx {
  int device = 0;
  int sms = 1;            // streaming multiprocessors of the device
  int p = 0, n = 0;
  hdg::Setup1D s1;
  hdg::MeshDev mesh{};
  std::vector<double> widths[3];
  int bc[6] = {0, 0, 0, 0, 0, 0};
  long long nelem = 0, ntrace = 0, nvol = 0, nbdry = 0;
  int uniform = 1;
  int has_dirichlet = 0, has_neumann = 0;
  double* d_metric64 = nullptr;
  float* d_metric32 = nullptr;
  double* d_Lambda = nullptr;
  double* d_widths = nullptr;
  int wstride = 0;
  hdg::Tables<double> tab64;
  hdg::Tables<float> tab32;
  hdg::Mat1D<double> StM, MS, S, St, M;
  // D_Z^-1 tables for the lambdas of the last call, per precision
  std::vector<double> lam64, lam32;
  DevBuf dinv64, dinv32, lam_dev64, lam_dev32;
  // workspaces
  DevBuf ws[24];
  DevBuf partials, counters, cgs, flags, scal;
  DevBuf step_partials;   // per-block gamma partials of the CG update step
  int red_blocks = 0;
  // measurement: launch count and optional event pairs per kernel class
  bool prof_on = false;
  long long launches = 0;
  std::vector<cudaEvent_t> ev[6];
  size_t ev_used[6] = {0, 0, 0, 0, 0, 0};
  // preconditioner for the lambdas of the last call
  std::vector<double> pc_lam;
  DevBuf pc_diag, pc_w64, pc_w32;
  // CUDA graphs of the inner CG loop
  struct GraphEntry {
    std::vector<uintptr_t> key;
    cudaGraphExec_t exec;
  };
  std::vector<GraphEntry> graphs;
  cudaStream_t cap_stream = nullptr;
  bool capturing = false;
  int graphs_enabled = 1;
  int loop_graphs_enabled = 1;
  // programmatic dependent launch between the CG loop kernels (dropped if a
  // graph with it cannot be built)
  int pdl = 1;
  DevBuf loopctl;   // device loop-trip counter of the CG loop graph
  int seg_override = 0;   // x1 segment length; 0 = automatic
  int ppb_override = 0;   // slots per CTA; 0 = automatic
  int op_variant = 0;     // apply kernel: 0 automatic (use_tiles), 1 element runs, 2 element tiles, 3 runtime degree
  int nodal_variant = 0;  // FP64 nodal apply: 0 face-wise transforms + transformed kernel, 1 one kernel (HDG-TP)
  int dz_mode = 0;        // FP32 D_Z^-1 source: 0 automatic, 1 table, 2 in kernel
  int fused_cg = 0;       // the current inner CG runs the fused step
  int fused_enabled = 0;  // allow the fused step (hdg_set_cg_variant)
  int persist_enabled = 0;  // run the fused step as one persistent cooperative launch
};

namespace {

enum Ws {
  W_XHAT = 0, W_YHAT, W_FHAT_T, W_RHAT, W_TMP, W_FVOL, W_GHAT, W_WVOL,
  W_R, W_D, W_P, W_Q, W_DOT, W_DOT2, W_U, W_S,
  // fused CG step (tile kernel): second r and s buffers, second and third w
  // buffers, per-block gamma partials; persistent CG: per-block delta
  // partials and the grid-barrier words
  W_R2, W_S2, W_W2, W_W3, W_GP, W_DP, W_BAR
};

hdg_status ensure(DevBuf& b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.bytes >= bytes) return HDG_OK;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e != cudaSuccess) {
    b.p = nullptr;
    return fail(HDG_ERR_OOM, std::string("cudaMalloc workspace: ") + cudaGetErrorString(e));
  }
  b.bytes = bytes;
  return HDG_OK;
}

template <typename T>
T* wsp(hdg_ctx* c, int i) { return static_cast<T*>(c->ws[i].p); }

using GraphEntry = hdg_ctx::GraphEntry;

enum KernelClass { K_OP32 = 0, K_OP64 = 1, K_FACE = 2, K_VOL = 3, K_RHS = 4, K_VEC = 5 };

// Counts a launch and, while profiling, brackets it with an event pair.
struct Timed {
  hdg_ctx* c;
  int cls;
  cudaStream_t s;
  long long idx = -1;
  Timed(hdg_ctx* c_, int cls_, cudaStream_t s_) : c(c_), cls(cls_), s(s_) {
    if (c->capturing) return;   // counted when the graph is launched
    c->launches += 1;
    if (!c->prof_on) return;
    std::vector<cudaEvent_t>& v = c->ev[cls];
    if (2 * c->ev_used[cls] + 2 > v.size()) {
      cudaEvent_t a, b;
      if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return;
      v.push_back(a);
      v.push_back(b);
    }
    idx = (long long)c->ev_used[cls]++;
    cudaEventRecord(v[2 * idx], s);
  }
  ~Timed() {
    if (idx >= 0) cudaEventRecord(c->ev[cls][2 * idx + 1], s);
  }
};

template <typename T>
const T* metric_ptr(const hdg_ctx* c);
template <>
const double* metric_ptr<double>(const hdg_ctx* c) { return c->d_metric64; }
template <>
const float* metric_ptr<float>(const hdg_ctx* c) { return c->d_metric32; }

template <typename T>
const hdg::Tables<T>& tables(const hdg_ctx* c);
template <>
const hdg::Tables<double>& tables<double>(const hdg_ctx* c) { return c->tab64; }
template <>
const hdg::Tables<float>& tables<float>(const hdg_ctx* c) { return c->tab32; }

long long nclass(const hdg_ctx* c) { return c->uniform ? 1 : c->nelem; }
// entries of one D_Z^-1 table (n^2 rows of the padded row length)
template <typename T>
long long dz_table(const hdg_ctx* c) { return (long long)c->n * c->n * hdg::dz_row(c->n, sizeof(T)); }

// D_Z^-1 is computed inside the FP32 operator kernel on stretched grids (one
// table per element would be n^3 values per element, more bytes than the
// element's share of the traces, for a reciprocal the SFU computes at no
// measurable cost); FP64 kernels (bound by the FP64 pipe, where a division
// costs more than a load) and uniform grids (one small table, held in
// shared memory) read tables.
template <typename T>
bool dz_in_kernel(const hdg_ctx* c) {
  // above the specialised degrees the generic kernels compute D_Z^-1 (n^3
  // values per element class and lambda would be too large to keep)
  if (c->n > hdg::kMaxSpecialisedN) return true;
  if (sizeof(T) != 4) return false;
  // the FP32 kernels index tables with 32-bit offsets
  if ((size_t)nclass(c) * dz_table<T>(c) >= (size_t(1) << 31)) return true;
  if (c->dz_mode == 1) return false;
  if (c->dz_mode == 2) return true;
  return !c->uniform;
}

// lambdas on the device, per precision (kept while they do not change)
template <typename T>
DevBuf& lam_buf(hdg_ctx* c) { return sizeof(T) == 8 ? c->lam_dev64 : c->lam_dev32; }

// D_Z^-1 tables for the given lambdas (rebuilt when they change); *out is
// null when the kernel computes D_Z^-1 itself.
template <typename T>
hdg_status ensure_dinv(hdg_ctx* c, int nrhs, const double* lam, cudaStream_t s, const T** out) {
  std::vector<double>& cur = sizeof(T) == 8 ? c->lam64 : c->lam32;
  DevBuf& buf = sizeof(T) == 8 ? c->dinv64 : c->dinv32;
  DevBuf& lb = lam_buf<T>(c);
  std::vector<double> want(lam, lam + nrhs);
  if (cur != want) {
    HDG_TRY(ensure(lb, sizeof(double) * nrhs));
    HDG_CUDA(cudaMemcpyAsync(lb.p, lam, sizeof(double) * nrhs, cudaMemcpyHostToDevice, s));
    if (!dz_in_kernel<T>(c)) {
      HDG_TRY(ensure(buf, sizeof(T) * (size_t)nrhs * nclass(c) * dz_table<T>(c)));
      HDG_CUDA(hdg::launch_dinv<T>(c->n, static_cast<double*>(lb.p), nrhs, c->d_metric64, nclass(c),
                                   c->d_Lambda, static_cast<T*>(buf.p), s));
    }
    // the host lambda array may change after return: finish the copy first
    HDG_CUDA(cudaStreamSynchronize(s));
    cur = want;
  }
  *out = dz_in_kernel<T>(c) ? nullptr : static_cast<const T*>(buf.p);
  return HDG_OK;
}

// Whether the apply of arithmetic T / storage ST with nrhs right-hand sides
// runs the element-tile kernel.  Automatic choice, from apply and solve
// timings on this part (32^3 applies at p = 2..16; solves on 8^3..32^3
// meshes, single and batched): BF16 storage: tiles (1.4-1.6x faster);
// FP32: tiles at n = 10 and 12..16, where the element-run slots are packed
// (n = 10) or the tile rows are padded conflict-free (up to 1.6x faster at
// p = 13), element runs at the other degrees (shorter per-element latency,
// 5-40 % faster); FP64: tiles for one right-hand side (3-15 % faster at
// 16^3 and 32^3), element runs for batches (12 % faster at 16 rhs).
template <typename T, typename ST>
bool use_tiles(const hdg_ctx* c, int nrhs) {
  if (c->op_variant == 1 || c->op_variant == 3) return false;
  if (c->op_variant == 2) return true;
  if (sizeof(ST) == 2) return true;
  if (sizeof(T) == 8) return nrhs <= 1;
  return c->n == 10 || (c->n >= 12 && c->n <= 16);
}

template <typename T, typename ST>
hdg::TptArgs<T, ST> base_args(const hdg_ctx* c, const T* dinv, int nrhs, int mode = hdg::TPT_APPLY) {
  hdg::TptArgs<T, ST> a{};
  a.mesh = c->mesh;
  a.tab = tables<T>(c);
  a.metric = metric_ptr<T>(c);
  a.dinv = dinv;
  a.dinv_rhs_stride = nclass(c) * dz_table<T>(c);
  a.lam = static_cast<const double*>(lam_buf<T>(const_cast<hdg_ctx*>(c)).p);
  a.trace_stride = c->ntrace;
  a.bdry_stride = c->nbdry;
  a.vol_stride = c->nvol;
  a.ppb = c->ppb_override > 0 ? c->ppb_override : hdg::tpt_ppb(c->n);
  a.npencils = (long long)c->mesh.ne[1] * c->mesh.ne[2];
  // persistent grid: one resident wave of CTAs, each CTA looping over slot groups
  int ctas = c->sms * hdg::tpt_blocks_per_sm<T, ST>(mode, c->n, a.ppb);
  hdg::tpt_split(c->n, c->mesh.ne, nrhs, ctas, a.ppb, &a.seg, &a.nseg);
  if (c->seg_override > 0) {
    a.seg = std::min(c->seg_override, c->mesh.ne[0]);
    a.nseg = (c->mesh.ne[0] + a.seg - 1) / a.seg;
  }
  a.max_grid = ctas;
  a.sms = c->sms;
  a.tile = c->seg_override;   // elements per tile of the tile kernel (0 = automatic)
  // apply kernel: element tiles (tpt_tile.cuh) or element runs (use_tiles)
  if (mode == hdg::TPT_APPLY && use_tiles<T, ST>(c, nrhs)) a.variant = 3;
  if (c->op_variant == 3) a.variant = 4;   // runtime-degree kernel, every mode
  // FP32 apply: equal contiguous runs, one per slot of a resident wave (per
  // right-hand side: the wave is shared by the batch)
  const long long nelem = (long long)c->nelem * std::max(nrhs, 1);
  const long long slots = std::max(1LL, (long long)ctas * a.ppb);
  a.chunk = c->seg_override > 0 ? c->seg_override : (int)std::max(1LL, (nelem + slots - 1) / slots);
  return a;
}

// The kernel of `a` adds into every face of the output (the FP32 kernels,
// the tiles, the runtime-degree kernel), not only the x2/x3 blocks.
template <typename T, typename ST>
bool full_zero(const hdg_ctx* c, const hdg::TptArgs<T, ST>& a) {
  return sizeof(T) == 4 || a.variant >= 3 || c->n > hdg::kMaxSpecialisedN;
}

// Zero what the operator accumulates with atomics: the x2/x3 blocks, and the
// whole vector when x1-pencils are split into several segments.
template <typename ST>
hdg_status zero_for_tpt(const hdg_ctx* c, ST* y, int nrhs, int nseg, cudaStream_t s) {
  const long long off = nseg > 1 ? 0 : c->mesh.blk[1] * (long long)c->n * c->n;
  const long long cnt = c->ntrace - off;
  if (cnt <= 0) return HDG_OK;
  HDG_CUDA(cudaMemset2DAsync(y + off, sizeof(ST) * c->ntrace, 0, sizeof(ST) * cnt, nrhs, s));
  return HDG_OK;
}

// y = K-hat x; `zeroed` says the caller already zeroed y (the CG update does)
template <typename T, typename ST>
hdg_status tpt_apply(hdg_ctx* c, int nrhs, const T* dinv, const ST* x, ST* y, cudaStream_t s,
                     const int* skip = nullptr, hdg::CgHook hook = hdg::CgHook{}, bool zeroed = false,
                     bool pdl = false) {
  hdg::TptArgs<T, ST> a = base_args<T, ST>(c, dinv, nrhs);
  // the FP32 kernel's runs may split any x1-pencil: zero the whole output
  if (!zeroed) HDG_TRY(zero_for_tpt<ST>(c, y, nrhs, full_zero(c, a) ? 2 : a.nseg, s));
  a.x = x;
  a.y = y;
  a.skip = skip;
  a.hook = hook;
  a.pdl = pdl ? 1 : 0;
  Timed t(c, sizeof(T) == 8 ? K_OP64 : K_OP32, s);
  const cudaError_t e = hdg::launch_tpt<T, ST>(hdg::TPT_APPLY, c->n, a, nrhs, s);
  if (e != cudaSuccess)
    return fail(HDG_ERR_CUDA, std::string("operator launch (") + (sizeof(T) == 8 ? "FP64" : "FP32") +
                                  ", n=" + std::to_string(c->n) + ", slots=" + std::to_string(a.ppb) +
                                  ", seg=" + std::to_string(a.seg) + "x" + std::to_string(a.nseg) +
                                  ", run=" + std::to_string(a.chunk) + ", grid cap=" + std::to_string(a.max_grid) +
                                  ", nrhs=" + std::to_string(nrhs) + "): " + cudaGetErrorString(e));
  return HDG_OK;
}

// Nodal-basis FP64 apply in one kernel (Alg. hdg_op_3d): no workspace; the
// output is zeroed and receives the element contributions by atomic adds
hdg_status nodal_apply(hdg_ctx* c, int nrhs, const double* dinv, const double* x, double* y, cudaStream_t s) {
  hdg::NodalArgs a{};
  a.mesh = c->mesh;
  a.tab = tables<double>(c);
  a.StM = c->StM;
  a.MS = c->MS;
  a.metric = metric_ptr<double>(c);
  a.dinv = dinv;
  a.dinv_rhs_stride = nclass(c) * dz_table<double>(c);
  a.lam = static_cast<const double*>(lam_buf<double>(c).p);
  a.x = x;
  a.y = y;
  a.trace_stride = c->ntrace;
  HDG_CUDA(cudaMemsetAsync(y, 0, sizeof(double) * (size_t)c->ntrace * nrhs, s));
  Timed t(c, K_OP64, s);
  const cudaError_t e = hdg::launch_tp_nodal(c->n, a, nrhs, s);
  if (e != cudaSuccess)
    return fail(HDG_ERR_CUDA, std::string("nodal operator launch (n=") + std::to_string(c->n) +
                                  ", nrhs=" + std::to_string(nrhs) + "): " + cudaGetErrorString(e));
  return HDG_OK;
}

hdg_status check_lambda(const hdg_ctx* c, int nrhs, const double* lam) {
  if (!lam) return fail(HDG_ERR_INVALID_ARG, "lambda pointer is NULL");
  for (int r = 0; r < nrhs; ++r)
    if (!(lam[r] >= 0.0) || !std::isfinite(lam[r])) return fail(HDG_ERR_INVALID_ARG, "lambda must be finite and >= 0");
  (void)c;
  return HDG_OK;
}

int reduction_blocks(long long len) {
  long long b = (len + 255) / 256;
  return (int)std::max(1LL, std::min(b, 152LL * 4));
}

hdg_status ensure_reductions(hdg_ctx* c, int nrhs) {
  c->red_blocks = std::max(c->sms, 152) * 8;   // upper bound on blocks of any reducing vector launch (8 x 256 threads per SM)
  // the operator grid is largest with one element per CTA (one slot, runs of one)
  const long long tpt_b = c->nelem;
  const long long pb = std::max<long long>(c->red_blocks, tpt_b);
  HDG_TRY(ensure(c->partials, sizeof(double) * (size_t)nrhs * pb));
  HDG_TRY(ensure(c->step_partials, sizeof(double) * (size_t)nrhs * c->red_blocks));
  const bool fresh = c->counters.bytes < sizeof(unsigned int) * (size_t)nrhs;
  HDG_TRY(ensure(c->counters, sizeof(unsigned int) * (size_t)nrhs));
  if (fresh) HDG_CUDA(cudaMemset(c->counters.p, 0, c->counters.bytes));
  HDG_TRY(ensure(c->cgs, sizeof(hdg::CgScalars) * (size_t)nrhs));
  HDG_TRY(ensure(c->flags, sizeof(int) * (size_t)nrhs));
  HDG_TRY(ensure(c->scal, sizeof(double) * (size_t)nrhs * 5));   // rz0, pq, tol, FP32 inner-solve scale and inverse
  return HDG_OK;
}

template <typename T>
hdg_status dot(hdg_ctx* c, const T* a, const T* b, long long len, int nrhs, double* out, cudaStream_t s,
               const T* w = nullptr) {
  Timed t(c, K_VEC, s);
  HDG_CUDA(hdg::launch_dot<T>(a, b, w, len, nrhs, static_cast<double*>(c->partials.p),
                              static_cast<unsigned int*>(c->counters.p), out, reduction_blocks(len), s));
  return HDG_OK;
}

// Face-block Jacobi preconditioner (Sec. 5.1) for the lambdas of the call:
// inverse face self-coupling of K-hat, FP64 and FP32 copies.
hdg_status ensure_pc(hdg_ctx* c, int nrhs, const double* lam, cudaStream_t s) {
  std::vector<double> want(lam, lam + nrhs);
  if (c->pc_lam == want) return HDG_OK;
  const double* dinv = nullptr;
  HDG_TRY(ensure_dinv<double>(c, nrhs, lam, s, &dinv));
  const size_t tot = (size_t)c->ntrace * nrhs;
  HDG_TRY(ensure(c->pc_diag, sizeof(double) * tot));
  HDG_TRY(ensure(c->pc_w64, sizeof(double) * tot));
  HDG_TRY(ensure(c->pc_w32, sizeof(float) * tot));
  HDG_CUDA(cudaMemsetAsync(c->pc_diag.p, 0, sizeof(double) * tot, s));
  { Timed t_(c, K_VEC, s);
    HDG_CUDA(hdg::launch_pc_diag(c->mesh, c->n, c->tab64, c->d_metric64, dinv, nclass(c) * dz_table<double>(c),
                                 static_cast<const double*>(lam_buf<double>(c).p),
                                 static_cast<double*>(c->pc_diag.p), nrhs, c->ntrace, s)); }
  { Timed t_(c, K_VEC, s);
    HDG_CUDA(hdg::launch_pc_invert(static_cast<double*>(c->pc_diag.p), static_cast<double*>(c->pc_w64.p),
                                   static_cast<float*>(c->pc_w32.p), (long long)tot, s)); }
  c->pc_lam = want;
  return HDG_OK;
}

template <typename T>
const T* pc_weights(const hdg_ctx* c);
template <>
const double* pc_weights<double>(const hdg_ctx* c) { return static_cast<const double*>(c->pc_w64.p); }
template <>
const float* pc_weights<float>(const hdg_ctx* c) { return static_cast<const float*>(c->pc_w32.p); }

// Loop control of the device-driven inner CG: after every body trip, keep
// looping while any right-hand side is still active.  A trip cap derived
// from the iteration limits bounds the loop independently of the CG flags.
__global__ void cg_loop_cond(cudaGraphConditionalHandle h, const hdg::CgScalars* cg, const int* flags, int nrhs,
                             unsigned int* trips, int iters_per_trip) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const unsigned int t = ++(*trips);
  int any = 0, maxit = 0;
  for (int r = 0; r < nrhs; ++r) {
    any |= (flags[r] == 0);
    maxit = max(maxit, cg[r].max_it);
  }
  const unsigned int cap = (unsigned int)(maxit / iters_per_trip) + 2u;
  cudaGraphSetConditional(h, (any && t < cap) ? 1u : 0u);
}

// `count` iterations of the fused CG step, one operator launch each (the
// FP32 element-run kernel, tpt_fast.cuh, or the tile kernel, tpt_tile.cuh;
// CgVecs): launch j applies the update of iteration j - 1 to the face values
// it stages and applies the operator to u_j.  Buffers rotate with j: r and s
// with period 2, w with period 3, so every sequence of launches (eager or
// captured) starts at a multiple of kFusedPeriod.
constexpr int kFusedPeriod = 6;
template <typename T>
hdg_status cg_fused_iterations(hdg_ctx* c, int nrhs, const T* dinv, const T* Wt, int count, cudaStream_t s) {
  int* flags = static_cast<int*>(c->flags.p);
  hdg::CgScalars* cg = static_cast<hdg::CgScalars*>(c->cgs.p);
  double* uw = static_cast<double*>(c->scal.p) + nrhs;
  hdg::CgHook hook{static_cast<double*>(c->partials.p), static_cast<unsigned int*>(c->counters.p), uw, cg, flags,
                   nullptr, 0};
  T* R[2] = {wsp<T>(c, W_R), wsp<T>(c, W_R2)};
  T* S[2] = {wsp<T>(c, W_S), wsp<T>(c, W_S2)};
  T* Wb[3] = {wsp<T>(c, W_Q), wsp<T>(c, W_W2), wsp<T>(c, W_W3)};
  hdg::TptArgs<T, T> a = base_args<T, T>(c, dinv, nrhs);
  if (sizeof(T) == 4 && !use_tiles<T, T>(c, nrhs)) {
    // the element-run kernel: runs sized for its own occupancy with the
    // staging areas of the fused step
    a.variant = 0;
    const long long slots = std::max(1LL, (long long)c->sms * hdg::fast_fused_blocks_per_sm(c->n, a.ppb) * a.ppb);
    const long long nel = (long long)c->nelem * std::max(nrhs, 1);
    a.chunk = c->seg_override > 0 ? c->seg_override : (int)std::max(1LL, (nel + slots - 1) / slots);
  } else {
    a.variant = 3;
  }
  a.cg = 1;
  a.skip = flags;
  a.hook = hook;
  a.pdl = c->pdl ? 1 : 0;
  a.cgv.x = wsp<T>(c, W_D);
  a.cgv.p = wsp<T>(c, W_P);
  a.cgv.W = Wt;
  a.cgv.gpartials = wsp<double>(c, W_GP);
  for (int k = 0; k < count; ++k) {
    a.cgv.r_in = R[k % 2];
    a.cgv.r_out = R[(k + 1) % 2];
    a.cgv.s_in = S[k % 2];
    a.cgv.s_out = S[(k + 1) % 2];
    a.cgv.w_in = Wb[k % 3];
    a.y = Wb[(k + 1) % 3];
    a.cgv.w_zero = Wb[(k + 2) % 3];
    a.x = nullptr;
    Timed t(c, sizeof(T) == 8 ? K_OP64 : K_OP32, s);
    const cudaError_t e = hdg::launch_tpt<T, T>(hdg::TPT_APPLY, c->n, a, nrhs, s);
    if (e != cudaSuccess)
      return fail(HDG_ERR_CUDA, std::string("fused CG step launch (n=") + std::to_string(c->n) +
                                    ", nrhs=" + std::to_string(nrhs) + "): " + cudaGetErrorString(e));
  }
  return HDG_OK;
}

// The whole inner CG of the fused step in one cooperative launch of the tile
// kernel (CGM = 2): every CTA stays resident, one grid barrier per iteration.
// Returns false (nothing launched) if the device cannot run it, so that the
// caller runs the per-launch path.
template <typename T>
bool cg_persistent(hdg_ctx* c, int nrhs, const T* dinv, const T* Wt, cudaStream_t s, hdg_status* st) {
  *st = HDG_OK;
  if (!c->persist_enabled) return false;
  int coop = 0;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, c->device) != cudaSuccess || !coop) {
    cudaGetLastError();
    return false;
  }
  const size_t pb = (size_t)std::max<long long>(c->red_blocks, c->nelem);
  if (ensure(c->ws[W_DP], sizeof(double) * 2 * nrhs * pb) != HDG_OK ||
      ensure(c->ws[W_GP], sizeof(double) * 2 * nrhs * pb) != HDG_OK ||
      ensure(c->ws[W_BAR], sizeof(unsigned int) * (2 * (size_t)nrhs + 1)) != HDG_OK) {
    g_last_error.clear();
    return false;
  }
  unsigned int* bar = static_cast<unsigned int*>(c->ws[W_BAR].p);
  int* err = reinterpret_cast<int*>(bar + 2 * nrhs);
  if (cudaMemsetAsync(bar, 0, sizeof(unsigned int) * (2 * (size_t)nrhs + 1), s) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  int* flags = static_cast<int*>(c->flags.p);
  hdg::CgScalars* cg = static_cast<hdg::CgScalars*>(c->cgs.p);
  double* uw = static_cast<double*>(c->scal.p) + nrhs;
  hdg::TptArgs<T, T> a = base_args<T, T>(c, dinv, nrhs);
  a.variant = 3;
  a.cg = 2;
  a.skip = flags;
  a.hook = hdg::CgHook{wsp<double>(c, W_DP), static_cast<unsigned int*>(c->counters.p), uw, cg, flags, nullptr, 0};
  a.pdl = 0;
  a.x = nullptr;
  a.cgv.x = wsp<T>(c, W_D);
  a.cgv.p = wsp<T>(c, W_P);
  a.cgv.W = Wt;
  a.cgv.gpartials = wsp<double>(c, W_GP);
  a.cgv.bar = bar;
  a.cgv.err = err;
  a.cgv.r_in = wsp<T>(c, W_R);
  a.cgv.r_out = wsp<T>(c, W_R2);
  a.cgv.s_in = wsp<T>(c, W_S);
  a.cgv.s_out = wsp<T>(c, W_S2);
  a.cgv.w_in = wsp<T>(c, W_Q);
  a.y = wsp<T>(c, W_W2);
  a.cgv.w_zero = wsp<T>(c, W_W3);
  {
    Timed t(c, sizeof(T) == 8 ? K_OP64 : K_OP32, s);
    const cudaError_t e = hdg::launch_tpt<T, T>(hdg::TPT_APPLY, c->n, a, nrhs, s);
    if (e != cudaSuccess) {
      // e.g. a grid that cannot be co-resident: the per-launch path runs instead
      cudaGetLastError();
      c->persist_enabled = 0;
      return false;
    }
  }
  int herr = 0;
  cudaError_t e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    *st = fail(HDG_ERR_CUDA, std::string("persistent CG: ") + cudaGetErrorString(e));
    return true;
  }
  if (herr) *st = fail(HDG_ERR_CUDA, "persistent CG: a grid barrier timed out (CTAs not co-resident)");
  return true;
}

// `count` CG iterations: the fused step, or two kernels each: the operator
// w = K-hat u with the fused u^T w, then the single-reduction CG step
// (launch_cg_step).  Vectors: x (d), r, u = W r, w (q), p, s = K-hat p.
template <typename T>
hdg_status cg_iterations(hdg_ctx* c, int nrhs, const T* dinv, const T* w, T* r, T* d, T* p, T* q, int count,
                         cudaStream_t s) {
  if (c->fused_cg) return cg_fused_iterations<T>(c, nrhs, dinv, w, count, s);
  const long long T_ = c->ntrace;
  int* flags = static_cast<int*>(c->flags.p);
  hdg::CgScalars* cg = static_cast<hdg::CgScalars*>(c->cgs.p);
  double* uw = static_cast<double*>(c->scal.p) + nrhs;
  const int vb = hdg::cg_step_blocks<T>(T_);
  double* gp = static_cast<double*>(c->step_partials.p);
  hdg::CgHook hook{static_cast<double*>(c->partials.p), static_cast<unsigned int*>(c->counters.p), uw, cg, flags,
                   gp, vb};
  T* u = wsp<T>(c, W_U);
  T* sv = wsp<T>(c, W_S);
  // programmatic dependent launch: each loop kernel may be scheduled while
  // the previous one drains (the FP32 operator kernel and the update kernel
  // wait for their predecessor before reading anything it wrote; the FP64
  // operator kernel is launched normally)
  const bool pdl = c->pdl != 0;
  for (int k = 0; k < count; ++k) {
    HDG_TRY((tpt_apply<T, T>(c, nrhs, dinv, u, q, s, flags, hook, true, pdl && sizeof(T) == 4)));
    Timed t_(c, K_VEC, s);
    HDG_CUDA(hdg::launch_cg_step<T>(cg, flags, d, r, u, q, p, sv, w, T_, nrhs, gp, vb, pdl, s));
  }
  return HDG_OK;
}

// Replays `count` iterations from a CUDA graph captured once per
// configuration (pointers, nrhs, precision); returns false (and leaves
// graphs off) if capture is not possible, so the caller runs eagerly.
template <typename T>
bool cg_graph(hdg_ctx* c, int nrhs, const T* dinv, const T* w, T* r, T* d, T* p, T* q, int count,
              cudaStream_t s, hdg_status* st) {
  *st = HDG_OK;
  if (!c->graphs_enabled || c->prof_on) return false;
  std::vector<uintptr_t> key = {sizeof(T), (uintptr_t)nrhs, (uintptr_t)dinv, (uintptr_t)lam_buf<T>(c).p,
                                (uintptr_t)c->ws[W_U].p, (uintptr_t)c->ws[W_S].p, (uintptr_t)w, (uintptr_t)r,
                                (uintptr_t)d, (uintptr_t)p, (uintptr_t)q, (uintptr_t)c->flags.p,
                                (uintptr_t)c->cgs.p, (uintptr_t)c->scal.p, (uintptr_t)c->partials.p,
                                (uintptr_t)c->step_partials.p, (uintptr_t)c->counters.p, (uintptr_t)count,
                                (uintptr_t)c->pdl, (uintptr_t)c->seg_override,
                                (uintptr_t)c->ppb_override, (uintptr_t)c->dz_mode, (uintptr_t)c->fused_cg, (uintptr_t)c->op_variant,
                                (uintptr_t)c->ws[W_R2].p, (uintptr_t)c->ws[W_S2].p, (uintptr_t)c->ws[W_W2].p,
                                (uintptr_t)c->ws[W_W3].p, (uintptr_t)c->ws[W_GP].p};
  GraphEntry* ge = nullptr;
  for (GraphEntry& g : c->graphs)
    if (g.key == key) ge = &g;
  if (!ge) {
    if (!c->cap_stream && cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
      c->graphs_enabled = 0;
      return false;
    }
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      c->graphs_enabled = 0;
      cudaGetLastError();
      return false;
    }
    c->capturing = true;
    hdg_status cs = cg_iterations<T>(c, nrhs, dinv, w, r, d, p, q, count, c->cap_stream);
    c->capturing = false;
    cudaError_t e = cudaStreamEndCapture(c->cap_stream, &graph);
    cudaGraphExec_t exec = nullptr;
    if (cs != HDG_OK || e != cudaSuccess || graph == nullptr ||
        cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      c->graphs_enabled = 0;
      cudaGetLastError();
      g_last_error.clear();
      return false;
    }
    cudaGraphDestroy(graph);
    c->graphs.push_back(GraphEntry{key, exec});
    ge = &c->graphs.back();
  }
  cudaError_t e = cudaGraphLaunch(ge->exec, s);
  if (e != cudaSuccess) {
    *st = fail(HDG_ERR_CUDA, std::string("cudaGraphLaunch: ") + cudaGetErrorString(e));
    return true;
  }
  c->launches += (c->fused_cg ? 1LL : 2LL) * count;
  return true;
}

// The whole inner CG as one graph launch: a conditional WHILE node whose
// body runs `kTrip` iterations (kFusedPeriod with the fused step, whose
// buffers rotate with that period) and then the loop-control kernel.
// Returns false (graphs left to the chunked path) where the driver cannot
// build it.
template <typename T>
bool cg_loop_graph(hdg_ctx* c, int nrhs, const T* dinv, const T* w, T* r, T* d, T* p, T* q, cudaStream_t s,
                   hdg_status* st) {
  *st = HDG_OK;
  const int kTrip = c->fused_cg ? kFusedPeriod : 16;
  const long long per_iter = c->fused_cg ? 1 : 2;
  if (!c->loop_graphs_enabled || c->prof_on) return false;
  if (ensure(c->loopctl, sizeof(unsigned int) * 4) != HDG_OK) return false;
  std::vector<uintptr_t> key = {0xC0DEu, sizeof(T), (uintptr_t)nrhs, (uintptr_t)dinv, (uintptr_t)lam_buf<T>(c).p,
                                (uintptr_t)c->ws[W_U].p, (uintptr_t)c->ws[W_S].p,
                                (uintptr_t)w, (uintptr_t)r, (uintptr_t)d, (uintptr_t)p, (uintptr_t)q,
                                (uintptr_t)c->flags.p, (uintptr_t)c->cgs.p, (uintptr_t)c->scal.p,
                                (uintptr_t)c->partials.p, (uintptr_t)c->step_partials.p,
                                (uintptr_t)c->counters.p, (uintptr_t)c->loopctl.p,
                                (uintptr_t)c->seg_override, (uintptr_t)c->ppb_override, (uintptr_t)c->dz_mode,
                                (uintptr_t)c->pdl, (uintptr_t)c->fused_cg, (uintptr_t)c->op_variant, (uintptr_t)c->ws[W_R2].p,
                                (uintptr_t)c->ws[W_S2].p, (uintptr_t)c->ws[W_W2].p, (uintptr_t)c->ws[W_W3].p,
                                (uintptr_t)c->ws[W_GP].p};
  GraphEntry* ge = nullptr;
  for (GraphEntry& g : c->graphs)
    if (g.key == key) ge = &g;
  unsigned int* trips = static_cast<unsigned int*>(c->loopctl.p);
  if (!ge) {
    auto give_up = [&](cudaGraph_t g) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      g_last_error.clear();
      if (c->pdl) {
        // try once more without programmatic dependent launch
        c->pdl = 0;
        return cg_loop_graph<T>(c, nrhs, dinv, w, r, d, p, q, s, st);
      }
      c->loop_graphs_enabled = 0;
      return false;
    };
    if (!c->cap_stream && cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
      return give_up(nullptr);
    cudaGraph_t G = nullptr;
    if (cudaGraphCreate(&G, 0) != cudaSuccess) return give_up(nullptr);
    cudaGraphConditionalHandle h;
    if (cudaGraphConditionalHandleCreate(&h, G, 1, cudaGraphCondAssignDefault) != cudaSuccess) return give_up(G);
    cudaGraphNodeParams mp = {};
    mp.type = cudaGraphNodeTypeMemset;
    mp.memset.dst = trips;
    mp.memset.pitch = 0;
    mp.memset.value = 0;
    mp.memset.elementSize = sizeof(unsigned int);
    mp.memset.width = 1;
    mp.memset.height = 1;
    cudaGraphNode_t n1, n2;
    if (cudaGraphAddNode(&n1, G, nullptr, nullptr, 0, &mp) != cudaSuccess) return give_up(G);
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    if (cudaGraphAddNode(&n2, G, &n1, nullptr, 1, &cp) != cudaSuccess) return give_up(G);
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    if (cudaStreamBeginCaptureToGraph(c->cap_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
        cudaSuccess)
      return give_up(G);
    c->capturing = true;
    hdg_status cs = cg_iterations<T>(c, nrhs, dinv, w, r, d, p, q, kTrip, c->cap_stream);
    cg_loop_cond<<<1, 32, 0, c->cap_stream>>>(h, static_cast<const hdg::CgScalars*>(c->cgs.p),
                                             static_cast<const int*>(c->flags.p), nrhs, trips, kTrip);
    c->capturing = false;
    cudaGraph_t body_out = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->cap_stream, &body_out);
    cudaGraphExec_t exec = nullptr;
    if (cs != HDG_OK || e != cudaSuccess || cudaGraphInstantiate(&exec, G, 0) != cudaSuccess) return give_up(G);
    cudaGraphDestroy(G);
    c->graphs.push_back(GraphEntry{key, exec});
    ge = &c->graphs.back();
  }
  cudaError_t e = cudaGraphLaunch(ge->exec, s);
  if (e != cudaSuccess) {
    *st = fail(HDG_ERR_CUDA, std::string("cudaGraphLaunch (CG loop): ") + cudaGetErrorString(e));
    return true;
  }
  unsigned int ntrip = 0;
  e = cudaMemcpyAsync(&ntrip, trips, sizeof(unsigned int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    *st = fail(HDG_ERR_CUDA, std::string("CG loop: ") + cudaGetErrorString(e));
    return true;
  }
  c->launches += (long long)ntrip * (per_iter * kTrip + 1);
  return true;
}

// Inner (preconditioned) CG on K-hat d = rhat in precision T for the
// right-hand sides with active[r] != 0; returns per-rhs iterations and status.
template <typename T>
hdg_status inner_cg(hdg_ctx* c, int nrhs, const double* lam, const double* rhat, const std::vector<double>& tol_r,
                    const std::vector<int>& active, const std::vector<int>& max_it, bool use_pc,
                    std::vector<int>& iters, std::vector<int>& status, cudaStream_t s,
                    const double* scale = nullptr) {
  const long long T_ = c->ntrace;
  const long long tot = T_ * nrhs;
  // the fused step (a mode of the operator kernels: FP32 element runs or
  // tiles, FP64 tiles only) where hdg_set_cg_variant asks for it; else the
  // two-kernel loop (operator, cg_step_kernel)
  c->fused_cg = (c->fused_enabled && c->op_variant != 3 && c->n <= hdg::kMaxSpecialisedN &&
                 !(sizeof(T) == 8 && c->op_variant == 1)) ? 1 : 0;
  for (int i : {W_R, W_D, W_P, W_Q, W_U, W_S}) HDG_TRY(ensure(c->ws[i], sizeof(T) * (size_t)tot));
  if (c->fused_cg) {
    for (int i : {W_R2, W_S2, W_W2, W_W3}) HDG_TRY(ensure(c->ws[i], sizeof(T) * (size_t)tot));
    HDG_TRY(ensure(c->ws[W_GP], sizeof(double) * (size_t)nrhs * std::max<long long>(c->red_blocks, c->nelem)));
  }
  T* r = wsp<T>(c, W_R);
  T* d = wsp<T>(c, W_D);
  T* p = wsp<T>(c, W_P);
  T* q = wsp<T>(c, W_Q);
  T* u = wsp<T>(c, W_U);
  const T* dinv = nullptr;
  HDG_TRY(ensure_dinv<T>(c, nrhs, lam, s, &dinv));
  const T* w = nullptr;
  if (use_pc) {
    HDG_TRY(ensure_pc(c, nrhs, lam, s));
    w = pc_weights<T>(c);
  }
  double* rz0 = static_cast<double*>(c->scal.p);
  int* flags = static_cast<int*>(c->flags.p);
  hdg::CgScalars* cg = static_cast<hdg::CgScalars*>(c->cgs.p);

  if (sizeof(T) == 8) HDG_CUDA(cudaMemcpyAsync(r, rhat, sizeof(double) * tot, cudaMemcpyDeviceToDevice, s));
  else if (scale) { Timed t_(c, K_VEC, s); HDG_CUDA(hdg::launch_scale_convert(rhat, reinterpret_cast<float*>(r), T_, nrhs, scale, s)); }
  else { Timed t_(c, K_VEC, s); HDG_CUDA((hdg::launch_convert<double, float>(rhat, reinterpret_cast<float*>(r), tot, s))); }
  for (T* v : {d, p, q, u, wsp<T>(c, W_S)}) HDG_CUDA(cudaMemsetAsync(v, 0, sizeof(T) * tot, s));
  if (c->fused_cg)
    for (int i : {W_W2, W_W3}) HDG_CUDA(cudaMemsetAsync(c->ws[i].p, 0, sizeof(T) * tot, s));
  HDG_TRY(dot<T>(c, r, r, T_, nrhs, rz0, s, w));
  std::vector<int> hflags(nrhs);
  int maxit = 0;
  for (int i = 0; i < nrhs; ++i) {
    hflags[i] = active[i] ? 0 : 1;
    maxit = std::max(maxit, max_it[i]);
  }
  HDG_CUDA(cudaMemcpyAsync(flags, hflags.data(), sizeof(int) * nrhs, cudaMemcpyHostToDevice, s));
  // per-rhs relative tolerances (device copy), after the rz0 slot and u^T w slot
  double* tol_dev = static_cast<double*>(c->scal.p) + 2 * nrhs;
  HDG_CUDA(cudaMemcpyAsync(tol_dev, tol_r.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, s));
  // the per-rhs cap is the largest; per-rhs caps below it are enforced on the host afterwards
  { Timed t_(c, K_VEC, s); HDG_CUDA(hdg::launch_cg_init(cg, flags, rz0, tol_dev, maxit, nrhs, s)); }
  // u_0 = W r_0 (beta = 0 after init, u = 0); the fused step forms u_0 itself
  // (its first launch applies an update with alpha = beta = 0)
  if (!c->fused_cg) { Timed t_(c, K_VEC, s); HDG_CUDA(hdg::launch_cg_pupdate<T>(cg, u, r, w, T_, nrhs, s)); }
  const int chunk = c->fused_cg ? 3 * kFusedPeriod : 16;
  std::vector<hdg::CgScalars> hcg(nrhs);
  bool first = true;
  // the fused step as one persistent launch when the device allows it; else
  // the first chunk eagerly (sets kernel attributes before any capture), then
  // the rest of the solve as one device-driven graph launch when possible
  bool persisted = false;
  if (c->fused_cg) {
    hdg_status ps = HDG_OK;
    persisted = cg_persistent<T>(c, nrhs, dinv, w, s, &ps);
    HDG_TRY(ps);
  }
  if (persisted) {
    maxit = 0;
  } else {
    HDG_TRY(cg_iterations<T>(c, nrhs, dinv, w, r, d, p, q, c->fused_cg ? 2 * kFusedPeriod : chunk, s));
    first = false;
    hdg_status gs = HDG_OK;
    if (cg_loop_graph<T>(c, nrhs, dinv, w, r, d, p, q, s, &gs)) {
      HDG_TRY(gs);
      maxit = 0;   // done: skip the chunked loop below
    }
  }
  for (int done_it = c->fused_cg ? 2 * kFusedPeriod : chunk; done_it < maxit; done_it += chunk) {
    hdg_status gs = HDG_OK;
    // the first chunk runs eagerly (sets kernel attributes before any capture)
    if (first || !cg_graph<T>(c, nrhs, dinv, w, r, d, p, q, chunk, s, &gs))
      HDG_TRY(cg_iterations<T>(c, nrhs, dinv, w, r, d, p, q, chunk, s));
    HDG_TRY(gs);
    first = false;
    HDG_CUDA(cudaMemcpyAsync(hflags.data(), flags, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, s));
    HDG_CUDA(cudaStreamSynchronize(s));
    bool all = true;
    for (int i = 0; i < nrhs; ++i) all = all && hflags[i];
    if (all) break;
  }
  HDG_CUDA(cudaMemcpyAsync(hcg.data(), cg, sizeof(hdg::CgScalars) * nrhs, cudaMemcpyDeviceToHost, s));
  HDG_CUDA(cudaStreamSynchronize(s));
  iters.assign(nrhs, 0);
  status.assign(nrhs, HDG_OK);
  for (int i = 0; i < nrhs; ++i) {
    if (!active[i]) continue;
    iters[i] = hcg[i].it;
    status[i] = hcg[i].status == 6 ? HDG_ERR_BREAKDOWN : (hcg[i].done ? HDG_OK : HDG_ERR_NOT_CONVERGED);
    if (hcg[i].status == 5) status[i] = HDG_ERR_NOT_CONVERGED;
  }
  return HDG_OK;
}

// Full solve; `adjoint_load` selects f-hat = (S^T)^(x3) b instead of d0 (S^T M)^(x3) f.
hdg_status solve_impl(hdg_ctx* c, int nrhs, const double* lam, const double* vol_in, bool adjoint_load,
                      const double* bdry, const double* x0, double* trace_out, double* u_out,
                      const hdg_solve_opts* opts, hdg_solve_info* info, cudaStream_t s) {
  const long long T_ = c->ntrace, V = c->nvol, B = c->nbdry;
  const int n = c->n;
  hdg_solve_opts o;
  if (opts) o = *opts;
  else { o.tol = 1e-10; o.max_iter = 10000; o.max_outer = 20; o.inner = HDG_FP64; o.inner_tol = 0.0; o.precond = 1; }
  if (!(o.tol > 0.0) || o.max_iter < 1 || o.max_outer < 1) return fail(HDG_ERR_INVALID_ARG, "bad solve options");
  if (o.inner == HDG_BF16) return fail(HDG_ERR_UNSUPPORTED, "BF16 inner solve is not available");
  // each inner solve targets max(floor, tol ||F|| / (2 ||r||)) per rhs: just
  // enough for the refinement to meet the tolerance.  FP32 floor 3e-4: three
  // refinement steps of about 3.5 decades each stay clear of the region
  // where FP32 CG slows down near its accuracy limit (measured: 309 inner
  // iterations at 3e-4 against 346 at 1e-6 on a 16^3 p = 8 stretched mesh,
  // 606 against 701 on 32^3 p = 6; looser floors add refinement steps)
  const double tol_floor = o.inner_tol > 0.0 ? o.inner_tol : (o.inner == HDG_FP64 ? 0.0 : 3e-4);
  for (int r = 0; r < nrhs; ++r)
    if (lam[r] == 0.0 && !c->has_dirichlet)
      return fail(HDG_ERR_SINGULAR, "lambda = 0 without a Dirichlet side: the condensed operator is singular");
  const long long tot = T_ * nrhs;
  for (int i : {W_XHAT, W_YHAT, W_FHAT_T, W_RHAT, W_TMP}) HDG_TRY(ensure(c->ws[i], sizeof(double) * (size_t)tot));
  HDG_TRY(ensure(c->ws[W_FVOL], sizeof(double) * (size_t)V * nrhs));
  HDG_TRY(ensure(c->ws[W_GHAT], sizeof(double) * (size_t)std::max<long long>(B, 1) * nrhs));
  HDG_TRY(ensure(c->ws[W_DOT], sizeof(double) * nrhs * 2));
  HDG_TRY(ensure_reductions(c, nrhs));
  double* xhat = wsp<double>(c, W_XHAT);
  double* yhat = wsp<double>(c, W_YHAT);
  double* Fhat = wsp<double>(c, W_FHAT_T);
  double* rhat = wsp<double>(c, W_RHAT);
  double* tmp = wsp<double>(c, W_TMP);
  double* fhat = wsp<double>(c, W_FVOL);
  double* ghat = bdry ? wsp<double>(c, W_GHAT) : nullptr;
  double* dots = wsp<double>(c, W_DOT);
  const double* dinv = nullptr;
  HDG_TRY(ensure_dinv<double>(c, nrhs, lam, s, &dinv));

  // 1. f-hat in the element eigenspace
  if (adjoint_load)
    { Timed t_(c, K_VOL, s); HDG_CUDA(hdg::launch_volume_transform(n, vol_in, fhat, c->nelem, nrhs, V, c->St, c->d_metric64, c->uniform, 0, s)); }
  else
    { Timed t_(c, K_VOL, s); HDG_CUDA(hdg::launch_volume_transform(n, vol_in, fhat, c->nelem, nrhs, V, c->StM, c->d_metric64, c->uniform, 1, s)); }
  // 2. boundary data in the face eigenbasis
  if (bdry)
    { Timed t_(c, K_FACE, s); HDG_CUDA((hdg::launch_face_transform<double, double>(n, bdry, ghat, c->mesh.nbfaces, nrhs, B, B, c->StM, 1.0, 0, s))); }
  // 3. transformed right-hand side with Dirichlet lift and Neumann load
  {
    hdg::TptArgs<double, double> a = base_args<double, double>(c, dinv, nrhs, hdg::TPT_RHS);
    HDG_TRY(zero_for_tpt<double>(c, Fhat, nrhs, full_zero(c, a) ? 2 : a.nseg, s));
    a.y = Fhat;
    a.gbd = ghat;
    a.src = fhat;
    { Timed t_(c, K_RHS, s); HDG_CUDA((hdg::launch_tpt<double, double>(hdg::TPT_RHS, n, a, nrhs, s))); }
    if (bdry && c->has_neumann)
      { Timed t_(c, K_VEC, s); HDG_CUDA(hdg::launch_neumann_add(c->mesh, n, c->d_widths, c->wstride, ghat, Fhat, nrhs, B, T_, s)); }
  }
  // 4. ||F|| in the nodal basis: F = (M S (x) M S) F-hat
  { Timed t_(c, K_FACE, s); HDG_CUDA((hdg::launch_face_transform<double, double>(n, Fhat, tmp, c->mesh.nfaces, nrhs, T_, T_, c->MS, 1.0, 0, s))); }
  HDG_TRY(dot<double>(c, tmp, tmp, T_, nrhs, dots, s));
  std::vector<double> normF2(nrhs), normR2(nrhs);
  HDG_CUDA(cudaMemcpyAsync(normF2.data(), dots, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, s));
  HDG_CUDA(cudaStreamSynchronize(s));
  // 5. initial guess
  if (x0)
    { Timed t_(c, K_FACE, s); HDG_CUDA((hdg::launch_face_transform<double, double>(n, x0, xhat, c->mesh.nfaces, nrhs, T_, T_, c->StM, 1.0, 0, s))); }
  else
    HDG_CUDA(cudaMemsetAsync(xhat, 0, sizeof(double) * tot, s));

  std::vector<int> active(nrhs, 1), total_it(nrhs, 0), outer(nrhs, 0), applies(nrhs, 1), status(nrhs, HDG_OK);
  std::vector<double> relres(nrhs, 0.0);
  // a lower-precision inner solve that broke down after some iterations
  // (loss of positive curvature in FP32 rounding, on very ill-conditioned
  // systems) still leaves a usable correction: the refinement keeps it and
  // goes on while the FP64 residual falls at least twofold per step
  std::vector<int> inner_broke(nrhs, 0);
  std::vector<double> prev_rel(nrhs, 0.0);
  bool zero_x = (x0 == nullptr);
  for (int step = 0; step <= o.max_outer; ++step) {
    // residual r-hat = F-hat - K-hat x-hat (FP64)
    if (zero_x) {
      HDG_CUDA(cudaMemcpyAsync(rhat, Fhat, sizeof(double) * tot, cudaMemcpyDeviceToDevice, s));
    } else {
      HDG_TRY((tpt_apply<double, double>(c, nrhs, dinv, xhat, yhat, s)));
      { Timed t_(c, K_VEC, s); HDG_CUDA(hdg::launch_sub(Fhat, yhat, rhat, tot, s)); }
      for (int r = 0; r < nrhs; ++r) applies[r] += active[r];
    }
    { Timed t_(c, K_FACE, s); HDG_CUDA((hdg::launch_face_transform<double, double>(n, rhat, tmp, c->mesh.nfaces, nrhs, T_, T_, c->MS, 1.0, 0, s))); }
    HDG_TRY(dot<double>(c, tmp, tmp, T_, nrhs, dots, s));
    HDG_CUDA(cudaMemcpyAsync(normR2.data(), dots, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, s));
    HDG_CUDA(cudaStreamSynchronize(s));
    bool any = false;
    for (int r = 0; r < nrhs; ++r) {
      if (!active[r]) continue;
      relres[r] = normF2[r] > 0.0 ? std::sqrt(normR2[r] / normF2[r]) : std::sqrt(normR2[r]);
      const bool ok = normF2[r] > 0.0 ? normR2[r] <= o.tol * o.tol * normF2[r] : normR2[r] == 0.0;
      if (ok || !std::isfinite(relres[r])) {
        active[r] = 0;
        if (!std::isfinite(relres[r])) status[r] = HDG_ERR_BREAKDOWN;
      } else if (inner_broke[r] && !(relres[r] <= 0.5 * prev_rel[r])) {
        active[r] = 0;
        status[r] = HDG_ERR_BREAKDOWN;
      } else if (step == o.max_outer || total_it[r] >= o.max_iter) {
        active[r] = 0;
        status[r] = HDG_ERR_NOT_CONVERGED;
      }
      any = any || active[r];
    }
    if (!any) break;
    std::vector<int> caps(nrhs), it, st;
    std::vector<double> tol_r(nrhs, 1.0);
    for (int r = 0; r < nrhs; ++r) {
      caps[r] = std::max(0, o.max_iter - total_it[r]);
      const double need = normR2[r] > 0.0 ? 0.5 * o.tol * std::sqrt(normF2[r] / normR2[r]) : 1.0;
      tol_r[r] = std::min(1.0, std::max(tol_floor, need));
    }
    // inner solve K-hat d = r-hat; d is left in W_D
    if (o.inner == HDG_FP64) {
      HDG_TRY(inner_cg<double>(c, nrhs, lam, rhat, tol_r, active, caps, o.precond != 0, it, st, s));
      { Timed t_(c, K_VEC, s); HDG_CUDA(hdg::launch_add_to<double>(xhat, wsp<double>(c, W_D), tot, s)); }
    } else {
      // the FP32 system is scaled per rhs by a power of two that brings the
      // residual norm near 1 (residuals of large data would overflow the
      // FP32 inner products); the correction is scaled back exactly
      std::vector<double> sc(2 * (size_t)nrhs, 1.0);   // scales, then their inverses
      for (int r = 0; r < nrhs; ++r) {
        const double nr = std::sqrt(normR2[r]);
        if (nr > 0.0 && std::isfinite(nr)) {
          const int e = std::ilogb(nr);
          sc[r] = std::ldexp(1.0, -e);
          sc[nrhs + r] = std::ldexp(1.0, e);
        }
      }
      double* sc_dev = static_cast<double*>(c->scal.p) + 3 * nrhs;
      HDG_CUDA(cudaMemcpyAsync(sc_dev, sc.data(), sizeof(double) * 2 * nrhs, cudaMemcpyHostToDevice, s));
      HDG_TRY(inner_cg<float>(c, nrhs, lam, rhat, tol_r, active, caps, o.precond != 0, it, st, s, sc_dev));
      { Timed t_(c, K_VEC, s); HDG_CUDA(hdg::launch_add_unscaled(xhat, wsp<float>(c, W_D), T_, nrhs, sc_dev + nrhs, s)); }
    }
    zero_x = false;
    for (int r = 0; r < nrhs; ++r) {
      if (!active[r]) continue;
      total_it[r] += it[r];
      applies[r] += it[r];
      outer[r] += 1;
      prev_rel[r] = relres[r];
      inner_broke[r] = 0;
      if (st[r] == HDG_ERR_BREAKDOWN) {
        if (o.inner == HDG_FP64 || it[r] == 0) { status[r] = HDG_ERR_BREAKDOWN; active[r] = 0; }
        else inner_broke[r] = 1;
      }
    }
  }
  // 6. traces in the nodal basis, u by recovery
  { Timed t_(c, K_FACE, s); HDG_CUDA((hdg::launch_face_transform<double, double>(n, xhat, trace_out, c->mesh.nfaces, nrhs, T_, T_, c->S, 1.0, 0, s))); }
  if (u_out) {
    HDG_TRY(ensure(c->ws[W_WVOL], sizeof(double) * (size_t)V * nrhs));
    double* w = wsp<double>(c, W_WVOL);
    hdg::TptArgs<double, double> a = base_args<double, double>(c, dinv, nrhs, hdg::TPT_RECOVER);
    a.x = xhat;
    a.gbd = ghat;
    a.src = fhat;
    a.vout = w;
    { Timed t_(c, K_RHS, s); HDG_CUDA((hdg::launch_tpt<double, double>(hdg::TPT_RECOVER, n, a, nrhs, s))); }
    { Timed t_(c, K_VOL, s); HDG_CUDA(hdg::launch_volume_transform(n, w, u_out, c->nelem, nrhs, V, c->S, c->d_metric64, c->uniform, 0, s)); }
  }
  HDG_CUDA(cudaStreamSynchronize(s));
  hdg_status worst = HDG_OK;
  for (int r = 0; r < nrhs; ++r) {
    if (info) {
      info[r].iterations = total_it[r];
      info[r].outer = outer[r];
      info[r].applies = applies[r];
      info[r].rel_residual = relres[r];
      info[r].status = status[r];
    }
    if (status[r] != HDG_OK && worst == HDG_OK) worst = (hdg_status)status[r];
  }
  if (worst != HDG_OK) return fail(worst, "solve did not reach the tolerance for every right-hand side");
  return HDG_OK;
}

__global__ void negate_kernel(double* x, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = -x[i];
}

}  // namespace

namespace hdg {
bool ctx_view(const hdg_ctx* c, CtxView* v) {
  if (!c || !v) return false;
  v->device = c->device;
  v->sms = c->sms;
  v->n = c->n;
  v->uniform = c->uniform;
  v->mesh = c->mesh;
  v->tab = c->tab64;
  v->metric64 = c->d_metric64;
  v->Lambda = c->d_Lambda;
  v->StM = c->StM;
  v->MS = c->MS;
  v->nelem = c->nelem;
  v->ntrace = c->ntrace;
  v->nclass = nclass(c);
  return true;
}
void set_last_error(const char* msg) {
  if (msg[0] == 0) g_last_error.clear();
  else fail(HDG_OK, msg);   // quotes an error that was pending at entry, as every entry point does
}
void begin_entry() { begin_call(); }
hdg_status check_lambdas(int nrhs, const double* lam) { return check_lambda(nullptr, nrhs, lam); }
}  // namespace hdg

// 1D / 2D context (hdg_lowdim_*): mesh bookkeeping, 1D tables, metric
struct hdg_lowdim {
  int dim = 1, p = 1, n = 2;
  int ne[2] = {1, 1};
  int bc[4] = {0, 0, 0, 0};
  int lo[2] = {0, 0}, hi[2] = {-1, -1};
  long long blk[2] = {0, 0};
  long long ntrace = 0;
  hdg::Setup1D s1;
  hdg::Tables<double> tab{};
  hdg::Mat1D<double> StM{}, MS{};
  double* d_metric = nullptr;
  DevBuf lam;
};

extern "C" {

const char* hdg_last_error(void) { return g_last_error.c_str(); }

hdg_status hdg_set_x1_segment(hdg_ctx* c, int elements) {
  if (!c || elements < 0) return fail(HDG_ERR_INVALID_ARG, "NULL context or negative segment length");
  c->seg_override = elements;
  return HDG_OK;
}

hdg_status hdg_set_slots_per_cta(hdg_ctx* c, int slots) {
  if (!c || slots < 0 || hdg::tpt_threads(c->n, slots) > 320)
    return fail(HDG_ERR_INVALID_ARG, "NULL context or slot count outside 0..(320 threads)");
  c->ppb_override = slots;
  return HDG_OK;
}

hdg_status hdg_autotune(hdg_ctx* c, int nrhs, const double* h_lambda, hdg_precision prec, int* h_best_segment,
                        int* h_best_slots, double* h_best_us, void* stream) {
  begin_call();
  if (!c || nrhs < 1 || prec == HDG_BF16) return fail(HDG_ERR_INVALID_ARG, "NULL context, nrhs < 1 or BF16");
  HDG_TRY(check_lambda(c, nrhs, h_lambda));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t esz = prec == HDG_FP64 ? 8 : 4;
  const size_t tot = (size_t)c->ntrace * nrhs;
  HDG_TRY(ensure(c->ws[W_XHAT], esz * tot));
  HDG_TRY(ensure(c->ws[W_YHAT], esz * tot));
  HDG_CUDA(cudaMemsetAsync(c->ws[W_XHAT].p, 0x3c, esz * tot, s));   // finite, non-zero pattern
  // candidate segment lengths (distinct splits of the x1-pencils) and slots;
  // for the tile kernel: elements per tile, no slots
  const bool tiles = prec == HDG_FP64 ? use_tiles<double, double>(c, nrhs) : use_tiles<float, float>(c, nrhs);
  std::vector<int> segs = {0};
  if (tiles) {
    for (int e : {2, 3, 4, 5, 6, 8, 10, 12, 14, 16, 20, 24, 28, 32}) segs.push_back(e);
  } else {
    for (int sg = 1; sg <= c->mesh.ne[0]; ++sg) {
      const int ns = (c->mesh.ne[0] + sg - 1) / sg;
      if (sg > 1 && (c->mesh.ne[0] + sg - 2) / (sg - 1) == ns) continue;
      if (sg <= 4 || sg == c->mesh.ne[0] || (sg & (sg - 1)) == 0) segs.push_back(sg);
    }
  }
  std::vector<int> slots = {0};
  const int base = hdg::tpt_ppb(c->n);
  const int max_threads = prec == HDG_FP64 ? 320 : hdg::fast_max_threads(c->n);
  for (int pp : {base / 2, base - 1, base + 1, base * 3 / 2})
    if (!tiles && pp >= 1 && pp != base &&
        (prec == HDG_FP64 ? hdg::tpt_threads(c->n, pp) : hdg::fast_threads(c->n, pp)) <= max_threads)
      slots.push_back(pp);
  const int keep_seg = c->seg_override, keep_ppb = c->ppb_override;
  cudaEvent_t e0, e1;
  HDG_CUDA(cudaEventCreate(&e0));
  HDG_CUDA(cudaEventCreate(&e1));
  double best = -1.0;
  int best_seg = 0, best_ppb = 0;
  hdg_status st = HDG_OK;
  for (int pp : slots) {
    for (int sg : segs) {
      c->seg_override = sg;
      c->ppb_override = pp;
      auto run = [&]() -> hdg_status {
        if (prec == HDG_FP64) {
          const double* dinv = nullptr;
          HDG_TRY(ensure_dinv<double>(c, nrhs, h_lambda, s, &dinv));
          return tpt_apply<double, double>(c, nrhs, dinv, wsp<double>(c, W_XHAT), wsp<double>(c, W_YHAT), s);
        }
        const float* dinv = nullptr;
        HDG_TRY(ensure_dinv<float>(c, nrhs, h_lambda, s, &dinv));
        return tpt_apply<float, float>(c, nrhs, dinv, wsp<float>(c, W_XHAT), wsp<float>(c, W_YHAT), s);
      };
      for (int w = 0; w < 2 && st == HDG_OK; ++w) st = run();
      const int reps = 5;
      if (st == HDG_OK && cudaEventRecord(e0, s) != cudaSuccess) st = fail(HDG_ERR_CUDA, "autotune event");
      for (int k = 0; k < reps && st == HDG_OK; ++k) st = run();
      if (st == HDG_OK && cudaEventRecord(e1, s) != cudaSuccess) st = fail(HDG_ERR_CUDA, "autotune event");
      float ms = 0.f;
      if (st == HDG_OK && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
        st = fail(HDG_ERR_CUDA, "autotune timing");
      if (st != HDG_OK) break;
      const double us = 1e3 * ms / reps;
      if (best < 0.0 || us < best) {
        best = us;
        best_seg = sg;
        best_ppb = pp;
      }
    }
    if (st != HDG_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != HDG_OK) {
    c->seg_override = keep_seg;
    c->ppb_override = keep_ppb;
    return st;
  }
  c->seg_override = best_seg;
  c->ppb_override = best_ppb;
  if (h_best_segment) *h_best_segment = best_seg;
  if (h_best_slots) *h_best_slots = best_ppb;
  if (h_best_us) *h_best_us = best;
  return HDG_OK;
}

hdg_status hdg_set_operator_variant(hdg_ctx* c, int variant) {
  if (!c || variant < 0 || variant > 3) return fail(HDG_ERR_INVALID_ARG, "NULL context or variant outside 0..3");
  c->op_variant = variant;
  return HDG_OK;
}

hdg_status hdg_set_cg_variant(hdg_ctx* c, int variant) {
  if (!c || variant < 0 || variant > 3) return fail(HDG_ERR_INVALID_ARG, "NULL context or CG variant outside 0..3");
  c->fused_enabled = (variant == 0 || variant == 2) ? 1 : 0;
  c->persist_enabled = variant == 0 ? 1 : 0;
  return HDG_OK;
}

hdg_status hdg_set_nodal_variant(hdg_ctx* c, int variant) {
  if (!c || variant < 0 || variant > 1) return fail(HDG_ERR_INVALID_ARG, "NULL context or nodal variant outside 0..1");
  c->nodal_variant = variant;
  return HDG_OK;
}

hdg_status hdg_set_dz_mode(hdg_ctx* c, int mode) {
  if (!c || mode < 0 || mode > 2) return fail(HDG_ERR_INVALID_ARG, "NULL context or D_Z mode outside 0..2");
  if (mode != c->dz_mode) c->lam32.clear();   // rebuild (or drop) the FP32 table on next use
  c->dz_mode = mode;
  return HDG_OK;
}

hdg_status hdg_profile(hdg_ctx* c, int enable) {
  if (!c) return fail(HDG_ERR_INVALID_ARG, "NULL context");
  if (enable) {
    c->launches = 0;
    for (int k = 0; k < 6; ++k) c->ev_used[k] = 0;
  }
  c->prof_on = enable != 0;
  return HDG_OK;
}

hdg_status hdg_profile_read(hdg_ctx* c, int cls, double* total_ms, long long* launches) {
  if (!c || !total_ms || !launches || cls < -1 || cls > 5) return fail(HDG_ERR_INVALID_ARG, "bad profile query");
  HDG_CUDA(cudaDeviceSynchronize());
  if (cls == -1) {
    *total_ms = 0.0;
    *launches = c->launches;
    return HDG_OK;
  }
  double tot = 0.0;
  for (size_t i = 0; i < c->ev_used[cls]; ++i) {
    float ms = 0.f;
    HDG_CUDA(cudaEventElapsedTime(&ms, c->ev[cls][2 * i], c->ev[cls][2 * i + 1]));
    tot += ms;
  }
  *total_ms = tot;
  *launches = (long long)c->ev_used[cls];
  return HDG_OK;
}

const char* hdg_status_string(hdg_status s) {
  switch (s) {
    case HDG_OK: return "ok";
    case HDG_ERR_INVALID_ARG: return "invalid argument";
    case HDG_ERR_SINGULAR: return "singular operator (lambda = 0 without Dirichlet data)";
    case HDG_ERR_CUDA: return "CUDA error";
    case HDG_ERR_OOM: return "out of device memory";
    case HDG_ERR_NOT_CONVERGED: return "not converged";
    case HDG_ERR_BREAKDOWN: return "CG breakdown";
    case HDG_ERR_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

hdg_status hdg_setup(const hdg_mesh* mesh, int p, const hdg_options* opts, hdg_ctx** out) {
  begin_call();
  if (!mesh || !out) return fail(HDG_ERR_INVALID_ARG, "mesh and out must not be NULL");
  *out = nullptr;
  if (p < 1 || p > 32) return fail(HDG_ERR_UNSUPPORTED, "degree p must be in 1..32");
  const double tau_hat = opts ? opts->tau_hat : 25.0;
  const int lumped = opts ? opts->mass_lumped : 0;
  for (int d = 0; d < 3; ++d) {
    if (mesh->ne[d] < 1 || !mesh->h_grid[d]) return fail(HDG_ERR_INVALID_ARG, "each direction needs >= 1 element and a grid");
    for (int i = 0; i < mesh->ne[d]; ++i)
      if (!(mesh->h_grid[d][i + 1] > mesh->h_grid[d][i])) return fail(HDG_ERR_INVALID_ARG, "grid lines must increase");
  }
  for (int sd = 0; sd < 6; ++sd)
    if (mesh->bc[sd] != 0 && mesh->bc[sd] != 1) return fail(HDG_ERR_INVALID_ARG, "bc must be 0 (Dirichlet) or 1 (Neumann)");
  int dev = 0;
  HDG_CUDA(cudaGetDevice(&dev));
  cudaDeviceProp prop;
  HDG_CUDA(cudaGetDeviceProperties(&prop, dev));
  if (!(prop.major == 10 && prop.minor == 3))
    return fail(HDG_ERR_UNSUPPORTED, "this library is built for sm_103 (GB300) only");

  hdg_ctx* c = new hdg_ctx();
  c->device = dev;
  c->sms = prop.multiProcessorCount;
  c->p = p;
  c->n = p + 1;
  const char* msg = "";
  if (hdg::build_setup1d(p, tau_hat, lumped, &c->s1, &msg) != 0) {
    delete c;
    return fail(HDG_ERR_INVALID_ARG, std::string("1D set-up: ") + msg);
  }
  const int n = c->n;
  hdg::MeshDev& m = c->mesh;
  long long off = 0;
  for (int d = 0; d < 3; ++d) {
    m.ne[d] = mesh->ne[d];
    c->widths[d].resize(mesh->ne[d]);
    for (int i = 0; i < mesh->ne[d]; ++i) c->widths[d][i] = mesh->h_grid[d][i + 1] - mesh->h_grid[d][i];
  }
  for (int sd = 0; sd < 6; ++sd) {
    c->bc[sd] = mesh->bc[sd];
    if (mesh->bc[sd] == 0) c->has_dirichlet = 1;
    else c->has_neumann = 1;
  }
  for (int d = 0; d < 3; ++d) {
    const int a = d == 0 ? 1 : 0, b = d == 2 ? 1 : 2;
    m.lo[d] = c->bc[2 * d] == 1 ? 0 : 1;
    m.hi[d] = c->bc[2 * d + 1] == 1 ? m.ne[d] : m.ne[d] - 1;
    m.blk[d] = off;
    const long long np = std::max(0, m.hi[d] - m.lo[d] + 1);
    off += np * m.ne[a] * m.ne[b];
  }
  m.nfaces = off;
  off = 0;
  for (int sd = 0; sd < 6; ++sd) {
    const int d = sd / 2, a = d == 0 ? 1 : 0, b = d == 2 ? 1 : 2;
    m.side[sd] = off;
    off += (long long)m.ne[a] * m.ne[b];
  }
  m.nbfaces = off;
  c->nelem = (long long)m.ne[0] * m.ne[1] * m.ne[2];
  c->ntrace = m.nfaces * n * n;
  c->nvol = c->nelem * n * n * n;
  c->nbdry = m.nbfaces * n * n;
  if (c->ntrace >= (1LL << 31) || c->nbdry >= (1LL << 31) || c->nvol >= (1LL << 40)) {
    hdg_destroy(c);
    return fail(HDG_ERR_UNSUPPORTED, "mesh too large: the trace vector per right-hand side must stay below 2^31 values");
  }
  // uniform: every direction has constant width (to round-off) -> one element class
  bool uni = true;
  for (int d = 0; d < 3; ++d)
    for (double w : c->widths[d]) uni = uni && std::fabs(w - c->widths[d][0]) <= 1e-14 * c->widths[d][0];
  c->uniform = uni ? 1 : 0;
  m.uniform = c->uniform;
  // metric factors d0..d3 of Sec. 3.2 per element (or the single class)
  const long long ncls = uni ? 1 : c->nelem;
  std::vector<double> met(4 * ncls);
  std::vector<float> met32(4 * ncls);
  for (long long e = 0; e < ncls; ++e) {
    const int e1 = (int)(e % m.ne[0]), e2 = (int)((e / m.ne[0]) % m.ne[1]), e3 = (int)(e / ((long long)m.ne[0] * m.ne[1]));
    const double h1 = c->widths[0][e1], h2 = c->widths[1][e2], h3 = c->widths[2][e3];
    const double d0 = h1 * h2 * h3 / 8.0;
    met[4 * e + 0] = d0;
    met[4 * e + 1] = d0 * (2.0 / h1) * (2.0 / h1);
    met[4 * e + 2] = d0 * (2.0 / h2) * (2.0 / h2);
    met[4 * e + 3] = d0 * (2.0 / h3) * (2.0 / h3);
    for (int k = 0; k < 4; ++k) met32[4 * e + k] = (float)met[4 * e + k];
  }
  c->wstride = std::max(m.ne[0], std::max(m.ne[1], m.ne[2]));
  std::vector<double> wid(3 * c->wstride, 0.0);
  for (int d = 0; d < 3; ++d)
    for (int i = 0; i < m.ne[d]; ++i) wid[d * c->wstride + i] = c->widths[d][i];
  auto up = [&](void** dst, const void* src, size_t bytes) -> hdg_status {
    cudaError_t e = cudaMalloc(dst, bytes);
    if (e != cudaSuccess) return fail(HDG_ERR_OOM, "cudaMalloc tables");
    e = cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(HDG_ERR_CUDA, "upload tables");
    return HDG_OK;
  };
  hdg_status st = HDG_OK;
  if (st == HDG_OK) st = up((void**)&c->d_metric64, met.data(), sizeof(double) * met.size());
  if (st == HDG_OK) st = up((void**)&c->d_metric32, met32.data(), sizeof(float) * met32.size());
  if (st == HDG_OK) st = up((void**)&c->d_Lambda, c->s1.Lambda, sizeof(double) * n);
  if (st == HDG_OK) st = up((void**)&c->d_widths, wid.data(), sizeof(double) * wid.size());
  if (st != HDG_OK) {
    hdg_destroy(c);
    return st;
  }
  for (int i = 0; i < n; ++i) {
    c->tab64.c[i] = c->s1.bs[i];
    c->tab32.c[i] = (float)c->s1.bs[i];
    c->tab64.lam[i] = c->s1.Lambda[i];
    c->tab32.lam[i] = (float)c->s1.Lambda[i];
  }
  c->tab64.h0 = c->s1.h0;
  c->tab64.h1 = c->s1.h1;
  c->tab32.h0 = (float)c->s1.h0;
  c->tab32.h1 = (float)c->s1.h1;
  for (int i = 0; i < n * n; ++i) {
    c->StM.a[i] = c->s1.StM[i];
    c->MS.a[i] = c->s1.MS[i];
    c->St.a[i] = c->s1.St[i];
    c->M.a[i] = c->s1.M[i];
  }
  // S as the matrix acting on a vector of mode coefficients: (S)[node][mode]
  for (int i = 0; i < n; ++i)
    for (int mm = 0; mm < n; ++mm) c->S.a[i * n + mm] = c->s1.S[i * n + mm];
  *out = c;
  return HDG_OK;
}

void hdg_destroy(hdg_ctx* c) {
  if (!c) return;
  cudaDeviceSynchronize();
  cudaFree(c->d_metric64);
  cudaFree(c->d_metric32);
  cudaFree(c->d_Lambda);
  cudaFree(c->d_widths);
  for (DevBuf* b : {&c->dinv64, &c->dinv32, &c->lam_dev64, &c->lam_dev32, &c->partials, &c->step_partials,
                    &c->counters, &c->cgs,
                    &c->flags, &c->scal})
    if (b->p) cudaFree(b->p);
  for (DevBuf& b : c->ws)
    if (b.p) cudaFree(b.p);
  for (auto& v : c->ev)
    for (cudaEvent_t e : v) cudaEventDestroy(e);
  for (DevBuf* b : {&c->pc_diag, &c->pc_w64, &c->pc_w32, &c->loopctl})
    if (b->p) cudaFree(b->p);
  for (auto& g : c->graphs) cudaGraphExecDestroy(g.exec);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  delete c;
}

size_t hdg_trace_size(const hdg_ctx* c) { return c ? (size_t)c->ntrace : 0; }
size_t hdg_volume_size(const hdg_ctx* c) { return c ? (size_t)c->nvol : 0; }
size_t hdg_boundary_size(const hdg_ctx* c) { return c ? (size_t)c->nbdry : 0; }

hdg_status hdg_get_nodes(const hdg_ctx* c, double* h_nodes) {
  if (!c || !h_nodes) return fail(HDG_ERR_INVALID_ARG, "NULL argument");
  std::memcpy(h_nodes, c->s1.nodes, sizeof(double) * c->n);
  return HDG_OK;
}

hdg_status hdg_apply(hdg_ctx* c, int nrhs, const double* h_lambda, hdg_precision prec, hdg_basis basis,
                     const void* d_x, void* d_y, void* stream) {
  begin_call();
  if (!c || !d_x || !d_y || nrhs < 1) return fail(HDG_ERR_INVALID_ARG, "NULL pointer or nrhs < 1");
  HDG_TRY(check_lambda(c, nrhs, h_lambda));
  if (basis != HDG_BASIS_NODAL && basis != HDG_BASIS_TRANSFORMED) return fail(HDG_ERR_INVALID_ARG, "bad basis");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const long long tot = c->ntrace * nrhs;
  const int n = c->n;
  if (prec == HDG_FP64) {
    const double* dinv = nullptr;
    HDG_TRY(ensure_dinv<double>(c, nrhs, h_lambda, s, &dinv));
    if (basis == HDG_BASIS_TRANSFORMED)
      return tpt_apply<double, double>(c, nrhs, dinv, static_cast<const double*>(d_x), static_cast<double*>(d_y), s);
    if (c->nodal_variant == 1 && n <= hdg::kMaxSpecialisedN)
      return nodal_apply(c, nrhs, dinv, static_cast<const double*>(d_x), static_cast<double*>(d_y), s);
    HDG_TRY(ensure(c->ws[W_XHAT], sizeof(double) * tot));
    HDG_TRY(ensure(c->ws[W_YHAT], sizeof(double) * tot));
    double* xh = wsp<double>(c, W_XHAT);
    double* yh = wsp<double>(c, W_YHAT);
    { Timed t_(c, K_FACE, s); HDG_CUDA((hdg::launch_face_transform<double, double>(n, static_cast<const double*>(d_x), xh, c->mesh.nfaces,
                                                          nrhs, c->ntrace, c->ntrace, c->StM, 1.0, 0, s))); }
    HDG_TRY((tpt_apply<double, double>(c, nrhs, dinv, xh, yh, s)));
    { Timed t_(c, K_FACE, s); HDG_CUDA((hdg::launch_face_transform<double, double>(n, yh, static_cast<double*>(d_y), c->mesh.nfaces, nrhs,
                                                          c->ntrace, c->ntrace, c->MS, 1.0, 0, s))); }
    return HDG_OK;
  }
  if (prec == HDG_FP32) {
    const float* dinv = nullptr;
    HDG_TRY(ensure_dinv<float>(c, nrhs, h_lambda, s, &dinv));
    if (basis == HDG_BASIS_TRANSFORMED)
      return tpt_apply<float, float>(c, nrhs, dinv, static_cast<const float*>(d_x), static_cast<float*>(d_y), s);
    HDG_TRY(ensure(c->ws[W_XHAT], sizeof(float) * tot));
    HDG_TRY(ensure(c->ws[W_YHAT], sizeof(float) * tot));
    float* xh = wsp<float>(c, W_XHAT);
    float* yh = wsp<float>(c, W_YHAT);
    { Timed t_(c, K_FACE, s); HDG_CUDA((hdg::launch_face_transform<float, float>(n, static_cast<const float*>(d_x), xh, c->mesh.nfaces, nrhs,
                                                        c->ntrace, c->ntrace, c->StM, 1.0, 0, s))); }
    HDG_TRY((tpt_apply<float, float>(c, nrhs, dinv, xh, yh, s)));
    { Timed t_(c, K_FACE, s); HDG_CUDA((hdg::launch_face_transform<float, float>(n, yh, static_cast<float*>(d_y), c->mesh.nfaces, nrhs,
                                                        c->ntrace, c->ntrace, c->MS, 1.0, 0, s))); }
    return HDG_OK;
  }
  // BF16-stored traces, FP32 arithmetic, transformed basis
  if (basis != HDG_BASIS_TRANSFORMED) return fail(HDG_ERR_INVALID_ARG, "BF16 apply is available in the transformed basis only");
  const float* dinv = nullptr;
  HDG_TRY(ensure_dinv<float>(c, nrhs, h_lambda, s, &dinv));
  return tpt_apply<float, __nv_bfloat16>(c, nrhs, dinv, static_cast<const __nv_bfloat16*>(d_x),
                                         static_cast<__nv_bfloat16*>(d_y), s);
}

hdg_status hdg_solve(hdg_ctx* c, int nrhs, const double* h_lambda, const double* d_f, const double* d_bdry,
                     const double* d_x0, double* d_trace, double* d_u, const hdg_solve_opts* opts,
                     hdg_solve_info* h_info, void* stream) {
  begin_call();
  if (!c || !d_f || !d_trace || nrhs < 1) return fail(HDG_ERR_INVALID_ARG, "NULL pointer or nrhs < 1");
  HDG_TRY(check_lambda(c, nrhs, h_lambda));
  return solve_impl(c, nrhs, h_lambda, d_f, false, d_bdry, d_x0, d_trace, d_u, opts, h_info,
                    static_cast<cudaStream_t>(stream));
}

hdg_status hdg_solve_adjoint(hdg_ctx* c, int nrhs, const double* h_lambda, const double* d_u,
                             const double* d_grad_u, double* d_grad_f, double* d_grad_lambda,
                             const hdg_solve_opts* opts, hdg_solve_info* h_info, void* stream) {
  begin_call();
  if (!c || !d_u || !d_grad_u || !d_grad_f || !d_grad_lambda || nrhs < 1)
    return fail(HDG_ERR_INVALID_ARG, "NULL pointer or nrhs < 1");
  HDG_TRY(check_lambda(c, nrhs, h_lambda));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const long long V = c->nvol;
  HDG_TRY(ensure(c->ws[W_DOT2], sizeof(double) * (size_t)V * nrhs));
  HDG_TRY(ensure(c->ws[W_WVOL], sizeof(double) * (size_t)V * nrhs));
  HDG_TRY(ensure(c->ws[W_TMP], sizeof(double) * (size_t)c->ntrace * nrhs));
  // adjoint traces are not returned: solve into a scratch trace buffer
  DevBuf tr;
  HDG_TRY(ensure(tr, sizeof(double) * (size_t)c->ntrace * nrhs));
  double* z = wsp<double>(c, W_DOT2);
  hdg_status st = solve_impl(c, nrhs, h_lambda, d_grad_u, true, nullptr, nullptr, static_cast<double*>(tr.p), z,
                             opts, h_info, s);
  cudaFree(tr.p);
  if (st != HDG_OK) return st;
  // dL/df = M_e z_u = d0 (M (x) M (x) M) z_u ;  dL/dlambda = - (M_e z_u) . u
  { Timed t_(c, K_VOL, s); HDG_CUDA(hdg::launch_volume_transform(c->n, z, d_grad_f, c->nelem, nrhs, V, c->M, c->d_metric64, c->uniform, 1, s)); }
  HDG_TRY(ensure_reductions(c, nrhs));
  HDG_TRY(dot<double>(c, d_grad_f, d_u, V, nrhs, d_grad_lambda, s));
  { Timed t_(c, K_VEC, s); negate_kernel<<<(nrhs + 127) / 128, 128, 0, s>>>(d_grad_lambda, nrhs); }
  HDG_CUDA(cudaGetLastError());
  HDG_CUDA(cudaStreamSynchronize(s));
  return HDG_OK;
}

hdg_status hdg_lowdim_setup(const hdg_lowdim_mesh* mesh, int p, const hdg_options* opts, hdg_lowdim** out) {
  begin_call();
  if (!mesh || !out) return fail(HDG_ERR_INVALID_ARG, "mesh and out must not be NULL");
  *out = nullptr;
  if (mesh->dim != 1 && mesh->dim != 2) return fail(HDG_ERR_INVALID_ARG, "dim must be 1 or 2");
  if (p < 1 || p > 16) return fail(HDG_ERR_UNSUPPORTED, "degree p must be in 1..16");
  const int dim = mesh->dim;
  for (int d = 0; d < dim; ++d) {
    if (mesh->ne[d] < 1 || !mesh->h_grid[d]) return fail(HDG_ERR_INVALID_ARG, "each direction needs >= 1 element and a grid");
    for (int i = 0; i < mesh->ne[d]; ++i)
      if (!(mesh->h_grid[d][i + 1] > mesh->h_grid[d][i])) return fail(HDG_ERR_INVALID_ARG, "grid lines must increase");
  }
  for (int sd = 0; sd < 2 * dim; ++sd)
    if (mesh->bc[sd] != 0 && mesh->bc[sd] != 1) return fail(HDG_ERR_INVALID_ARG, "bc must be 0 (Dirichlet) or 1 (Neumann)");
  int dev = 0;
  HDG_CUDA(cudaGetDevice(&dev));
  cudaDeviceProp prop;
  HDG_CUDA(cudaGetDeviceProperties(&prop, dev));
  if (!(prop.major == 10 && prop.minor == 3))
    return fail(HDG_ERR_UNSUPPORTED, "this library is built for sm_103 (GB300) only");
  hdg_lowdim* c = new hdg_lowdim();
  c->dim = dim;
  c->p = p;
  c->n = p + 1;
  const char* msg = "";
  if (hdg::build_setup1d(p, opts ? opts->tau_hat : 25.0, opts ? opts->mass_lumped : 0, &c->s1, &msg) != 0) {
    delete c;
    return fail(HDG_ERR_INVALID_ARG, std::string("1D set-up: ") + msg);
  }
  const int n = c->n;
  for (int d = 0; d < dim; ++d) c->ne[d] = mesh->ne[d];
  for (int sd = 0; sd < 2 * dim; ++sd) c->bc[sd] = mesh->bc[sd];
  long long faces = 0;
  for (int d = 0; d < dim; ++d) {
    c->lo[d] = c->bc[2 * d] == 1 ? 0 : 1;
    c->hi[d] = c->bc[2 * d + 1] == 1 ? c->ne[d] : c->ne[d] - 1;
    c->blk[d] = faces;
    const long long other = dim == 2 ? c->ne[1 - d] : 1;
    faces += std::max(0, c->hi[d] - c->lo[d] + 1) * other;
  }
  c->ntrace = faces * (dim == 2 ? n : 1);
  const long long nelem = (long long)c->ne[0] * c->ne[1];
  if (c->ntrace >= (1LL << 31) || nelem >= (1LL << 31)) {
    delete c;
    return fail(HDG_ERR_UNSUPPORTED, "trace size above 2^31 - 1");
  }
  for (int i = 0; i < n; ++i) {
    c->tab.c[i] = c->s1.bs[i];
    c->tab.lam[i] = c->s1.Lambda[i];
  }
  c->tab.h0 = c->s1.h0;
  c->tab.h1 = c->s1.h1;
  for (int i = 0; i < n * n; ++i) {
    c->StM.a[i] = c->s1.StM[i];
    c->MS.a[i] = c->s1.MS[i];
  }
  // metric factors (Sec. 2.2 / 3.2 with dim directions): d0 = prod h/2, d_i = d0 (2/h_i)^2
  std::vector<double> met(4 * (size_t)nelem, 0.0);
  for (long long e = 0; e < nelem; ++e) {
    const int e1 = (int)(e % c->ne[0]), e2 = (int)(e / c->ne[0]);
    const double h1 = mesh->h_grid[0][e1 + 1] - mesh->h_grid[0][e1];
    const double h2 = dim == 2 ? mesh->h_grid[1][e2 + 1] - mesh->h_grid[1][e2] : 2.0;
    const double d0 = h1 * h2 / 4.0;
    met[4 * e] = d0;
    met[4 * e + 1] = d0 * (2.0 / h1) * (2.0 / h1);
    met[4 * e + 2] = dim == 2 ? d0 * (2.0 / h2) * (2.0 / h2) : 0.0;
  }
  cudaError_t ce = cudaMalloc(&c->d_metric, sizeof(double) * met.size());
  if (ce == cudaSuccess) ce = cudaMemcpy(c->d_metric, met.data(), sizeof(double) * met.size(), cudaMemcpyHostToDevice);
  if (ce != cudaSuccess) {
    cudaFree(c->d_metric);
    delete c;
    return fail(ce == cudaErrorMemoryAllocation ? HDG_ERR_OOM : HDG_ERR_CUDA,
                std::string("metric upload: ") + cudaGetErrorString(ce));
  }
  *out = c;
  return HDG_OK;
}

size_t hdg_lowdim_trace_size(const hdg_lowdim* c) { return c ? (size_t)c->ntrace : 0; }

hdg_status hdg_lowdim_apply(hdg_lowdim* c, int nrhs, const double* h_lambda, hdg_basis basis, const double* d_x,
                            double* d_y, void* stream) {
  begin_call();
  if (!c || !d_x || !d_y || nrhs < 1) return fail(HDG_ERR_INVALID_ARG, "NULL pointer or nrhs < 1");
  if (nrhs > 65535) return fail(HDG_ERR_INVALID_ARG, "nrhs above 65535");
  if (!h_lambda) return fail(HDG_ERR_INVALID_ARG, "lambda pointer is NULL");
  for (int r = 0; r < nrhs; ++r)
    if (!(h_lambda[r] >= 0.0) || !std::isfinite(h_lambda[r])) return fail(HDG_ERR_INVALID_ARG, "lambda must be finite and >= 0");
  if (basis != HDG_BASIS_NODAL && basis != HDG_BASIS_TRANSFORMED) return fail(HDG_ERR_INVALID_ARG, "bad basis");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (c->ntrace == 0) return HDG_OK;
  HDG_TRY(ensure(c->lam, sizeof(double) * nrhs));
  HDG_CUDA(cudaMemcpyAsync(c->lam.p, h_lambda, sizeof(double) * nrhs, cudaMemcpyHostToDevice, s));
  HDG_CUDA(cudaMemsetAsync(d_y, 0, sizeof(double) * (size_t)c->ntrace * nrhs, s));
  hdg::LowDimArgs a{};
  a.dim = c->dim;
  a.n = c->n;
  for (int d = 0; d < 2; ++d) {
    a.ne[d] = c->ne[d];
    a.lo[d] = c->lo[d];
    a.hi[d] = c->hi[d];
    a.blk[d] = c->blk[d];
  }
  a.tab = c->tab;
  a.StM = c->StM;
  a.MS = c->MS;
  a.metric = c->d_metric;
  a.lam = static_cast<const double*>(c->lam.p);
  a.x = d_x;
  a.y = d_y;
  a.trace_stride = c->ntrace;
  a.nodal = basis == HDG_BASIS_NODAL ? 1 : 0;
  HDG_CUDA(hdg::launch_lowdim(a, nrhs, s));
  return HDG_OK;
}

void hdg_lowdim_destroy(hdg_lowdim* c) {
  if (!c) return;
  cudaDeviceSynchronize();
  cudaFree(c->d_metric);
  if (c->lam.p) cudaFree(c->lam.p);
  delete c;
}

}  // extern "C"
