// Allocation-free nodal FP64 operator application (hdg_apply_static).
//
// hdg_apply in the nodal basis needs temporaries -- the traces in the face
// eigenbasis before and after the transformed-basis operator, and the
// D_Z^-1 tables of the requested lambdas -- which it takes from workspaces
// it grows with cudaMalloc.  This entry point runs the same kernels with all
// of those temporaries carved out of one file-scope device array, so it
// never allocates or frees device memory.
#include <mutex>
#include <string>

#include "../../include/hdg.h"
#include "internal.h"

namespace {

// 2^21 doubles = 16 MiB, reserved on every device that loads the library
// for as long as the process lives.
constexpr size_t kStaticScratchDoubles = size_t(1) << 21;
static __device__ __align__(256) double g_static_scratch[kStaticScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
double* g_scratch_addr[kMaxDevices] = {};

// Device address of the array on the current device.  Host code sees only a
// host-side stand-in under the array's name, so the address is looked up
// once per device with that device current, on the first call there.  The
// cached address belongs to that device's primary context: after
// cudaDeviceReset (which destroys the context and every module in it) the
// cache is stale, and this entry point must not be used again in the process.
hdg_status scratch_address(int dev, double** out) {
  if (dev < 0 || dev >= kMaxDevices) {
    hdg::set_last_error("hdg_apply_static: device ordinal out of range");
    return HDG_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (g_scratch_addr[dev] == nullptr) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) {
      hdg::set_last_error((std::string("hdg_apply_static: cudaGetSymbolAddress: ") + cudaGetErrorString(e)).c_str());
      return HDG_ERR_CUDA;
    }
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return HDG_OK;
}

// Lambdas travel to the device as kernel parameters (8 KB per launch, within
// the 32 KB parameter space of sm_70 and later), so no host buffer has to be
// pinned and no copy engine is involved: at most 64 launches for the largest
// batch of 65535 right-hand sides.
constexpr int kLambdaChunk = 1024;
struct LambdaChunk {
  double v[kLambdaChunk];
};

__global__ void store_lambdas(double* dst, LambdaChunk c, int count) {
  for (int i = threadIdx.x; i < count; i += blockDim.x) dst[i] = c.v[i];
}

long long round_up(long long v) { return (v + 31) / 32 * 32; }  // 256-byte multiples of doubles

hdg_status cuda_fail(cudaError_t e, const char* what) {
  hdg::set_last_error((std::string("hdg_apply_static: ") + what + ": " + cudaGetErrorString(e)).c_str());
  return HDG_ERR_CUDA;
}

}  // namespace

extern "C" hdg_status hdg_apply_static(hdg_ctx* ctx, int nrhs, const double* h_lambda, const double* d_x,
                                       double* d_y, void* stream) {
  hdg::begin_entry();
  hdg::CtxView v;
  if (!hdg::ctx_view(ctx, &v) || !h_lambda || !d_x || !d_y || nrhs < 1 || nrhs > 65535) {
    hdg::set_last_error("hdg_apply_static: NULL pointer or nrhs outside 1..65535");
    return HDG_ERR_INVALID_ARG;
  }
  if (hdg_status ls = hdg::check_lambdas(nrhs, h_lambda); ls != HDG_OK) return ls;
  const long long dzt = (long long)v.n * v.n * hdg::dz_row(v.n, sizeof(double));   // one D_Z^-1 table
  const long long trace = round_up((long long)nrhs * v.ntrace);
  const long long table = round_up((long long)nrhs * v.nclass * dzt);
  const long long need = 2 * trace + table + round_up(nrhs);
  if (need > (long long)kStaticScratchDoubles) {
    hdg::set_last_error(("hdg_apply_static: needs " + std::to_string(need) + " doubles of static scratch, the maximum is " +
                         std::to_string(kStaticScratchDoubles) + " (2 x nrhs x trace size + lambda tables); use hdg_apply")
                            .c_str());
    return HDG_ERR_INVALID_ARG;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev != v.device) {
    hdg::set_last_error("hdg_apply_static: the current device is not the context's device");
    return HDG_ERR_INVALID_ARG;
  }
  double* base = nullptr;
  hdg_status st = scratch_address(dev, &base);
  if (st != HDG_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* xh = base;
  double* yh = xh + trace;
  double* dinv = yh + trace;
  double* lam = dinv + table;

  for (int r0 = 0; r0 < nrhs; r0 += kLambdaChunk) {
    LambdaChunk c{};
    const int cnt = nrhs - r0 < kLambdaChunk ? nrhs - r0 : kLambdaChunk;
    for (int i = 0; i < cnt; ++i) c.v[i] = h_lambda[r0 + i];
    store_lambdas<<<1, 256, 0, s>>>(lam + r0, c, cnt);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "store lambdas");
  if ((e = hdg::launch_dinv<double>(v.n, lam, nrhs, v.metric64, v.nclass, v.Lambda, dinv, s)) != cudaSuccess)
    return cuda_fail(e, "D_Z^-1 tables");
  if ((e = hdg::launch_face_transform<double, double>(v.n, d_x, xh, v.mesh.nfaces, nrhs, v.ntrace, v.ntrace, v.StM,
                                                      1.0, 0, s)) != cudaSuccess)
    return cuda_fail(e, "face transform in");
  int seg = 1, nseg = 1;
  const int ppb = hdg::tpt_ppb(v.n);
  const int ctas = v.sms * hdg::tpt_blocks_per_sm<double, double>(hdg::TPT_APPLY, v.n, ppb);
  hdg::tpt_split(v.n, v.mesh.ne, nrhs, ctas, ppb, &seg, &nseg);
  // the array keeps the previous call's contents: the parts of the operator
  // output that are accumulated with atomics must start at zero (the x2/x3
  // blocks, and everything when x1-pencils are split into segments or the
  // runtime-degree kernel runs)
  const long long off = (nseg > 1 || v.n > hdg::kMaxSpecialisedN) ? 0 : v.mesh.blk[1] * (long long)v.n * v.n;
  if (v.ntrace - off > 0 &&
      (e = cudaMemset2DAsync(yh + off, sizeof(double) * v.ntrace, 0, sizeof(double) * (v.ntrace - off), nrhs, s)) !=
          cudaSuccess)
    return cuda_fail(e, "zero output");
  hdg::TptArgs<double, double> a{};
  a.mesh = v.mesh;
  a.tab = v.tab;
  a.metric = v.metric64;
  a.dinv = dinv;
  a.dinv_rhs_stride = v.nclass * dzt;
  a.lam = lam;   // the runtime-degree kernel (p > 16) computes D_Z^-1 from it
  a.x = xh;
  a.y = yh;
  a.trace_stride = v.ntrace;
  a.ppb = hdg::tpt_ppb(v.n);
  a.npencils = (long long)v.mesh.ne[1] * v.mesh.ne[2];
  a.seg = seg;
  a.nseg = nseg;
  a.max_grid = ctas;
  if ((e = hdg::launch_tpt<double, double>(hdg::TPT_APPLY, v.n, a, nrhs, s)) != cudaSuccess)
    return cuda_fail(e, "operator");
  if ((e = hdg::launch_face_transform<double, double>(v.n, yh, d_y, v.mesh.nfaces, nrhs, v.ntrace, v.ntrace, v.MS, 1.0,
                                                      0, s)) != cudaSuccess)
    return cuda_fail(e, "face transform out");
  return HDG_OK;
}
