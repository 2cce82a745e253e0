// Device helpers of the fused CG step, shared by the operator kernels that
// run it (tpt_tile.cuh, tpt_fast.cuh): the launch of iteration i + 1
// applies the CG update of iteration i to every face value it reads (the
// face value's one owner stores the updated vectors) and then the operator
// (single-reduction preconditioned CG, the iterates of Alg.
// (hdg_transformed_cg) in exact arithmetic).
#pragma once

#include "tpt_kernel.cuh"

namespace hdg {

// A CG state vector load: through L2 (ld.cg) in the persistent kernel, whose
// CTAs read values other CTAs wrote during the same launch (never a stale L1
// line); a plain load otherwise.
template <int CGM, typename T>
__device__ __forceinline__ T ld_state(const T* p) {
  if constexpr (CGM == 2) return __ldcg(p);
  else return *p;
}

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

// Generation barrier over the gridDim.x CTAs of one right-hand side row of a
// cooperative launch (every CTA resident), called by one thread per CTA after
// the CTA's memory operations were fenced.  bar[0] counts arrivals, bar[1]
// holds the number of barriers passed; the last CTA to arrive resets the
// count and advances the generation.  Every wait is bounded: after
// kBarrierSpins polls the barrier gives up, sets *err and returns 0, so a
// fault in the launch configuration ends the kernel instead of hanging it.
constexpr long long kBarrierSpins = 1LL << 20;
__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int grid_barrier(unsigned int* bar, unsigned int gen, int* err) {
  const unsigned int arrived = atomicAdd(bar, 1u);
  if (arrived == gridDim.x - 1) {
    atomicExch(bar, 0u);
    __threadfence();
    atomicExch(bar + 1, gen + 1u);
    return 1;
  }
  for (long long spin = 0; spin < kBarrierSpins; ++spin) {
    if (ld_acquire(bar + 1) != gen) {
      __threadfence();
      return 1;
    }
    __nanosleep(64);
  }
  atomicExch(err, 1);
  return 0;
}

// End of one iteration of the persistent CG kernel (every CTA): per-block
// partial sums of delta = u^T K u and gamma = r . u, one grid barrier, then
// the step scalars of the next iteration formed by every CTA from all
// partials in the same fixed order (deterministic, identical in every CTA).
// The partials are double-buffered by the parity of the iteration.  Returns
// false if the barrier gave up.
template <typename T>
__device__ __forceinline__ bool persistent_step(const CgHook& hook, const CgVecs<T>& v, int rhs, int iter, T dot,
                                                T gam, CgScalars* s_cg, unsigned int* bar_gen) {
  __shared__ double psum[2][32];
  __shared__ int ok;
  const int tid = threadIdx.x;
  const int nb = gridDim.x;
  const T dv = warp_sum(dot), gv = warp_sum(gam);
  if ((tid & 31) == 0) {
    psum[0][tid >> 5] = static_cast<double>(dv);
    psum[1][tid >> 5] = static_cast<double>(gv);
  }
  __threadfence();   // this thread's stores and reductions of the iteration
  __syncthreads();
  const long long base = ((long long)(iter & 1) * gridDim.y + rhs) * nb;
  if (tid == 0) {
    double sd = 0.0, sg = 0.0;
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) {
      sd += psum[0][w];
      sg += psum[1][w];
    }
    hook.partials[base + blockIdx.x] = 0.5 * sd;
    v.gpartials[base + blockIdx.x] = sg;
    __threadfence();
    ok = grid_barrier(v.bar + 2 * rhs, *bar_gen, v.err);
    *bar_gen += 1u;
  }
  __syncthreads();
  if (!ok) return false;
  if (tid < 32) {
    double sd = 0.0, sg = 0.0;
    for (int b = tid; b < nb; b += 32) {
      sd += __ldcg(hook.partials + base + b);
      sg += __ldcg(v.gpartials + base + b);
    }
    sd = warp_sum(sd);
    sg = warp_sum(sg);
    if (tid == 0) {
      int flag = 0;
      cg_scalars(s_cg, *s_cg, &flag, sd, sg);
    }
  }
  __syncthreads();
  return true;
}


// Asynchronous 4-byte global -> shared copy (cp.async, completion by
// cp_async_wait_all in the issuing thread); `valid` false zero-fills the
// destination without reading the source.
__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool valid) {
  const unsigned int sa = static_cast<unsigned int>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(sa), "l"(src), "r"(valid ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

}  // namespace hdg
