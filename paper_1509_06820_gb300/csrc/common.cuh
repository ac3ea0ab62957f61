// Shared device-side helpers for the RQRCP kernels: status words, a bounded
// software grid barrier for cooperative launches, small reductions.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/rqrcp.h"

namespace rq {

// Device status word layout (one int in the handle's workspace):
//   0                       -> ok
//   RQRCP_INFO_RESAMPLED    -> an exactly singular R11 forced a re-sample
//   RQRCP_INFO_TIMEOUT      -> a grid barrier gave up waiting
//   RQRCP_INFO_NONFINITE    -> the sample held NaN or Inf
// Several conditions OR together.

// Grid barrier state; one per concurrently running cooperative kernel.
struct GridBarrier {
  unsigned int count;
  unsigned int gen;
  unsigned int abort;
  unsigned int pad;
};

// Upper bound on the polls of one barrier wait.  A healthy barrier on a
// GB300 completes in a few microseconds; this bound is ~1 s of polling.
constexpr unsigned int kBarrierMaxPolls = 1u << 23;

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_u32(unsigned int* p, unsigned int v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// All CTAs of a cooperative launch call this.  Returns false when the wait
// ran out (or another CTA already gave up): the status word then carries
// RQRCP_INFO_TIMEOUT and the caller must return without further barriers.
__device__ __forceinline__ bool grid_barrier(GridBarrier* bar, unsigned int nblocks, int* status) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    unsigned int g = ld_acquire_u32(&bar->gen);
    __threadfence();
    unsigned int arrived = atomicAdd(&bar->count, 1u);
    if (arrived == nblocks - 1) {
      atomicExch(&bar->count, 0u);
      __threadfence();
      st_release_u32(&bar->gen, g + 1);
    } else {
      unsigned int polls = 0;
      while (ld_acquire_u32(&bar->gen) == g) {
        if (ld_acquire_u32(&bar->abort)) { ok = 0; break; }
        if (++polls > kBarrierMaxPolls) {
          atomicExch(&bar->abort, 1u);
          atomicOr(status, RQRCP_INFO_TIMEOUT);
          ok = 0;
          break;
        }
        if (polls > 64) __nanosleep(64);
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

__host__ __device__ __forceinline__ int64_t imax64(int64_t a, int64_t b) { return a > b ? a : b; }
__host__ __device__ __forceinline__ int64_t imin64(int64_t a, int64_t b) { return a < b ? a : b; }

template <int W>
__device__ __forceinline__ double group_sum(double v) {
#pragma unroll
  for (int o = W / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_sum(double v) { return group_sum<32>(v); }

// LAPACK-convention reflector scalars from alpha = x_0 and the 2-norm of the
// tail x_1..: beta = -sign(alpha) ||x|| (sign(+-0) = +), tau = (beta-alpha)/beta,
// scale = 1/(alpha-beta) multiplies the tail into v.  A zero tail gives the
// identity (tau = 0, beta = alpha, scale = 0).
__device__ __forceinline__ void house_scalars(double alpha, double xnorm, double* beta,
                                              double* tau, double* scale) {
  if (xnorm == 0.0) {
    *beta = alpha;
    *tau = 0.0;
    *scale = 0.0;
    return;
  }
  double h = hypot(alpha, xnorm);
  double bb = (alpha >= 0.0) ? -h : h;
  *beta = bb;
  *tau = (bb - alpha) / bb;
  *scale = 1.0 / (alpha - bb);
}

}  // namespace rq
