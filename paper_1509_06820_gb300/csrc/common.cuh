// Shared device-side helpers for the RQRCP kernels: status words, a bounded
// software grid barrier for cooperative launches, small reductions.
#pragma once

#include <atomic>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/rqrcp.h"

namespace rq {

// Raise a kernel's dynamic shared-memory limit to `bytes` on the current
// device, once per device (the attribute belongs to the device, and several
// host threads may launch): `done` keeps one bit per device ordinal < 64.
template <typename Kernel>
inline cudaError_t ensure_smem_attr(Kernel kernel, int bytes, std::atomic<uint64_t>& done) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const uint64_t bit = dev < 64 ? (uint64_t{1} << dev) : 0;
  if (bit != 0 && (done.load(std::memory_order_acquire) & bit) != 0) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess && bit != 0) done.fetch_or(bit, std::memory_order_acq_rel);
  return e;
}

// Device status word layout (one int in the handle's workspace):
//   0                       -> ok
//   RQRCP_INFO_RESAMPLED    -> an exactly singular R11 forced a re-sample
//   RQRCP_INFO_TIMEOUT      -> a grid barrier gave up waiting
//   RQRCP_INFO_NONFINITE    -> the sample held NaN or Inf
// Several conditions OR together.

// Grid barrier state; one per concurrently running cooperative kernel.  The
// launcher zeroes it before every launch.  `count` only grows during a launch:
// barrier k of a grid of G CTAs is complete once count >= k G.
struct GridBarrier {
  unsigned int count;
  unsigned int unused;
  unsigned int abort;
  unsigned int pad;
};

// Upper bound on the polls of one barrier wait.  A healthy barrier on a
// GB300 completes in a few microseconds; this bound is ~1 s of polling.
constexpr unsigned int kBarrierMaxPolls = 1u << 23;
// Poll bound of the test-only phantom-CTA barrier (RQRCP_OPT_TEST_BARRIER_TIMEOUT):
// a few milliseconds, so that a wait that cannot complete ends quickly.
constexpr unsigned int kBarrierTestPolls = 1u << 14;

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned int atom_add_release_u32(unsigned int* p, unsigned int v) {
  unsigned int old;
  asm volatile("atom.add.release.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

// All CTAs of a cooperative launch call this.  Thread 0 arrives with one
// release-ordered atomic add (its return value tells which barrier this is)
// and polls the counter with acquire loads until the whole grid has arrived.
// Returns false when the wait ran out (or another CTA already gave up): the
// status word then carries RQRCP_INFO_TIMEOUT and the caller must return
// without further barriers.  `nblocks` is the number of arrivals that
// complete a barrier (the grid size; more only in the test of the timeout
// path) and `max_polls` bounds the wait of each CTA.
__device__ __forceinline__ bool grid_barrier(GridBarrier* bar, unsigned int nblocks, int* status,
                                             unsigned int max_polls = kBarrierMaxPolls) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    __threadfence();
    const unsigned int old = atom_add_release_u32(&bar->count, 1u);
    const unsigned int target = (old / nblocks + 1u) * nblocks;
    unsigned int polls = 0;
    while ((int)(ld_acquire_u32(&bar->count) - target) < 0) {
      if (ld_acquire_u32(&bar->abort)) { ok = 0; break; }
      if (++polls > max_polls) {
        atomicExch(&bar->abort, 1u);
        atomicOr(status, RQRCP_INFO_TIMEOUT);
        ok = 0;
        break;
      }
      if (polls > 256) __nanosleep(32);
    }
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

// The same scalars from alpha and the squared tail norm sigma2 = ||x_1..||^2:
// beta = -sign(alpha) sqrt(alpha^2 + sigma2) (one square root instead of a
// square root and a scaled hypot; sigma2 is itself a sum of squares, so the
// unscaled form adds no overflow that the caller has not already risked).
__device__ __forceinline__ void house_scalars_sq(double alpha, double sigma2, double* beta,
                                                 double* tau, double* scale) {
  if (sigma2 == 0.0) {
    *beta = alpha;
    *tau = 0.0;
    *scale = 0.0;
    return;
  }
  const double h = sqrt(fma(alpha, alpha, sigma2));
  const double bb = (alpha >= 0.0) ? -h : h;
  *beta = bb;
  *tau = (bb - alpha) / bb;
  *scale = 1.0 / (alpha - bb);
}

}  // namespace rq
