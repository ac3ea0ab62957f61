// Sample update of Eq. (3): B1 = S12 - S11 R11^{-1} R12, B2 = S22.
// This kernel forms W11 = S11 R11^{-1} (b x b, upper triangular because S11
// and R11 are) by forward substitution over the columns of R11, one thread
// per row of S11; the host then enqueues the GEMM S12 -= W11 R12 in place in
// the sample buffer (S22 already sits below it).  If R11 has an exactly zero
// diagonal entry the formula is undefined: the kernel raises the re-sample
// flag, which gates that GEMM off and gates on a fresh sketch of the trailing
// matrix (an Alg. 5 step).
#include "kernels.cuh"

namespace rq {
namespace {

__global__ void w11_kernel(const double* __restrict__ S, int ell, const double* __restrict__ R,
                           int64_t ldr, int bJ, double* __restrict__ W, int* flag, int* status) {
  __shared__ int s_sing;
  if (threadIdx.x == 0) s_sing = 0;
  __syncthreads();
  for (int j = threadIdx.x; j < bJ; j += blockDim.x)
    if (R[j + j * ldr] == 0.0) s_sing = 1;
  __syncthreads();
  if (s_sing) {
    if (threadIdx.x == 0) {
      *flag = 1;
      atomicOr(status, RQRCP_INFO_RESAMPLED);
    }
    return;
  }
  if (threadIdx.x == 0) *flag = 0;
  for (int r = threadIdx.x; r < bJ; r += blockDim.x) {
    for (int j = 0; j < bJ; ++j) {
      double s = (r <= j) ? S[r + (int64_t)j * ell] : 0.0;
      for (int t = r; t < j; ++t) s = fma(-W[r + t * bJ], R[t + j * ldr], s);
      W[r + j * bJ] = (r <= j) ? s / R[j + j * ldr] : 0.0;
    }
  }
}

}  // namespace

cudaError_t launch_w11(const double* S, int ell, const double* R11, int64_t ldr, int bJ,
                       double* W11, int* flag, int* status, cudaStream_t st) {
  w11_kernel<<<1, 128, 0, st>>>(S, ell, R11, ldr, bJ, W11, flag, status);
  return cudaGetLastError();
}

}  // namespace rq
