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

constexpr int W11_ROWS = 8;  // rows of W11 per CTA, one warp each

// W11 = S11 R11^{-1}: CTA c owns rows 8c..8c+7 of W11; R11 (columns >= the
// CTA's first row) is staged in shared memory; warp w computes row r of W11
// left to right, W(r, j) = (S(r, j) - sum_{r <= t < j} W(r, t) R(t, j)) / R(j, j),
// its lanes splitting the sum over t (fixed-order shuffle reduction).
__global__ void w11_kernel(const double* __restrict__ S, int ell, const double* __restrict__ R,
                           int64_t ldr, int bJ, double* __restrict__ W, int* flag, int* status) {
  extern __shared__ double sm[];
  double* Rs = sm;                    // bJ x bJ, ld bJ
  double* Wr = sm + bJ * bJ;          // W11_ROWS x bJ
  __shared__ int s_sing;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_sing = 0;
  __syncthreads();
  for (int e = tid; e < bJ * bJ; e += blockDim.x) {
    const int r = e % bJ, c = e / bJ;
    Rs[e] = (r <= c) ? R[r + c * ldr] : 0.0;
  }
  for (int j = tid; j < bJ; j += blockDim.x)
    if (R[j + j * ldr] == 0.0) s_sing = 1;
  __syncthreads();
  if (s_sing) {
    if (blockIdx.x == 0 && tid == 0) {
      *flag = 1;
      atomicOr(status, RQRCP_INFO_RESAMPLED);
    }
    return;
  }
  if (blockIdx.x == 0 && tid == 0) *flag = 0;
  const int r = blockIdx.x * W11_ROWS + warp;
  if (r >= bJ) return;
  double* wrow = Wr + warp * bJ;
  for (int j = lane; j < bJ; j += 32) wrow[j] = 0.0;
  __syncwarp();
  for (int j = r; j < bJ; ++j) {
    double s = 0.0;
    for (int t = r + lane; t < j; t += 32) s = fma(wrow[t], Rs[t + j * bJ], s);
    s = warp_sum(s);
    if (lane == 0) wrow[j] = (S[r + (int64_t)j * ell] - s) / Rs[j + j * bJ];
    __syncwarp();
  }
  for (int j = lane; j < bJ; j += 32) W[r + j * bJ] = wrow[j];
}

}  // namespace

cudaError_t launch_w11(const double* S, int ell, const double* R11, int64_t ldr, int bJ,
                       double* W11, int* flag, int* status, cudaStream_t st) {
  const size_t smem = ((size_t)bJ * bJ + (size_t)W11_ROWS * bJ) * sizeof(double);
  static std::atomic<uint64_t> attr_done{0};
  cudaError_t e = ensure_smem_attr(w11_kernel, (128 * 128 + W11_ROWS * 128) * (int)sizeof(double),
                                   attr_done);
  if (e != cudaSuccess) return e;
  const int grid = (bJ + W11_ROWS - 1) / W11_ROWS;
  w11_kernel<<<grid, 32 * W11_ROWS, smem, st>>>(S, ell, R11, ldr, bJ, W11, flag, status);
  return cudaGetLastError();
}

}  // namespace rq
