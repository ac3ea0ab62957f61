// Sample update of Eq. (3): B1 = S12 - S11 R11^{-1} R12, B2 = S22.
// This kernel forms W11 = S11 R11^{-1} (b x b, upper triangular because S11
// and R11 are) by forward substitution over the columns of R11, one thread
// per row of S11; the host then enqueues the GEMM S12 -= W11 R12 in place in
// the sample buffer (S22 already sits below it).  If R11 has an exactly zero
// diagonal entry the formula is undefined: the kernel sets W11 = 0 and raises
// the re-sample flag, which gates that GEMM off and gates on a fresh sketch of
// the trailing matrix (an Alg. 5 step).
#include "kernels.cuh"

namespace rq {
namespace {

constexpr int W11_ROWS = 2;     // rows of W11 per CTA, one warp each
constexpr int W11_THREADS = 256;  // threads per CTA (all stage R11; W11_ROWS warps solve)
constexpr int W11_MAXQ = 4;     // columns per lane (b <= 128)

// W11 = S11 R11^{-1}: CTA c owns rows 2c, 2c + 1 of W11 (two rows per SM: the
// recurrence's FP64 FMAs of eight rows on one SM had waited on the SM's FP64
// unit at every step); R11's upper triangle and the reciprocals of its
// diagonal are staged in shared memory by the whole CTA; warp w < 2 computes
// row r of W11 left to right by the right-looking recurrence
//   W(r, j) = acc_j / R(j, j),  acc_c -= W(r, j) R(j, c) for c > j,
// with acc_c = S(r, c) initially and lane l keeping acc_c for c = l (mod 32):
// one shuffle, one multiply and a few FMAs per step, no reductions.
__global__ void w11_kernel(const double* __restrict__ S, int ell, const double* __restrict__ R,
                           int64_t ldr, int bJ, double* __restrict__ W, int* flag, int* status) {
  extern __shared__ double sm[];
  double* Rs = sm;              // bJ x bJ, ld bJ, zeros below the diagonal
  double* rinv = sm + bJ * bJ;  // bJ
  __shared__ int s_sing;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_sing = 0;
  __syncthreads();
  // 8 independent loads in flight per thread
  const int total = bJ * bJ;
  for (int e0 = tid; e0 < total; e0 += (int)blockDim.x * 8) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + u * (int)blockDim.x;
      v[u] = 0.0;
      if (e < total) {
        const int r = e % bJ, c = e / bJ;
        if (r <= c) v[u] = R[r + c * ldr];
      }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + u * (int)blockDim.x;
      if (e < total) Rs[e] = v[u];
    }
  }
  for (int j = tid; j < bJ; j += blockDim.x) {
    const double d = R[j + j * ldr];
    if (d == 0.0) s_sing = 1;
    rinv[j] = 1.0 / d;
  }
  __syncthreads();
  if (s_sing) {
    if (blockIdx.x == 0 && tid == 0) {
      *flag = 1;
      atomicOr(status, RQRCP_INFO_RESAMPLED);
    }
    // W11 = 0: a product that is not gated by the flag leaves S12 unchanged
    // for the re-sample to overwrite
    const int r = blockIdx.x * W11_ROWS + warp;
    if (warp < W11_ROWS && r < bJ)
      for (int c = lane; c < bJ; c += 32) W[r + c * bJ] = 0.0;
    return;
  }
  if (blockIdx.x == 0 && tid == 0) *flag = 0;
  const int r = blockIdx.x * W11_ROWS + warp;
  if (warp >= W11_ROWS || r >= bJ) return;
  double acc[W11_MAXQ];
#pragma unroll
  for (int q = 0; q < W11_MAXQ; ++q) {
    const int c = lane + 32 * q;
    acc[q] = (c >= r && c < bJ) ? S[r + (int64_t)c * ell] : 0.0;
  }
  for (int c = lane; c < r; c += 32) W[r + c * bJ] = 0.0;
  for (int j = r; j < bJ; ++j) {
    const int qj = j >> 5;  // warp-uniform
    double aj = 0.0;
#pragma unroll
    for (int q = 0; q < W11_MAXQ; ++q)
      if (q == qj) aj = acc[q];
    const double wj = __shfl_sync(0xffffffffu, aj, j & 31) * rinv[j];
    if (lane == (j & 31)) W[r + j * bJ] = wj;
    const double* Rj = Rs + j;  // row j: R(j, c) at Rj[c * bJ]
#pragma unroll
    for (int q = 0; q < W11_MAXQ; ++q) {
      const int c = lane + 32 * q;
      if (c > j && c < bJ) acc[q] = fma(-wj, Rj[(size_t)c * bJ], acc[q]);
    }
  }
}

}  // namespace

cudaError_t launch_w11(const double* S, int ell, const double* R11, int64_t ldr, int bJ,
                       double* W11, int* flag, int* status, cudaStream_t st) {
  if (bJ < 1 || bJ > 32 * W11_MAXQ) return cudaErrorInvalidValue;
  const size_t smem = ((size_t)bJ * bJ + (size_t)bJ) * sizeof(double);
  static std::atomic<uint64_t> attr_done{0};
  cudaError_t e = ensure_smem_attr(w11_kernel, (128 * 128 + 128) * (int)sizeof(double), attr_done);
  if (e != cudaSuccess) return e;
  const int grid = (bJ + W11_ROWS - 1) / W11_ROWS;
  w11_kernel<<<grid, W11_THREADS, smem, st>>>(S, ell, R11, ldr, bJ, W11, flag, status);
  return cudaGetLastError();
}

}  // namespace rq
