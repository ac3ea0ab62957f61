// FP64 GEMM on the CUDA cores: C = alpha op(A) op(B) + beta C, column-major.
//
// On the GB300 the FP64 rate of the FMA pipe and of the FP64 mma.sync path
// measure the same (about 1.0 TFLOP/s), so this kernel is a plain
// register-blocked FFMA GEMM: a 64x64 tile per CTA, k-slices of 16 staged in
// shared memory, a 4x4 register tile per thread.  It serves the sketch
// B = Omega A (Alg. 4), the block-reflector products of the trailing update
// W = T^T (Y^T A2) and A2 -= Y W (Sec. 2.2), the sample update
// S12 - W11 R12 (Eq. 3) and the TRQRCP/TUXV products (Alg. 6, Alg. 7).
// Split-K writes deterministic partial sums that a second kernel adds in a
// fixed order.
#include <algorithm>

#include "kernels.cuh"

namespace rq {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

template <char TA, int AMODE>
__device__ __forceinline__ double load_a(const double* __restrict__ A, int64_t lda, int64_t M,
                                         int64_t K, int64_t i, int64_t kk) {
  if (i >= M || kk >= K) return 0.0;
  // stored-matrix coordinates (r, c) of op(A)(i, kk)
  int64_t r = (TA == 'N') ? i : kk;
  int64_t c = (TA == 'N') ? kk : i;
  if (AMODE == 1) {
    if (r < c) return 0.0;
    if (r == c) return 1.0;
  } else if (AMODE == 2) {
    if (r > c) return 0.0;
  }
  return A[r + c * lda];
}

template <char TB>
__device__ __forceinline__ double load_b(const double* __restrict__ B, int64_t ldb, int64_t K,
                                         int64_t N, int64_t kk, int64_t j,
                                         const int64_t* __restrict__ bcols) {
  if (kk >= K || j >= N) return 0.0;
  if (TB == 'N') return B[kk + (bcols != nullptr ? bcols[j] : j) * ldb];
  return B[j + kk * ldb];
}

// One staged k-slice into the 4 x 4 register tile: rows tx + 16a for a < NA
// (NA = 1 for a tile whose live rows all fall in a = 0, so that a ragged
// last row tile -- e.g. rows 64..71 of the l = 72 sketch -- issues a quarter
// of the FP64 FMAs instead of computing on zeros), columns ty + 16c.
template <int NA>
__device__ __forceinline__ void fma_slice(const double (*As)[BM], const double (*Bs)[BN], int tx,
                                          int ty, double (&acc)[4][4]) {
#pragma unroll
  for (int kk = 0; kk < BK; ++kk) {
    double av[NA], bv[4];
#pragma unroll
    for (int a = 0; a < NA; ++a) av[a] = As[kk][tx + 16 * a];
#pragma unroll
    for (int c = 0; c < 4; ++c) bv[c] = Bs[kk][ty + 16 * c];
#pragma unroll
    for (int a = 0; a < NA; ++a)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][c] = fma(av[a], bv[c], acc[a][c]);
  }
}

template <char TA, char TB, int AMODE>
__global__ void __launch_bounds__(NT) gemm_kernel(GemmArgs g, int64_t kchunk, double* partial) {
  if (g.gate != nullptr && *g.gate != g.gate_run) return;
  __shared__ double As[BK][BM];
  __shared__ double Bs[BK][BN];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int64_t i0 = (int64_t)blockIdx.x * BM;
  const int64_t j0 = (int64_t)blockIdx.y * BN;
  const int64_t kbeg = (int64_t)blockIdx.z * kchunk;
  const int64_t kend = imin64(g.K, kbeg + kchunk);
  const bool thin = g.M - i0 <= 16;  // the same for the whole CTA

  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[a][c] = 0.0;

  for (int64_t k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int li, lk;
      if (TA == 'N') { li = tid % 64; lk = tid / 64 + 4 * r; }
      else { lk = tid % 16; li = tid / 16 + 16 * r; }
      As[lk][li] = load_a<TA, AMODE>(g.A, g.lda, g.M, kend, i0 + li, k0 + lk);
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int lj, lk;
      if (TB == 'N') { lk = tid % 16; lj = tid / 16 + 16 * r; }
      else { lj = tid % 64; lk = tid / 64 + 4 * r; }
      Bs[lk][lj] = load_b<TB>(g.B, g.ldb, kend, g.N, k0 + lk, j0 + lj, g.bcols);
    }
    __syncthreads();
    if (thin)
      fma_slice<1>(As, Bs, tx, ty, acc);
    else
      fma_slice<4>(As, Bs, tx, ty, acc);
    __syncthreads();
  }

#pragma unroll
  for (int a = 0; a < 4; ++a) {
    int64_t i = i0 + tx + 16 * a;
    if (i >= g.M) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      int64_t j = j0 + ty + 16 * c;
      if (j >= g.N) continue;
      if (partial != nullptr) {
        partial[(int64_t)blockIdx.z * g.M * g.N + i + j * g.M] = g.alpha * acc[a][c];
      } else {
        double* cp = g.C + i + j * g.ldc;
        double v = g.alpha * acc[a][c];
        if (g.beta != 0.0) v = fma(g.beta, *cp, v);
        *cp = v;
      }
    }
  }
}

__global__ void splitk_reduce(GemmArgs g, int splits, const double* __restrict__ partial) {
  if (g.gate != nullptr && *g.gate != g.gate_run) return;
  int64_t total = g.M * g.N;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int z = 0; z < splits; ++z) s += partial[(int64_t)z * total + e];
    int64_t i = e % g.M, j = e / g.M;
    double* cp = g.C + i + j * g.ldc;
    if (g.beta != 0.0) s = fma(g.beta, *cp, s);
    *cp = s;
  }
}

template <char TA, char TB>
cudaError_t dispatch_amode(const GemmArgs& g, dim3 grid, int64_t kchunk, double* partial,
                           cudaStream_t st) {
  switch (g.amode) {
    case 0: gemm_kernel<TA, TB, 0><<<grid, NT, 0, st>>>(g, kchunk, partial); break;
    case 1: gemm_kernel<TA, TB, 1><<<grid, NT, 0, st>>>(g, kchunk, partial); break;
    default: gemm_kernel<TA, TB, 2><<<grid, NT, 0, st>>>(g, kchunk, partial); break;
  }
  return cudaGetLastError();
}

}  // namespace

// Split-K factor: the FP64 pipe is the bottleneck, so pick the factor whose
// CTA count fills whole waves of the resident slots (4 CTAs per SM at 64
// registers x 256 threads) best, keeping at least 256 of K per split.
int gemm_pick_splits(int64_t M, int64_t N, int64_t K, int num_sms) {
  const int64_t tiles = ((M + BM - 1) / BM) * ((N + BN - 1) / BN);
  const int64_t slots = 4LL * num_sms;
  if (tiles >= 8 * slots) return 1;
  const int64_t kmax = std::max<int64_t>(1, std::min<int64_t>(64, K / 256));
  int best = 1;
  double best_eff = 0.0;
  for (int64_t s = 1; s <= kmax; ++s) {
    const int64_t ctas = tiles * s;
    const int64_t waves = (ctas + slots - 1) / slots;
    const double eff = (double)ctas / (double)(waves * slots);
    if (eff > best_eff + 0.02) {
      best_eff = eff;
      best = (int)s;
    }
  }
  return best;
}

cudaError_t launch_gemm(const GemmArgs& g, int splits, double* partial, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0) return cudaSuccess;
  if (g.K <= 0) {
    // no k-slices: the epilogue alone gives C = beta C
    dim3 grid((unsigned)((g.M + BM - 1) / BM), (unsigned)((g.N + BN - 1) / BN), 1);
    GemmArgs z = g;
    z.K = 0;
    gemm_kernel<'N', 'N', 0><<<grid, NT, 0, st>>>(z, BK, nullptr);
    return cudaGetLastError();
  }
  if (splits < 1 || partial == nullptr) splits = 1;
  int64_t kchunk = (g.K + splits - 1) / splits;
  kchunk = ((kchunk + BK - 1) / BK) * BK;
  splits = (int)((g.K + kchunk - 1) / kchunk);
  dim3 grid((unsigned)((g.M + BM - 1) / BM), (unsigned)((g.N + BN - 1) / BN), (unsigned)splits);
  double* part = splits > 1 ? partial : nullptr;
  cudaError_t e;
  if (g.transA == 'N' && g.transB == 'N') e = dispatch_amode<'N', 'N'>(g, grid, kchunk, part, st);
  else if (g.transA == 'N') e = dispatch_amode<'N', 'T'>(g, grid, kchunk, part, st);
  else if (g.transB == 'N') e = dispatch_amode<'T', 'N'>(g, grid, kchunk, part, st);
  else e = dispatch_amode<'T', 'T'>(g, grid, kchunk, part, st);
  if (e != cudaSuccess || splits == 1) return e;
  int64_t total = g.M * g.N;
  int blocks = (int)imin64((total + 255) / 256, 152 * 16);
  splitk_reduce<<<blocks, 256, 0, st>>>(g, splits, partial);
  return cudaGetLastError();
}

}  // namespace rq
