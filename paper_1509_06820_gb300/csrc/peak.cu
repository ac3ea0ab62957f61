// Arithmetic-peak probes (instrumentation; the paper has no counterpart).
//
// They measure the rates that bound the FP64 kernels of this library on the
// GPU they run on, so that a roofline fraction is read against a measured
// figure rather than a datasheet one:
//   kind 0  FP64 FMA on the CUDA cores (the pipe of the FP64 GEMM, panel,
//           sample QRCP): every thread runs kChains independent FMA chains
//   kind 1  FP64 tensor-core MMA, mma.sync m8n8k4 (DMMA)
//   kind 2  FP64 tensor-core MMA, mma.sync m16n8k16
//   kind 3  FP32 FMA on the CUDA cores
//   kind 4  FP64 FMA in the register-blocked outer-product pattern of a GEMM
// Each launch is `grid` CTAs of 256 threads; `iters` rounds per thread or
// warp.  Each thread writes the sum of its accumulators to sink[global id],
// so no chain can be dropped by the compiler.
#include "kernels.cuh"

namespace rq {
namespace {

constexpr int kPeakThreads = 256;
constexpr int kChains = 8;

template <typename T>
__global__ void __launch_bounds__(kPeakThreads) fma_chain_kernel(int64_t iters, T a, T c, T* sink) {
  T x[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) x[j] = (T)(threadIdx.x + j) * (T)1e-3;
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int j = 0; j < kChains; ++j) x[j] = fma(x[j], a, c);
  }
  T s = 0;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += x[j];
  sink[(int64_t)blockIdx.x * kPeakThreads + threadIdx.x] = s;
}

// D = A B + D on the FP64 tensor cores, 4 independent accumulator tiles per
// warp (m8n8k4: A 1, B 1, C/D 2 doubles per lane).
__global__ void __launch_bounds__(kPeakThreads) dmma_m8n8k4_kernel(int64_t iters, double* sink) {
  const double a = 1e-3 * (threadIdx.x & 7), b = 1e-3 * ((threadIdx.x >> 3) & 3);
  double d[4][2];
#pragma unroll
  for (int t = 0; t < 4; ++t) d[t][0] = d[t][1] = 0.0;
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int t = 0; t < 4; ++t)
      asm volatile(
          "mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};\n"
          : "+d"(d[t][0]), "+d"(d[t][1])
          : "d"(a), "d"(b));
  }
  double s = 0.0;
#pragma unroll
  for (int t = 0; t < 4; ++t) s += d[t][0] + d[t][1];
  sink[(int64_t)blockIdx.x * kPeakThreads + threadIdx.x] = s;
}

// m16n8k16: A 8, B 4, C/D 4 doubles per lane; 2 independent tiles per warp.
__global__ void __launch_bounds__(kPeakThreads) dmma_m16n8k16_kernel(int64_t iters, double* sink) {
  double a[8], b[4], d[2][4];
#pragma unroll
  for (int j = 0; j < 8; ++j) a[j] = 1e-3 * ((threadIdx.x + j) & 7);
#pragma unroll
  for (int j = 0; j < 4; ++j) b[j] = 1e-3 * ((threadIdx.x + 3 * j) & 3);
#pragma unroll
  for (int t = 0; t < 2; ++t)
#pragma unroll
    for (int j = 0; j < 4; ++j) d[t][j] = 0.0;
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int t = 0; t < 2; ++t)
      asm volatile(
          "mma.sync.aligned.m16n8k16.row.col.f64.f64.f64.f64 {%0, %1, %2, %3}, "
          "{%4, %5, %6, %7, %8, %9, %10, %11}, {%12, %13, %14, %15}, {%0, %1, %2, %3};\n"
          : "+d"(d[t][0]), "+d"(d[t][1]), "+d"(d[t][2]), "+d"(d[t][3])
          : "d"(a[0]), "d"(a[1]), "d"(a[2]), "d"(a[3]), "d"(a[4]), "d"(a[5]), "d"(a[6]),
            "d"(a[7]), "d"(b[0]), "d"(b[1]), "d"(b[2]), "d"(b[3]));
  }
  double s = 0.0;
#pragma unroll
  for (int t = 0; t < 2; ++t) s += d[t][0] + d[t][1] + d[t][2] + d[t][3];
  sink[(int64_t)blockIdx.x * kPeakThreads + threadIdx.x] = s;
}

// The register-blocked outer product of a GEMM's inner loop: 4 x 4
// accumulators per thread updated from 4 + 4 operands that change every
// round (16 independent FMA chains, operands in distinct registers).
__global__ void __launch_bounds__(kPeakThreads) fma_outer_kernel(int64_t iters, double* sink) {
  double a[4], b[4], c[4][4];
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    a[x] = 1e-3 * (threadIdx.x + x);
    b[x] = 1e-3 * (threadIdx.x - x);
#pragma unroll
    for (int y = 0; y < 4; ++y) c[x][y] = 0.0;
  }
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) c[x][y] = fma(a[x], b[y], c[x][y]);
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      a[x] = fma(a[x], 0.999999, 1e-7);
      b[x] = fma(b[x], 0.999999, -1e-7);
    }
  }
  double s = 0.0;
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) s += c[x][y];
  sink[(int64_t)blockIdx.x * kPeakThreads + threadIdx.x] = s;
}

}  // namespace
}  // namespace rq

extern "C" int rqrcp_peak_probe(int kind, int64_t iters, int grid, void* d_sink, void* cuda_stream,
                                double* flops) {
  using namespace rq;
  if (kind < 0 || kind > 4) return -1;
  if (iters < 1) return -2;
  if (grid < 1) return -3;
  if (!d_sink) return -4;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const double threads = (double)grid * kPeakThreads;
  const double warps = threads / 32.0;
  double fl = 0.0;
  switch (kind) {
    case 0:
      fma_chain_kernel<double><<<grid, kPeakThreads, 0, st>>>(iters, 0.999999, 1e-6,
                                                              static_cast<double*>(d_sink));
      fl = threads * (double)iters * 4.0 * kChains * 2.0;
      break;
    case 1:
      dmma_m8n8k4_kernel<<<grid, kPeakThreads, 0, st>>>(iters, static_cast<double*>(d_sink));
      fl = warps * (double)iters * 4.0 * (2.0 * 8 * 8 * 4);
      break;
    case 2:
      dmma_m16n8k16_kernel<<<grid, kPeakThreads, 0, st>>>(iters, static_cast<double*>(d_sink));
      fl = warps * (double)iters * 2.0 * (2.0 * 16 * 8 * 16);
      break;
    case 4:
      fma_outer_kernel<<<grid, kPeakThreads, 0, st>>>(iters, static_cast<double*>(d_sink));
      fl = threads * (double)iters * (16.0 + 8.0) * 2.0;
      break;
    default:
      fma_chain_kernel<float><<<grid, kPeakThreads, 0, st>>>(iters, 0.999999f, 1e-6f,
                                                             static_cast<float*>(d_sink));
      fl = threads * (double)iters * 4.0 * kChains * 2.0;
      break;
  }
  if (flops) *flops = fl;
  return cudaGetLastError() == cudaSuccess ? RQRCP_OK : RQRCP_ERR_CUDA;
}
