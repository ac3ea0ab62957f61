// Seeded Gaussian i.i.d. matrix: the compression matrix Omega of Alg. 4
// (and re-samples of Alg. 5), from Philox4x32-10 (Salmon, Moraes, Dror and
// Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11) and the
// Box-Muller transform.  One thread per (column r, row pair q): a single
// Philox block gives the two normals of rows 2q and 2q+1.
#include "kernels.cuh"
#include "philox.cuh"

namespace rq {
namespace {

using namespace px;

__global__ void gaussian_kernel(uint2 key, uint32_t stream_id, int64_t rows, int64_t cols,
                                int64_t npairs, double* __restrict__ out, int64_t ld,
                                const int* gate) {
  if (gate != nullptr && *gate == 0) return;
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t total = npairs * cols;
  for (; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
    // pairs fastest so that a warp writes neighbouring rows of one column
    int64_t q = idx % npairs;
    int64_t r = idx / npairs;
    uint4 c = make_uint4((uint32_t)(uint64_t)r, (uint32_t)((uint64_t)r >> 32), (uint32_t)q,
                         stream_id);
    uint4 x = philox10(c, key);
    double u1 = unit_open(x.x, x.y);
    double u2 = unit_open(x.z, x.w);
    double rho = sqrt(-2.0 * log(u1));
    double s, co;
    sincospi(2.0 * u2, &s, &co);
    int64_t i0 = 2 * q;
    out[i0 + r * ld] = rho * co;
    if (i0 + 1 < rows) out[i0 + 1 + r * ld] = rho * s;
  }
}

// The same matrix stored transposed: element (i, r) at out[r + i * ld]
// (columns fastest, so a warp writes neighbouring entries of one stored column).
__global__ void gaussian_t_kernel(uint2 key, uint32_t stream_id, int64_t rows, int64_t cols,
                                  int64_t npairs, double* __restrict__ out, int64_t ld) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t total = npairs * cols;
  for (; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = idx % cols;
    int64_t q = idx / cols;
    uint4 c = make_uint4((uint32_t)(uint64_t)r, (uint32_t)((uint64_t)r >> 32), (uint32_t)q,
                         stream_id);
    uint4 x = philox10(c, key);
    double u1 = unit_open(x.x, x.y);
    double u2 = unit_open(x.z, x.w);
    double rho = sqrt(-2.0 * log(u1));
    double s, co;
    sincospi(2.0 * u2, &s, &co);
    int64_t i0 = 2 * q;
    out[r + i0 * ld] = rho * co;
    if (i0 + 1 < rows) out[r + (i0 + 1) * ld] = rho * s;
  }
}

}  // namespace

cudaError_t launch_gaussian_t(uint64_t seed, uint32_t stream_id, int64_t rows, int64_t cols,
                              double* out, int64_t ld, cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  int64_t npairs = (rows + 1) / 2;
  int64_t total = npairs * cols;
  int threads = 256;
  int64_t blocks = (total + threads - 1) / threads;
  if (blocks > 152 * 64) blocks = 152 * 64;
  uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
  gaussian_t_kernel<<<(unsigned)blocks, threads, 0, st>>>(key, stream_id, rows, cols, npairs, out,
                                                           ld);
  return cudaGetLastError();
}

cudaError_t launch_gaussian(uint64_t seed, uint32_t stream_id, int64_t rows, int64_t cols,
                            double* out, int64_t ld, const int* gate, cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  int64_t npairs = (rows + 1) / 2;
  int64_t total = npairs * cols;
  int threads = 256;
  int64_t blocks = (total + threads - 1) / threads;
  if (blocks > 152 * 64) blocks = 152 * 64;
  uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
  gaussian_kernel<<<(unsigned)blocks, threads, 0, st>>>(key, stream_id, rows, cols, npairs, out,
                                                         ld, gate);
  return cudaGetLastError();
}

}  // namespace rq
