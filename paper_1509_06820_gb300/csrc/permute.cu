// Column permutation of one block (Alg. 4: permute A^[J-1] and the completed
// rows of R with P_b^[J]) plus small utility kernels.
//
// The b swaps chosen on the sample (position i <-> swaps[i], in order) are
// composed on the device into at most 2b (destination, source) moves; whole
// columns (all m rows, so completed rows of R move too) are gathered into
// scratch and scattered back, 16-byte vectorised when the layout allows.
// jpvt moves alongside.  The pivot list never leaves the device.
#include <algorithm>
#include <cstdint>

#include "kernels.cuh"

namespace rq {
namespace {

// map layout: map[0] = number of moves; moves at map[1 + 2t] (dest), map[2 + 2t] (src);
// the jpvt staging buffer follows at map[1 + 8*steps].
constexpr int kMaxSwapSteps = 128;  // the largest block size

__global__ void compose_swaps(const int64_t* __restrict__ swaps, int steps, int64_t* map) {
  // touched positions and the original position each holds, in shared
  // memory; one warp: the lanes search the touched list together
  __shared__ int64_t pos[2 * kMaxSwapSteps];
  __shared__ int64_t content[2 * kMaxSwapSteps];
  __shared__ int64_t sw[kMaxSwapSteps];
  if (blockIdx.x != 0 || threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  // the whole swap list in one round of loads (the loop below is sequential)
  for (int t = lane; t < steps; t += 32) sw[t] = swaps[t];
  __syncwarp();
  int ntouch = 0;  // identical in every lane
  for (int i = 0; i < steps; ++i) {
    const int64_t s = sw[i];
    if (s == i) continue;
    int ia = -1, ib = -1;  // positions are unique in pos[]: at most one hit each
    for (int t0 = 0; t0 < ntouch; t0 += 32) {
      const int t = t0 + lane;
      const int64_t p = t < ntouch ? pos[t] : -1;
      const unsigned ma = __ballot_sync(0xffffffffu, t < ntouch && p == i);
      const unsigned mb = __ballot_sync(0xffffffffu, t < ntouch && p == s);
      if (ma != 0u) ia = t0 + __ffs(ma) - 1;
      if (mb != 0u) ib = t0 + __ffs(mb) - 1;
    }
    if (ia < 0) {
      if (lane == 0) {
        pos[ntouch] = i;
        content[ntouch] = i;
      }
      ia = ntouch++;
    }
    if (ib < 0) {
      if (lane == 0) {
        pos[ntouch] = s;
        content[ntouch] = s;
      }
      ib = ntouch++;
    }
    __syncwarp();
    if (lane == 0) {
      const int64_t tmp = content[ia];
      content[ia] = content[ib];
      content[ib] = tmp;
    }
    __syncwarp();
  }
  // moved entries, in the order they were first touched
  int nm = 0;
  for (int t0 = 0; t0 < ntouch; t0 += 32) {
    const int t = t0 + lane;
    const bool mv = t < ntouch && content[t] != pos[t];
    const unsigned m = __ballot_sync(0xffffffffu, mv);
    if (mv) {
      const int k = nm + __popc(m & ((1u << lane) - 1u));
      map[1 + 2 * k] = pos[t];
      map[2 + 2 * k] = content[t];
    }
    nm += __popc(m);
  }
  if (lane == 0) map[0] = nm;
}

// gather (dir = 0): buf[:, t] = A[:, col0 + src_t]; scatter (dir = 1):
// A[:, col0 + dest_t] = buf[:, t].  blockIdx.y = move index.  V is a 16-byte
// vector of T (double2 or float4) used when the layout allows.
template <typename T, typename V, bool VEC>
__global__ void move_columns(T* __restrict__ A, int64_t lda, int64_t m, int64_t col0,
                             const int64_t* __restrict__ map, T* __restrict__ buf,
                             int64_t* __restrict__ jpvt, int64_t* __restrict__ jbuf, int dir) {
  constexpr int W = sizeof(V) / sizeof(T);
  const int t = blockIdx.y;
  if (t >= map[0]) return;
  const int64_t dest = map[1 + 2 * t], src = map[2 + 2 * t];
  const int64_t acol = col0 + (dir == 0 ? src : dest);
  T* a = A + acol * lda;
  T* bb = buf + (int64_t)t * m;
  if (VEC) {
    const int64_t mv = m / W;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < mv;
         r += (int64_t)gridDim.x * blockDim.x) {
      if (dir == 0) reinterpret_cast<V*>(bb)[r] = reinterpret_cast<const V*>(a)[r];
      else reinterpret_cast<V*>(a)[r] = reinterpret_cast<const V*>(bb)[r];
    }
    if (blockIdx.x == 0 && threadIdx.x < (unsigned)(m - mv * W)) {
      const int64_t r = mv * W + threadIdx.x;
      if (dir == 0) bb[r] = a[r];
      else a[r] = bb[r];
    }
  } else {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < m;
         r += (int64_t)gridDim.x * blockDim.x) {
      if (dir == 0) bb[r] = a[r];
      else a[r] = bb[r];
    }
  }
  if (jpvt != nullptr && blockIdx.x == 0 && threadIdx.x == 0) {
    if (dir == 0) jbuf[t] = jpvt[col0 + src];
    else jpvt[col0 + dest] = jbuf[t];
  }
}

__global__ void iota_kernel(int64_t* v, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    v[i] = i;
}

__global__ void fill_kernel(double* X, int64_t rows, int64_t cols, int64_t ld, double v) {
  const int64_t total = rows * cols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x)
    X[(e % rows) + (e / rows) * ld] = v;
}

__global__ void copy2d_kernel(const double* __restrict__ src, int64_t lds, double* __restrict__ dst,
                              int64_t ldd, int64_t rows, int64_t cols) {
  const int64_t total = rows * cols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e % rows, c = e / rows;
    dst[r + c * ldd] = src[r + c * lds];
  }
}

unsigned grid_for(int64_t work, int threads, int64_t cap) {
  int64_t b = (work + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (unsigned)b;
}

template <typename T, typename V>
cudaError_t apply_swaps_t(T* A, int64_t lda, int64_t m, int64_t col0, const int64_t* swaps,
                          int steps, int64_t* jpvt, int64_t* map, T* buf, cudaStream_t st) {
  if (steps <= 0) return cudaSuccess;
  if (steps > kMaxSwapSteps) return cudaErrorInvalidValue;
  compose_swaps<<<1, 32, 0, st>>>(swaps, steps, map);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  constexpr int W = sizeof(V) / sizeof(T);
  int64_t* jbuf = map + 1 + 8 * (int64_t)steps;
  const bool vec = (lda % W == 0) && ((reinterpret_cast<uintptr_t>(A) & 15) == 0) &&
                   ((reinterpret_cast<uintptr_t>(buf) & 15) == 0) && (m % W == 0);
  const int threads = 256;
  dim3 grid(grid_for(vec ? m / W : m, threads, 64), (unsigned)(2 * steps));
  for (int dir = 0; dir < 2; ++dir) {
    if (vec) move_columns<T, V, true><<<grid, threads, 0, st>>>(A, lda, m, col0, map, buf, jpvt, jbuf, dir);
    else move_columns<T, V, false><<<grid, threads, 0, st>>>(A, lda, m, col0, map, buf, jpvt, jbuf, dir);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace

cudaError_t launch_apply_swaps(double* A, int64_t lda, int64_t m, int64_t col0,
                               const int64_t* swaps, int steps, int64_t* jpvt, int64_t* map,
                               double* buf, cudaStream_t st) {
  return apply_swaps_t<double, double2>(A, lda, m, col0, swaps, steps, jpvt, map, buf, st);
}

cudaError_t launch_apply_swaps_f32(float* A, int64_t lda, int64_t m, int64_t col0,
                                   const int64_t* swaps, int steps, int64_t* jpvt, int64_t* map,
                                   float* buf, cudaStream_t st) {
  return apply_swaps_t<float, float4>(A, lda, m, col0, swaps, steps, jpvt, map, buf, st);
}

cudaError_t launch_iota(int64_t* v, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  iota_kernel<<<grid_for(n, 256, 1024), 256, 0, st>>>(v, n);
  return cudaGetLastError();
}

cudaError_t launch_fill(double* X, int64_t rows, int64_t cols, int64_t ld, double v,
                        cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  fill_kernel<<<grid_for(rows * cols, 256, 152 * 16), 256, 0, st>>>(X, rows, cols, ld, v);
  return cudaGetLastError();
}

cudaError_t launch_copy2d(const double* src, int64_t lds, double* dst, int64_t ldd,
                          int64_t rows, int64_t cols, cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  copy2d_kernel<<<grid_for(rows * cols, 256, 152 * 16), 256, 0, st>>>(src, lds, dst, ldd, rows,
                                                                        cols);
  return cudaGetLastError();
}

}  // namespace rq

namespace rq {
namespace {

__global__ void gather_cols_kernel(const double* __restrict__ src, int64_t lds, int64_t r0,
                                   int64_t rows, const int64_t* __restrict__ idx, int64_t ncols,
                                   double* __restrict__ dst, int64_t ldd) {
  const int64_t total = rows * ncols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e % rows, t = e / rows;
    dst[r + t * ldd] = src[(r0 + r) + idx[t] * lds];
  }
}

__global__ void scatter_transpose_kernel(const double* __restrict__ src, int64_t lds, int64_t rows,
                                         const int64_t* __restrict__ idx, int64_t ncols,
                                         double* __restrict__ dst, int64_t ldd) {
  const int64_t total = rows * ncols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e % rows, c = e / rows;
    dst[idx[c] + r * ldd] = src[r + c * lds];
  }
}

__global__ void split_qr_kernel(const double* __restrict__ F, int64_t ldf, int64_t rows,
                                int64_t cols, int64_t yrow0, double* __restrict__ Y, int64_t ldy,
                                double* __restrict__ R, int64_t ldr) {
  const int64_t total = rows * cols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e % rows, c = e / rows;
    const double f = F[r + c * ldf];
    if (Y != nullptr) Y[(yrow0 + r) + c * ldy] = (r > c) ? f : (r == c ? 1.0 : 0.0);
    if (R != nullptr && r < cols) R[r + c * ldr] = (r <= c) ? f : 0.0;
  }
}

// X = R^T for the upper triangle R of F's leading cols x cols block: the L of
// an LQ factorization computed as the QR of the transpose (Alg. 7).
__global__ void r_transposed_kernel(const double* __restrict__ F, int64_t ldf, int64_t cols,
                                    double* __restrict__ X, int64_t ldx) {
  const int64_t total = cols * cols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e % cols, c = e / cols;
    X[c + r * ldx] = (r <= c) ? F[r + c * ldf] : 0.0;
  }
}

// dst(r, c) = src(r, c) for a rows x cols block where one side is page-locked
// host memory mapped into the device address space: the SMs move the data
// over the host link with 16-byte accesses when both sides allow them.
__global__ void copy_mapped_kernel(const double* __restrict__ src, int64_t lds,
                                   double* __restrict__ dst, int64_t ldd, int64_t rows,
                                   int64_t cols, int vec) {
  for (int64_t c = blockIdx.y; c < cols; c += gridDim.y) {
    const double* s = src + c * lds;
    double* d = dst + c * ldd;
    if (vec) {
      const int64_t r2 = rows / 2;
      const double2* s2 = reinterpret_cast<const double2*>(s);
      double2* d2 = reinterpret_cast<double2*>(d);
      for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < r2;
           i += (int64_t)gridDim.x * blockDim.x)
        d2[i] = s2[i];
      if ((rows & 1) && blockIdx.x == 0 && threadIdx.x == 0) d[rows - 1] = s[rows - 1];
    } else {
      for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < rows;
           i += (int64_t)gridDim.x * blockDim.x)
        d[i] = s[i];
    }
  }
}

unsigned grid2(int64_t work) {
  int64_t b = (work + 255) / 256;
  if (b < 1) b = 1;
  if (b > 152 * 16) b = 152 * 16;
  return (unsigned)b;
}

}  // namespace

cudaError_t launch_gather_cols(const double* src, int64_t lds, int64_t r0, int64_t rows,
                               const int64_t* idx, int64_t ncols, double* dst, int64_t ldd,
                               cudaStream_t st) {
  if (rows <= 0 || ncols <= 0) return cudaSuccess;
  gather_cols_kernel<<<grid2(rows * ncols), 256, 0, st>>>(src, lds, r0, rows, idx, ncols, dst, ldd);
  return cudaGetLastError();
}

cudaError_t launch_scatter_transpose(const double* src, int64_t lds, int64_t rows,
                                     const int64_t* idx, int64_t ncols, double* dst, int64_t ldd,
                                     cudaStream_t st) {
  if (rows <= 0 || ncols <= 0) return cudaSuccess;
  scatter_transpose_kernel<<<grid2(rows * ncols), 256, 0, st>>>(src, lds, rows, idx, ncols, dst,
                                                                 ldd);
  return cudaGetLastError();
}

cudaError_t launch_split_qr(const double* F, int64_t ldf, int64_t rows, int64_t cols, int64_t yrow0,
                            double* Y, int64_t ldy, double* Rout, int64_t ldr, cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  split_qr_kernel<<<grid2(rows * cols), 256, 0, st>>>(F, ldf, rows, cols, yrow0, Y, ldy, Rout, ldr);
  return cudaGetLastError();
}

cudaError_t launch_copy_mapped(const double* src, int64_t lds, double* dst, int64_t ldd,
                               int64_t rows, int64_t cols, cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  const bool vec = ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15) == 0 &&
                   (lds % 2) == 0 && (ldd % 2) == 0;
  const int64_t per_col = (rows + 2 * 256 - 1) / (2 * 256);   // blocks covering a column once
  dim3 grid((unsigned)std::min<int64_t>(std::max<int64_t>(per_col / 4, 1), 64),
            (unsigned)std::min<int64_t>(cols, 65535));
  copy_mapped_kernel<<<grid, 256, 0, st>>>(src, lds, dst, ldd, rows, cols, vec ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_r_transposed(const double* F, int64_t ldf, int64_t cols, double* X,
                                int64_t ldx, cudaStream_t st) {
  if (cols <= 0) return cudaSuccess;
  r_transposed_kernel<<<grid2(cols * cols), 256, 0, st>>>(F, ldf, cols, X, ldx);
  return cudaGetLastError();
}

}  // namespace rq

namespace rq {
namespace {
__global__ void eye_kernel(double* Q, int64_t rows, int64_t cols, int64_t ld) {
  const int64_t total = rows * cols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e % rows, c = e / rows;
    Q[r + c * ld] = (r == c) ? 1.0 : 0.0;
  }
}
}  // namespace

cudaError_t launch_eye(double* Q, int64_t rows, int64_t cols, int64_t ld, cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  int64_t b = (rows * cols + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  eye_kernel<<<(unsigned)b, 256, 0, st>>>(Q, rows, cols, ld);
  return cudaGetLastError();
}
}  // namespace rq

namespace rq {
namespace {
template <typename TI, typename TO>
__global__ void convert_kernel(const TI* __restrict__ src, int64_t lds, TO* __restrict__ dst,
                               int64_t ldd, int64_t rows, int64_t cols) {
  const int64_t total = rows * cols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e % rows, c = e / rows;
    dst[r + c * ldd] = (TO)src[r + c * lds];
  }
}

// Mixed-precision panel write-back: P64 (rows x cols, ld ldp) holds the FP64
// factored panel; its R part and reflectors go to the FP32 array (ld lda),
// the explicit unit-lower reflector block to Y32 (ld ldy) and R's diagonal
// to rdiag in FP64.
__global__ void panel_writeback_kernel(const double* __restrict__ P, int64_t ldp, int64_t rows,
                                       int64_t cols, float* __restrict__ A, int64_t lda,
                                       float* __restrict__ Y, int64_t ldy, double* __restrict__ rdiag) {
  const int64_t total = rows * cols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e % rows, c = e / rows;
    const double v = P[r + c * ldp];
    A[r + c * lda] = (float)v;
    Y[r + c * ldy] = (r > c) ? (float)v : (r == c ? 1.0f : 0.0f);
    if (r == c) rdiag[c] = v;
  }
}
__global__ void gather_cols_f32_kernel(const float* __restrict__ src, int64_t lds, int64_t r0,
                                       int64_t rows, const int64_t* __restrict__ idx, int64_t ncols,
                                       float* __restrict__ dst, int64_t ldd) {
  const int64_t total = rows * ncols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e % rows, t = e / rows;
    dst[r + t * ldd] = src[(r0 + r) + idx[t] * lds];
  }
}

__global__ void copy_upper_f32_kernel(const float* __restrict__ src, int64_t lds, int64_t cols,
                                      float* __restrict__ dst, int64_t ldd) {
  const int64_t total = cols * cols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e % cols, c = e / cols;
    dst[r + c * ldd] = (r <= c) ? src[r + c * lds] : 0.0f;
  }
}
}  // namespace

cudaError_t launch_gather_cols_f32(const float* src, int64_t lds, int64_t r0, int64_t rows,
                                   const int64_t* idx, int64_t ncols, float* dst, int64_t ldd,
                                   cudaStream_t st) {
  if (rows <= 0 || ncols <= 0) return cudaSuccess;
  gather_cols_f32_kernel<<<grid2(rows * ncols), 256, 0, st>>>(src, lds, r0, rows, idx, ncols, dst,
                                                               ldd);
  return cudaGetLastError();
}

cudaError_t launch_copy_upper_f32(const float* src, int64_t lds, int64_t cols, float* dst,
                                  int64_t ldd, cudaStream_t st) {
  if (cols <= 0) return cudaSuccess;
  copy_upper_f32_kernel<<<grid2(cols * cols), 256, 0, st>>>(src, lds, cols, dst, ldd);
  return cudaGetLastError();
}

cudaError_t launch_convert_f32_f64(const float* src, int64_t lds, double* dst, int64_t ldd,
                                   int64_t rows, int64_t cols, cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  convert_kernel<float, double><<<grid2(rows * cols), 256, 0, st>>>(src, lds, dst, ldd, rows, cols);
  return cudaGetLastError();
}

cudaError_t launch_convert_f64_f32(const double* src, int64_t lds, float* dst, int64_t ldd,
                                   int64_t rows, int64_t cols, cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  convert_kernel<double, float><<<grid2(rows * cols), 256, 0, st>>>(src, lds, dst, ldd, rows, cols);
  return cudaGetLastError();
}

cudaError_t launch_panel_writeback(const double* P, int64_t ldp, int64_t rows, int64_t cols,
                                   float* A, int64_t lda, float* Y, int64_t ldy, double* rdiag,
                                   cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  panel_writeback_kernel<<<grid2(rows * cols), 256, 0, st>>>(P, ldp, rows, cols, A, lda, Y, ldy,
                                                              rdiag);
  return cudaGetLastError();
}
}  // namespace rq
