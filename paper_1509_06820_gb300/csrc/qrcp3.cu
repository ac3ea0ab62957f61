// Deterministic QR with column pivoting with level-3 BLAS reflection blocking
// (the Quintana-Orti scheme the paper describes as Alg. qrcp3 in Sec. 2): the
// comparison method whose per-column pass over the whole trailing matrix the
// randomized sample avoids.
//
// One cooperative kernel runs the column loop of one block (up to bJ pivots):
//   B  pivot = argmax of the trailing norms (ties: lowest position); swap it
//      into column j; bring the new column up to date with the block's
//      reflectors, a_j -= Y W(p, :)^T (rows j..m-1); partial sums of squares.
//   C  reflector y_j, tau_j from the updated column; stage y_j in shared memory;
//      y_j^T A for every other column of the block and of the trailing matrix
//      (the level-2 pass: it reads the whole trailing matrix), split into row
//      chunks when there are fewer columns than warps.
//   D  adjusted inner products w_j(c) = tau_j (y_j^T a_c - (y_j^T Y) W(c, :)^T),
//      the row update A(j, c) -= Y(j, :) W(c, :)^T, the norm downdate and the
//      next argmax candidates.
// with one grid barrier after each phase.  A downdated norm that lost too many
// digits (the LAPACK xLAQPS criterion) flags its column and ends the block
// after the current column; the next block's kernel recomputes the flagged
// norms exactly from the updated trailing matrix, so the pivots follow the
// unblocked algorithm (Alg. 1 with exact recomputation).  Between blocks the
// host applies A22 -= Y W^T with the FP64 GEMM.
//
// Data written by other CTAs during the launch is read with L1-bypassing
// loads.  All sums run in a fixed order: the result is reproducible.
#include <climits>

#include "kernels.cuh"

namespace rq {
namespace {

constexpr int Q3NT = 512;
constexpr int Q3W = Q3NT / 32;
constexpr double Q3TOL3Z = 1.4901161193847656e-08;  // sqrt(2^-52)

__device__ __forceinline__ double q3_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ long long q3_key(double d) {
  if (isnan(d)) d = -1.0;
  const long long b = __double_as_longlong(d);
  return b >= 0 ? b : (b ^ 0x7FFFFFFFFFFFFFFFLL);
}

__device__ __forceinline__ void q3_better(long long& k, long long& p, long long k2, long long p2) {
  if (k2 > k || (k2 == k && p2 < p)) {
    k = k2;
    p = p2;
  }
}

__device__ __forceinline__ void q3_warp_best(long long& k, long long& p) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long k2 = __shfl_xor_sync(0xffffffffu, k, o);
    const long long p2 = __shfl_xor_sync(0xffffffffu, p, o);
    q3_better(k, p, k2, p2);
  }
}

// Contiguous share of CTA g among G of the columns [lo, n).
__device__ __forceinline__ void q3_slice(int64_t lo, int64_t n, int g, int G, int64_t* c0,
                                         int64_t* c1) {
  const int64_t len = n - lo;
  const int64_t per = len > 0 ? (len + G - 1) / G : 0;
  int64_t a = lo + (int64_t)g * per;
  if (a > n) a = n;
  int64_t b = a + per;
  if (b > n) b = n;
  *c0 = a;
  *c1 = b;
}

// Block-wide argmax of vn1 over [c0, c1); thread 0 writes the candidate.
__device__ void q3_cta_argmax(const Qrcp3Args& a, int64_t c0, int64_t c1, long long* s_k,
                              long long* s_p) {
  long long k = q3_key(-2.0), p = LLONG_MAX;
  for (int64_t c = c0 + threadIdx.x; c < c1; c += Q3NT) q3_better(k, p, q3_key(__ldcg(a.vn1 + c)), c);
  q3_warp_best(k, p);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    s_k[warp] = k;
    s_p[warp] = p;
  }
  __syncthreads();
  if (warp == 0) {
    k = lane < Q3W ? s_k[lane] : q3_key(-2.0);
    p = lane < Q3W ? s_p[lane] : LLONG_MAX;
    q3_warp_best(k, p);
    if (lane == 0) {
      a.cand[2 * blockIdx.x] = k;
      a.cand[2 * blockIdx.x + 1] = p;
    }
  }
}

__global__ void __launch_bounds__(Q3NT, 1) qrcp3_block_kernel(Qrcp3Args a) {
  extern __shared__ double s_y[];  // staged reflector rows j..j+cap-1
  __shared__ double s_wp[kQrcp3MaxB], s_aux[kQrcp3MaxB], s_yrow[kQrcp3MaxB];
  __shared__ double s_red[Q3W];
  __shared__ long long s_k[Q3W], s_p[Q3W];
  __shared__ long long s_piv;

  const int G = gridDim.x, g = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t m = a.m, n = a.n, i0 = a.i0, lda = a.lda;
  double* A = a.A;
  const int64_t rstride = (int64_t)G * Q3NT;
  const int64_t gthread = (int64_t)g * Q3NT + tid;
  const int total_warps = G * Q3W;
  const int gwarp = g * Q3W + warp;

  // ---- set-up: exact norms of flagged columns (rows i0..m-1), candidates
  {
    int64_t c0, c1;
    q3_slice(i0, n, g, G, &c0, &c1);
    for (int64_t c = c0 + warp; c < c1; c += Q3W) {
      if (__ldcg(a.redo + c) == 0) continue;
      const double* col = A + c * lda;
      double s = 0.0;
      for (int64_t r = i0 + lane; r < m; r += 32) {
        const double v = __ldcg(col + r);
        s = fma(v, v, s);
      }
      s = q3_warp_sum(s);
      if (lane == 0) {
        const double nr = sqrt(s);
        a.vn1[c] = nr;
        a.vn2[c] = nr;
        a.redo[c] = 0;
      }
    }
    __syncthreads();
    q3_cta_argmax(a, c0, c1, s_k, s_p);
  }
  if (!grid_barrier(a.bar, G, a.status)) return;

  int nb = 0;
  for (int jj = 0; jj < a.bJ; ++jj) {
    const int64_t j = i0 + jj;
    // ---- B: pivot, swap, column update, partial norm
    if (warp == 0) {
      long long k = q3_key(-3.0), p = LLONG_MAX;
      for (int q = lane; q < G; q += 32) q3_better(k, p, __ldcg(a.cand + 2 * q), __ldcg(a.cand + 2 * q + 1));
      q3_warp_best(k, p);
      if (lane == 0) s_piv = p;
    }
    __syncthreads();
    const int64_t p = s_piv;
    if (tid < jj) s_wp[tid] = __ldcg(a.W + p + (int64_t)tid * n);
    __syncthreads();
    double ss = 0.0;
    for (int64_t r = gthread; r < m; r += rstride) {
      const double aj = __ldcg(A + r + j * lda);
      double v = __ldcg(A + r + p * lda);
      if (r >= j) {
        for (int t = 0; t < jj; ++t) v = fma(-__ldcg(A + r + (i0 + t) * lda), s_wp[t], v);
        a.ys[r] = v;
        if (r > j) ss = fma(v, v, ss);
      }
      if (p != j) A[r + p * lda] = aj;
      A[r + j * lda] = v;
    }
    ss = q3_warp_sum(ss);
    if (lane == 0) s_red[warp] = ss;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < Q3W; ++w) t += s_red[w];
      a.npart[g] = t;
    }
    if (!grid_barrier(a.bar, G, a.status)) return;

    // ---- C: reflector, deferred swaps, staged y, level-2 pass
    double beta, tau, scale;
    {
      double sigma2 = 0.0;
      for (int q = 0; q < G; ++q) sigma2 += __ldcg(a.npart + q);
      house_scalars_sq(__ldcg(a.ys + j), sigma2, &beta, &tau, &scale);
    }
    if (g == 0) {
      if (tid == 0) {
        a.tau[j] = tau;
        A[j + j * lda] = beta;
        if (p != j) {
          const double v1j = __ldcg(a.vn1 + j), v1p = __ldcg(a.vn1 + p);
          const double v2j = __ldcg(a.vn2 + j), v2p = __ldcg(a.vn2 + p);
          a.vn1[j] = v1p;
          a.vn1[p] = v1j;
          a.vn2[j] = v2p;
          a.vn2[p] = v2j;
          const int64_t q = a.jpvt[j];
          a.jpvt[j] = a.jpvt[p];
          a.jpvt[p] = q;
        }
      }
      if (p != j && tid < jj) {
        const int64_t o = (int64_t)tid * n;
        const double wj = __ldcg(a.W + j + o), wp = __ldcg(a.W + p + o);
        a.W[j + o] = wp;
        a.W[p + o] = wj;
      }
    }
    const int64_t mj = m - j;
    const int64_t staged = mj < a.smem_rows ? mj : a.smem_rows;
    for (int64_t r = tid; r < staged; r += Q3NT)
      s_y[r] = (r == 0) ? 1.0 : __ldcg(a.ys + j + r) * scale;
    for (int64_t r = gthread; r < m; r += rstride)
      if (r > j) A[r + j * lda] = __ldcg(a.ys + r) * scale;
    __syncthreads();
    const int64_t ncol = n - i0 - 1;
    int nch = 1;
    if (ncol > 0 && ncol < total_warps) {
      nch = (int)((total_warps + ncol - 1) / ncol);
      const int64_t maxch = (mj + 511) / 512;
      if (nch > maxch) nch = (int)maxch;
      if (nch > kQrcp3Chunks) nch = kQrcp3Chunks;
      if (nch < 1) nch = 1;
    }
    const int64_t clen = (((mj + nch - 1) / nch) + 31) / 32 * 32;
    const int64_t items = ncol * nch;
    for (int64_t it = gwarp; it < items; it += total_warps) {
      const int64_t ci = it / nch;
      const int ch = (int)(it % nch);
      const int64_t c = i0 + ci + (ci >= jj ? 1 : 0);
      const int64_t q0 = (int64_t)ch * clen;   // offsets from row j
      int64_t q1 = q0 + clen;
      if (q1 > mj) q1 = mj;
      const double* col = A + j + c * lda;
      double acc[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) acc[u] = 0.0;
      int64_t q = q0 + lane;
      const int64_t qs = q1 < staged ? q1 : staged;
      if (q + 7 * 32 < qs) {
        // software-pipelined: the next 8 loads are in flight while the FP64
        // pipe works through the current 8 products
        double x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) x[u] = __ldcg(col + q + u * 32);
        while (true) {
          const int64_t qn = q + 8 * 32;
          const bool more = qn + 7 * 32 < qs;
          double xn[8];
          if (more) {
#pragma unroll
            for (int u = 0; u < 8; ++u) xn[u] = __ldcg(col + qn + u * 32);
          }
#pragma unroll
          for (int u = 0; u < 8; ++u) acc[u] = fma(s_y[q + u * 32], x[u], acc[u]);
          q = qn;
          if (!more) break;
#pragma unroll
          for (int u = 0; u < 8; ++u) x[u] = xn[u];
        }
      }
      for (; q < qs; q += 32) acc[0] = fma(s_y[q], __ldcg(col + q), acc[0]);
      // rows beyond the staged part: y from global memory
      for (; q < q1; q += 32) acc[1] = fma(__ldcg(a.ys + j + q) * scale, __ldcg(col + q), acc[1]);
      double d = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
      d = q3_warp_sum(d);
      if (lane == 0) a.dots[(int64_t)ch * n + c] = d;
    }
    if (!grid_barrier(a.bar, G, a.status)) return;

    // ---- D: inner products, row update, norm downdate, candidates
    if (tid < jj) {
      double s = 0.0;
      for (int ch = 0; ch < nch; ++ch) s += __ldcg(a.dots + (int64_t)ch * n + i0 + tid);
      s_aux[tid] = s;
      s_yrow[tid] = __ldcg(A + j + (i0 + tid) * lda);
    }
    __syncthreads();
    int64_t c0, c1;
    q3_slice(j + 1, n, g, G, &c0, &c1);
    int mark = 0;
    for (int64_t c = c0 + tid; c < c1; c += Q3NT) {
      double d = 0.0;
      for (int ch = 0; ch < nch; ++ch) d += __ldcg(a.dots + (int64_t)ch * n + c);
      double sa = 0.0, sr = 0.0;
      for (int t = 0; t < jj; ++t) {
        const double wt = __ldcg(a.W + c + (int64_t)t * n);
        sa = fma(s_aux[t], wt, sa);
        sr = fma(s_yrow[t], wt, sr);
      }
      const double w = tau * (d - sa);
      a.W[c + (int64_t)jj * n] = w;
      const double rowv = (__ldcg(A + j + c * lda) - sr) - w;
      A[j + c * lda] = rowv;
      const double v1 = __ldcg(a.vn1 + c);
      if (v1 != 0.0) {
        const double rr = fabs(rowv) / v1;
        const double f = fmax(0.0, (1.0 - rr) * (1.0 + rr));
        const double qn = v1 / __ldcg(a.vn2 + c);
        if (f * qn * qn <= Q3TOL3Z) {
          a.redo[c] = 1;
          mark = 1;
        } else {
          a.vn1[c] = v1 * sqrt(f);
        }
      }
    }
    if (__syncthreads_or(mark) && tid == 0) atomicOr(a.ctl, 1);
    q3_cta_argmax(a, c0, c1, s_k, s_p);
    if (!grid_barrier(a.bar, G, a.status)) return;
    nb = jj + 1;
    if (__ldcg(a.ctl) != 0) break;
  }
  if (g == 0 && tid == 0) a.ctl[1] = nb;
}

}  // namespace

size_t qrcp3_smem_bytes(int64_t m) {
  const int64_t rows = m < kQrcp3SmemRows ? m : kQrcp3SmemRows;
  return (size_t)(rows > 0 ? rows : 1) * sizeof(double);
}

cudaError_t launch_qrcp3_block(const Qrcp3Args& a, int num_sms, cudaStream_t st) {
  if (a.bJ < 1 || a.bJ > kQrcp3MaxB) return cudaErrorInvalidValue;
  static std::atomic<uint64_t> attr_done{0};
  cudaError_t e = ensure_smem_attr(qrcp3_block_kernel, (int)(kQrcp3SmemRows * sizeof(double)),
                                   attr_done);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(a.bar, 0, sizeof(GridBarrier), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.ctl, 0, 2 * sizeof(int), st);
  if (e != cudaSuccess) return e;
  Qrcp3Args args = a;
  args.smem_rows = a.m < kQrcp3SmemRows ? a.m : kQrcp3SmemRows;
  void* params[] = {&args};
  return cudaLaunchCooperativeKernel((const void*)qrcp3_block_kernel, dim3((unsigned)num_sms),
                                     dim3(Q3NT), params, qrcp3_smem_bytes(a.m), st);
}

}  // namespace rq
