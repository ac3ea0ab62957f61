// SVD of the k x k connection matrix X of Alg. 7 (TUXV): the paper notes that
// the diagonal of X already approximates the leading singular values and that
// an SVD of the small X gives better ones.  X = Ux diag(sigma) Vs^T by
// one-sided (Hestenes) Jacobi: column pairs (i, j) of a working copy G of X
// are rotated until every pair is orthogonal to working precision; the
// accumulated rotations form Vs, the column norms of G are sigma and the
// normalised columns of G are Ux.
//
// Parallel order: the k (rounded up to even) indices are paired by the circle
// method, k/2 disjoint pairs per round and every pair once in k - 1 rounds
// (one sweep).  One warp handles one pair; the rounds are separated by grid
// barriers (cooperative launch) or by __syncthreads for a one-CTA grid.  All
// sums are warp reductions in a fixed order, so results are reproducible.
//
// The working matrices live in global memory (L2-resident at these sizes) and
// are read with L1-bypassing loads because other CTAs update them between
// barriers.
#include "kernels.cuh"

namespace rq {
namespace {

constexpr int JNT = 256;                // threads per CTA (8 warps)
constexpr int JWARPS = JNT / 32;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Pair q of round r for kp (even) indices: index kp - 1 stays put, the others
// rotate around it.
__device__ __forceinline__ void round_pair(int r, int q, int kp, int* a, int* b) {
  if (q == 0) {
    *a = kp - 1;
    *b = r;
  } else {
    *a = (r + q) % (kp - 1);
    *b = (r - q + (kp - 1)) % (kp - 1);
  }
}

__device__ __forceinline__ bool sync_all(const JacobiArgs& a) {
  if (gridDim.x == 1) {
    __syncthreads();
    return true;
  }
  return grid_barrier(a.bar, gridDim.x, a.status);
}

__global__ void __launch_bounds__(JNT) jacobi_svd_kernel(JacobiArgs a) {
  const int k = a.k;
  const int64_t kk = (int64_t)k * k;
  const int lane = threadIdx.x & 31;
  const int gwarp = blockIdx.x * JWARPS + (threadIdx.x >> 5);
  const int nwarps = gridDim.x * JWARPS;
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t gthreads = (int64_t)gridDim.x * blockDim.x;
  double* G = a.G;
  double* V = a.Vx;

  for (int64_t e = gtid; e < kk; e += gthreads) {
    const int64_t r = e % k, c = e / k;
    G[e] = a.X[r + c * a.ldx];
    V[e] = (r == c) ? 1.0 : 0.0;
  }
  if (!sync_all(a)) return;

  const int kp = k + (k & 1);
  const double tol = sqrt((double)k) * 0x1p-53;
  int sweep = 0;
  for (; sweep < kJacobiMaxSweeps; ++sweep) {
    for (int r = 0; r < kp - 1; ++r) {
      for (int q = gwarp; q < kp / 2; q += nwarps) {
        int i, j;
        round_pair(r, q, kp, &i, &j);
        if (i >= k || j >= k) continue;
        if (i > j) {
          const int t = i;
          i = j;
          j = t;
        }
        double* gi = G + (int64_t)i * k;
        double* gj = G + (int64_t)j * k;
        double al = 0.0, be = 0.0, ga = 0.0;
        for (int t = lane; t < k; t += 32) {
          const double x = __ldcg(gi + t), y = __ldcg(gj + t);
          al = fma(x, x, al);
          be = fma(y, y, be);
          ga = fma(x, y, ga);
        }
        al = warp_sum(al);
        be = warp_sum(be);
        ga = warp_sum(ga);
        if (ga == 0.0 || !(fabs(ga) > tol * sqrt(al) * sqrt(be))) continue;
        // rotation that makes columns i and j orthogonal: the smaller root t
        // of t^2 + 2 zeta t - 1 = 0 with zeta = (beta - alpha) / (2 gamma)
        const double zeta = (be - al) / (2.0 * ga);
        const double az = fabs(zeta);
        const double t = (az > 1e150) ? 0.5 / zeta
                                       : copysign(1.0, zeta) / (az + sqrt(fma(zeta, zeta, 1.0)));
        const double c = 1.0 / sqrt(fma(t, t, 1.0));
        const double s = c * t;
        for (int u = lane; u < k; u += 32) {
          const double x = __ldcg(gi + u), y = __ldcg(gj + u);
          gi[u] = c * x - s * y;
          gj[u] = s * x + c * y;
        }
        double* vi = V + (int64_t)i * k;
        double* vj = V + (int64_t)j * k;
        for (int u = lane; u < k; u += 32) {
          const double x = __ldcg(vi + u), y = __ldcg(vj + u);
          vi[u] = c * x - s * y;
          vj[u] = s * x + c * y;
        }
        if (lane == 0) a.rotated[sweep] = 1;
      }
      if (!sync_all(a)) return;
    }
    if (__ldcg(a.rotated + sweep) == 0) break;
  }
  if (sweep == kJacobiMaxSweeps && gtid == 0) atomicOr(a.status, RQRCP_INFO_NOCONV);

  // column norms of G are the singular values (unsorted)
  for (int i = gwarp; i < k; i += nwarps) {
    const double* gi = G + (int64_t)i * k;
    double s2 = 0.0;
    for (int t = lane; t < k; t += 32) {
      const double x = __ldcg(gi + t);
      s2 = fma(x, x, s2);
    }
    s2 = warp_sum(s2);
    if (lane == 0) a.sraw[i] = sqrt(s2);
  }
  if (!sync_all(a)) return;

  // descending order (ties by index): column i goes to position rank(i)
  for (int i = gwarp; i < k; i += nwarps) {
    const double si = __ldcg(a.sraw + i);
    int cnt = 0;
    for (int j = lane; j < k; j += 32) {
      const double sj = __ldcg(a.sraw + j);
      cnt += (sj > si || (sj == si && j < i)) ? 1 : 0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    const int64_t rk = cnt;
    if (lane == 0) a.sigma[rk] = si;
    const double inv = (si > 0.0) ? 1.0 / si : 0.0;
    const double* gi = G + (int64_t)i * k;
    const double* vi = V + (int64_t)i * k;
    for (int t = lane; t < k; t += 32) {
      a.Ux[t + rk * k] = __ldcg(gi + t) * inv;
      a.Vs[t + rk * k] = __ldcg(vi + t);
    }
  }
}

}  // namespace

int jacobi_grid(int k, int num_sms) {
  const int kp = k + (k & 1);
  int g = (kp / 2 + JWARPS - 1) / JWARPS;
  if (g > num_sms) g = num_sms;
  return g < 1 ? 1 : g;
}

cudaError_t launch_jacobi_svd(const JacobiArgs& a, int num_sms, cudaStream_t st) {
  if (a.k < 1) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(a.rotated, 0, sizeof(int) * kJacobiMaxSweeps, st);
  if (e != cudaSuccess) return e;
  const int G = jacobi_grid(a.k, num_sms);
  if (G == 1) {
    jacobi_svd_kernel<<<1, JNT, 0, st>>>(a);
    return cudaGetLastError();
  }
  e = cudaMemsetAsync(a.bar, 0, sizeof(GridBarrier), st);
  if (e != cudaSuccess) return e;
  JacobiArgs args = a;
  void* params[] = {&args};
  return cudaLaunchCooperativeKernel((const void*)jacobi_svd_kernel, dim3((unsigned)G), dim3(JNT),
                                     params, 0, st);
}

}  // namespace rq
