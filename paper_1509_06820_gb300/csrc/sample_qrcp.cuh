// Partial QRCP on the sample matrix (Alg. 1 halted after b pivots) as a
// device function over a group of co-resident CTAs: the body of the
// cooperative sample-QRCP kernel, shared with the persistent batched kernel.
// The algorithm and its data layout are described in sample_qrcp.cu.
#pragma once

#include <climits>

#include "kernels.cuh"

namespace rq {
namespace sq {


constexpr int NT = 256;
constexpr int LPC = 8;                 // lanes per column
constexpr int GROUPS = NT / LPC;       // columns processed concurrently
constexpr int MAX_ELL = 192;
constexpr double TOL3Z = 1.4901161193847656e-08;  // sqrt(2^-52)
// the same safeguard for a sample held in single precision: sqrt(2^-23)
constexpr double TOL3Z_F32 = 3.4526698300124393e-04;

// Sum over groups of W lanes of a warp, in the type of the sample.
template <int W, typename T>
__device__ __forceinline__ T lane_group_sum(T v) {
#pragma unroll
  for (int o = W / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

struct Cand {
  long long key; // order-preserving integer image of the norm (see sort_key);
                 // the norm -1 for NaN, -2 when the CTA has no trailing column
  long long pos; // logical position
  int who;       // CTA index or local column index
};

// Integer with the same order as the double d (also for negative d): the
// comparisons of the argmax then run on the integer pipe instead of FP64.
__device__ __forceinline__ long long sort_key(double d) {
  const long long b = __double_as_longlong(d);
  return b >= 0 ? b : (b ^ 0x7FFFFFFFFFFFFFFFLL);
}

__device__ __forceinline__ bool better(const Cand& a, const Cand& b) {
  return a.key > b.key || (a.key == b.key && a.pos < b.pos);
}

// Best candidate over the 32 lanes of a warp (all lanes get it).
__device__ __forceinline__ Cand warp_argmax(Cand c) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    Cand d;
    d.key = __shfl_xor_sync(0xffffffffu, c.key, o);
    d.pos = __shfl_xor_sync(0xffffffffu, c.pos, o);
    d.who = __shfl_xor_sync(0xffffffffu, c.who, o);
    if (better(d, c)) c = d;
  }
  return c;
}

// The sample QRCP on CTA g of a group of G co-resident CTAs (the whole grid
// of the standalone kernel, or one team of the persistent batched kernel);
// smem_raw: sample_qrcp_smem_bytes(ell, chunk, sizeof(T)) bytes of dynamic
// shared memory.  T is the type the sample is held and the reflectors are
// applied in: double, or float for a sample that is only single-precision
// accurate to begin with (the mixed-precision and served paths, whose sketch
// is BF16 or FP32).  The reflectors are generated in FP64 and the norms are
// kept and downdated in FP64 either way.
template <typename T>
__device__ __forceinline__ void sample_qrcp_body(const SampleQrcpArgs& a, int g, int G,
                                                 unsigned char* smem_raw) {
  const int ell = a.ell;
  const int64_t chunk = (a.nc + G - 1) / G;
  const int64_t c_lo = (int64_t)g * chunk;
  const int ncol = (int)imax64(0, imin64(a.nc, c_lo + chunk) - c_lo);

  double* vn = reinterpret_cast<double*>(smem_raw);             // chunk
  double* vn0 = vn + chunk;                                     // chunk
  long long* lpos = reinterpret_cast<long long*>(vn0 + chunk);  // chunk
  double* xv = reinterpret_cast<double*>(lpos + chunk);         // MAX_ELL (reflector v)
  T* xt = reinterpret_cast<T*>(xv + MAX_ELL);                   // MAX_ELL (v in type T)
  T* col = xt + MAX_ELL;                                        // ell x chunk
  int* done = reinterpret_cast<int*>(col + (size_t)ell * chunk);  // chunk
  constexpr double tol3z = sizeof(T) == 4 ? TOL3Z_F32 : TOL3Z;
  __shared__ Cand red[2];
  __shared__ double s_scal[4];

  const int tid = threadIdx.x;
  const int grp = tid / LPC, lig = tid % LPC;

  // load the owned columns, logical position = index
  for (int64_t e = tid; e < (int64_t)ncol * ell; e += NT) {
    const int64_t c = e / ell, r = e % ell;
    col[e] = (T)__ldcg(a.B + (c_lo + c) * a.ldb + r);
  }
  for (int c = tid; c < ncol; c += NT) {
    lpos[c] = c_lo + c;
    done[c] = 0;
  }
  __syncthreads();
  // exact initial norms (rounds of GROUPS columns keep the shuffles warp-uniform)
  for (int base = 0; base < ncol; base += GROUPS) {
    const int c = base + grp;
    const bool act = c < ncol;
    double s = 0.0;
    if (act)
      for (int r = lig; r < ell; r += LPC) {
        const double x = col[r + c * ell];
        s = fma(x, x, s);
      }
    s = group_sum<LPC>(s);
    if (act && lig == 0) {
      double nv = sqrt(s);
      if (!isfinite(nv)) atomicOr(a.status, RQRCP_INFO_NONFINITE);
      vn[c] = nv;
      vn0[c] = nv;
    }
  }
  __syncthreads();

  for (int i = 0; i < a.steps; ++i) {
    // ---- local candidate: warp 0 scans the owned columns
    double* cand = a.cand + (size_t)(i & 1) * G * 2;
    double* ccol = a.candcol + (size_t)(i & 1) * G * ell;
    if (tid < 32) {
      Cand mine{sort_key(-2.0), LLONG_MAX, -1};
      for (int c = tid; c < ncol; c += 32) {
        if (done[c]) continue;
        Cand t{sort_key(isnan(vn[c]) ? -1.0 : vn[c]), lpos[c], c};
        if (better(t, mine)) mine = t;
      }
      mine = warp_argmax(mine);
      if (tid == 0) {
        red[0] = mine;
        cand[2 * g] = __longlong_as_double(mine.key);       // bit pattern
        cand[2 * g + 1] = __longlong_as_double(mine.pos);
      }
    }
    __syncthreads();
    const int my_pivot = red[0].who;  // local column index of this CTA's candidate
    if (my_pivot >= 0)
      for (int r = tid; r < ell; r += NT) ccol[(size_t)g * ell + r] = col[r + my_pivot * ell];
    if (!grid_barrier(a.bar, G + a.phantom, a.status,
                      a.phantom ? kBarrierTestPolls : kBarrierMaxPolls)) {
      // the wait ran out (RQRCP_INFO_TIMEOUT is set): leave valid swap
      // partners (no exchange) for the steps not taken, so that whatever
      // consumes the list stays within its columns
      if (g == 0)
        for (int t = i + tid; t < a.steps; t += NT) a.swaps[t] = t;
      return;
    }

    // ---- global winner (identical in every CTA): warp 0 scans the G
    // candidates, then builds the reflector from the winner's rows i..ell-1
    if (tid < 32) {
      Cand w{sort_key(-3.0), LLONG_MAX, -1};
      for (int q = tid; q < G; q += 32) {
        Cand t{__double_as_longlong(__ldcg(cand + 2 * q)),
               __double_as_longlong(__ldcg(cand + 2 * q + 1)), q};
        if (better(t, w)) w = t;
      }
      w = warp_argmax(w);
      // the winner's rows i..ell-1; each lane rescales the rows it loaded
      const double* wc = ccol + (size_t)w.who * ell;
      double s = 0.0;
      for (int r = i + tid; r < ell; r += 32) {
        const double x = __ldcg(wc + r);
        xv[r] = x;
        if (r > i) s = fma(x, x, s);
      }
      s = warp_sum(s);
      __syncwarp();
      const double alpha = xv[i];
      __syncwarp();  // every lane has read alpha before lane 0 overwrites it
      double beta, tau, scale;
      house_scalars_sq(alpha, s, &beta, &tau, &scale);
      for (int r = i + tid; r < ell; r += 32) {
        const double v = (r == i) ? 1.0 : xv[r] * scale;
        xv[r] = v;
        xt[r] = (T)v;
      }
      if (tid == 0) {
        s_scal[0] = beta;
        s_scal[1] = tau;
        red[1] = w;
      }
    }
    __syncthreads();
    const Cand w = red[1];
    const long long Lstar = w.pos;
    const double beta = s_scal[0], tau = s_scal[1];
    if (g == 0 && tid == 0) a.swaps[i] = Lstar;
    // the trailing column at logical position i moves to Lstar (the pivot
    // itself sits at Lstar != i, so it is not matched here)
    if (Lstar != i) {
      for (int c = tid; c < ncol; c += NT)
        if (!done[c] && lpos[c] == i) lpos[c] = Lstar;
    }
    __syncthreads();
    if (g == w.who && my_pivot >= 0) {
      // finish the pivot column: S(i, i) = beta, zeros below, position i
      for (int r = i + 1 + tid; r < ell; r += NT) col[r + my_pivot * ell] = (T)0;
      if (tid == 0) {
        col[i + my_pivot * ell] = (T)beta;
        done[my_pivot] = 1;
        lpos[my_pivot] = i;
      }
    }
    __syncthreads();
    // ---- apply H = I - tau v v^T to the trailing columns (LPC lanes per
    // column, rounds of GROUPS columns keep the shuffles warp-uniform)
    if (tau != 0.0) {
      const T taut = (T)tau;
      for (int base = 0; base < ncol; base += GROUPS) {
        const int c = base + grp;
        const bool act = c < ncol && !done[c];
        if (__any_sync(0xffffffffu, act)) {
          T* cc = col + (size_t)(act ? c : 0) * ell;
          T s = (T)0;
          if (act)
            for (int r = i + lig; r < ell; r += LPC) s = fma(xt[r], cc[r], s);
          s = lane_group_sum<LPC>(s) * taut;
          if (act)
            for (int r = i + lig; r < ell; r += LPC) cc[r] = fma(-s, xt[r], cc[r]);
        }
      }
      __syncthreads();
    }
    // ---- downdate the norms, one thread per column; a column whose
    // downdated norm lost too many digits is recomputed exactly from rows
    // i+1.. (rare: a second pass only when some column needs it)
    int need_any = 0;
    for (int c = tid; c < ncol; c += NT) {
      if (done[c] || vn[c] == 0.0) continue;
      const double rr = fabs((double)col[i + (size_t)c * ell]) / vn[c];
      const double f = fmax(0.0, (1.0 - rr) * (1.0 + rr));
      const double q = vn[c] / vn0[c];
      if (f * q * q <= tol3z) {
        vn[c] = -1.0;  // recompute below
        need_any = 1;
      } else {
        vn[c] *= sqrt(f);
      }
    }
    if (__syncthreads_or(need_any)) {
      for (int base = 0; base < ncol; base += GROUPS) {
        const int c = base + grp;
        const bool act = c < ncol && !done[c] && vn[c] < 0.0;
        double t = 0.0;
        if (act) {
          const T* cc = col + (size_t)c * ell;
          for (int r = i + 1 + lig; r < ell; r += LPC) {
            const double x = cc[r];
            t = fma(x, x, t);
          }
        }
        t = group_sum<LPC>(t);
        if (act && lig == 0) {
          vn[c] = sqrt(t);
          vn0[c] = vn[c];
        }
      }
      __syncthreads();
    }
  }

  // every CTA finished loading before the first barrier: write S back in the
  // permuted (logical) order
  for (int c = 0; c < ncol; ++c) {
    const long long L = lpos[c];
    for (int r = tid; r < ell; r += NT) a.B[L * a.ldb + r] = (double)col[r + (size_t)c * ell];
  }
}

// dynamic shared memory of sample_qrcp_body<T> (tsize = sizeof(T))
__host__ __device__ inline size_t sample_qrcp_smem_bytes(int ell, int64_t chunk,
                                                        size_t tsize = 8) {
  return (size_t)chunk * ((size_t)ell * tsize + 8 + 8 + 8 + 4) + MAX_ELL * (8 + tsize) + 16;
}

}  // namespace sq
}  // namespace rq
