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
// is BF16 or FP32).  The reflectors are generated in FP64 and the squared
// norms are kept and downdated in FP64 either way.
template <typename T>
__device__ __forceinline__ void sample_qrcp_body(const SampleQrcpArgs& a, int g, int G,
                                                 unsigned char* smem_raw) {
  // lanes per column in the reflector apply: FP64 is issue-bound, so fewer
  // lanes (fewer shuffle-add levels per column); FP32 is latency-bound
  constexpr int LPA = sizeof(T) == 4 ? 8 : 4;
  constexpr int GRA = NT / LPA;
  const int ell = a.ell;
  const int64_t chunk = (a.nc + G - 1) / G;
  const int64_t c_lo = (int64_t)g * chunk;
  const int ncol = (int)imax64(0, imin64(a.nc, c_lo + chunk) - c_lo);

  // vn: squared trailing norms (downdated); thr: tol3z x the squared norm at
  // its last exact computation (the recompute threshold)
  double* vn = reinterpret_cast<double*>(smem_raw);             // chunk
  double* thr = vn + chunk;                                     // chunk
  long long* lpos = reinterpret_cast<long long*>(thr + chunk);  // chunk
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
  // exact initial squared norms (rounds of GROUPS columns keep the shuffles
  // warp-uniform)
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
      if (!isfinite(s)) atomicOr(a.status, RQRCP_INFO_NONFINITE);
      vn[c] = s;
      thr[c] = tol3z * s;
    }
  }
  __syncthreads();

  for (int i = 0; i < a.steps; ++i) {
    // ---- local candidate: warp 0 scans the owned columns and publishes the
    // best one's record (key, logical position, alpha = its row i, sigma2 =
    // the sum of squares of its rows i+1..) and its rows i+1..
    double* cand = a.cand + (size_t)(i & 1) * G * 4;
    double* ccol = a.candcol + (size_t)(i & 1) * G * ell;
    if (tid < 32) {
      Cand mine{sort_key(-2.0), LLONG_MAX, -1};
      for (int c = tid; c < ncol; c += 32) {
        if (done[c]) continue;
        Cand t{sort_key(isnan(vn[c]) ? -1.0 : vn[c]), lpos[c], c};
        if (better(t, mine)) mine = t;
      }
      mine = warp_argmax(mine);
      double alpha = 0.0, s = 0.0;
      if (mine.who >= 0) {
        const T* pc = col + (size_t)mine.who * ell;
        for (int r = i + 1 + tid; r < ell; r += 32) {
          const double x = pc[r];
          s = fma(x, x, s);
        }
        s = warp_sum(s);
        alpha = pc[i];
      }
      if (tid == 0) {
        red[0] = mine;
        cand[4 * g] = __longlong_as_double(mine.key);  // bit pattern
        cand[4 * g + 1] = __longlong_as_double(mine.pos);
        cand[4 * g + 2] = alpha;
        cand[4 * g + 3] = s;
      }
    }
    __syncthreads();
    const int my_pivot = red[0].who;  // local column index of this CTA's candidate
    if (my_pivot >= 0)
      for (int r = i + 1 + tid; r < ell; r += NT) ccol[(size_t)g * ell + r] = col[r + my_pivot * ell];
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
    // records, starts loading the winner's rows i+1.. and forms the reflector
    // scalars from the winner's alpha and sigma2 while those loads are in flight
    if (tid < 32) {
      Cand w{sort_key(-3.0), LLONG_MAX, -1};
      double wa = 0.0, ws = 0.0;
      for (int q = tid; q < G; q += 32) {
        const double2 kp = __ldcg(reinterpret_cast<const double2*>(cand + 4 * q));
        const double2 as = __ldcg(reinterpret_cast<const double2*>(cand + 4 * q + 2));
        const Cand t{__double_as_longlong(kp.x), __double_as_longlong(kp.y), q};
        if (better(t, w)) {
          w = t;
          wa = as.x;
          ws = as.y;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        Cand d;
        d.key = __shfl_xor_sync(0xffffffffu, w.key, o);
        d.pos = __shfl_xor_sync(0xffffffffu, w.pos, o);
        d.who = __shfl_xor_sync(0xffffffffu, w.who, o);
        const double da = __shfl_xor_sync(0xffffffffu, wa, o);
        const double ds = __shfl_xor_sync(0xffffffffu, ws, o);
        if (better(d, w)) {
          w = d;
          wa = da;
          ws = ds;
        }
      }
      const double* wc = ccol + (size_t)w.who * ell;
      constexpr int RPL = MAX_ELL / 32;
      double xr[RPL];
#pragma unroll
      for (int q = 0; q < RPL; ++q) {
        const int r = i + 1 + tid + 32 * q;
        xr[q] = r < ell ? __ldcg(wc + r) : 0.0;
      }
      double beta, tau, scale;
      house_scalars_sq(wa, ws, &beta, &tau, &scale);
#pragma unroll
      for (int q = 0; q < RPL; ++q) {
        const int r = i + 1 + tid + 32 * q;
        if (r < ell) {
          const double v = xr[q] * scale;
          xv[r] = v;
          xt[r] = (T)v;
        }
      }
      if (tid == 0) {
        xv[i] = 1.0;
        xt[i] = (T)1;
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
    // ---- apply H = I - tau v v^T to the trailing columns (LPA lanes per
    // column, rounds of GRA columns keep the shuffles warp-uniform)
    if (tau != 0.0) {
      const T taut = (T)tau;
      const int ga = tid / LPA, la = tid % LPA;
      for (int base = 0; base < ncol; base += GRA) {
        const int c = base + ga;
        const bool act = c < ncol && !done[c];
        if (__any_sync(0xffffffffu, act)) {
          T* cc = col + (size_t)(act ? c : 0) * ell;
          T s = (T)0;
          if (act)
            for (int r = i + la; r < ell; r += LPA) s = fma(xt[r], cc[r], s);
          s = lane_group_sum<LPA>(s) * taut;
          if (act)
            for (int r = i + la; r < ell; r += LPA) cc[r] = fma(-s, xt[r], cc[r]);
        }
      }
      __syncthreads();
    }
    // ---- downdate the squared norms, one thread per column: sigma2 -= x_i^2
    // (the same test as nrm^2 (1 - (x_i/nrm)^2) / nrm_ref^2 <= tol3z, with no
    // division or square root); a column that lost too many digits is
    // recomputed exactly from rows i+1.. (rare: a second pass only when some
    // column needs it)
    int need_any = 0;
    for (int c = tid; c < ncol; c += NT) {
      if (done[c] || vn[c] == 0.0) continue;
      const double x = col[i + (size_t)c * ell];
      const double v2 = fma(-x, x, vn[c]);
      if (v2 <= thr[c]) {
        vn[c] = -1.0;  // recompute below
        need_any = 1;
      } else {
        vn[c] = v2;
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
          vn[c] = t;
          thr[c] = tol3z * t;
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
