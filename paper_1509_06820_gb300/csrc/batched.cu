// Persistent batched TRQRCP: many uneven mixed-precision truncated RQRCP
// problems (Alg. 6) in ONE cooperative launch.
//
// The grid is split into teams of G co-resident CTAs (one CTA per SM).  A
// team claims the next problem from a work source -- a descriptor table in
// device memory (sorted longest-first by the host), or a request ring in
// mapped host memory that the host keeps filling (the serving loop) -- and
// runs all of Alg. 6 on it, phase after phase, separated by a software
// barrier over the team's CTAs (bounded waits, RQRCP_INFO_TIMEOUT on
// expiry).  Per-problem state (the sample, the panel, W^T, T, Z) lives in the
// team's slice of the handle's scratch; nothing returns to the host between
// problems, so the launch can be captured in a CUDA graph, and a problem's
// result depends only on the problem and G (the same alone and in a batch).
//
// Arithmetic of one problem (FP32 storage, FP64 where the method's pivoting
// and reflectors need it):
//   Omega     Philox4x32-10 stream 1 (as everywhere in this library), the
//             Box-Muller transform in FP32 (it only steers pivots)
//   B = Omega A                         FP32 products, stored FP64
//   sample QRCP (Alg. 1 halted)        reflectors generated and norms
//                                       downdated in FP64, the sample held
//                                       and the reflectors applied in FP32
//                                       (the same device code as the
//                                       cooperative sample kernel)
//   A_hat = A(:, sel) - Y1 W1^T(:, sel) FP32 products, FP64 panel
//   panel QR + T (Sec. 2.2)             FP64, the same device code as the
//                                       cooperative panel kernel; reflectors
//                                       rounded to FP32 with tau = 2/v^T v
//   W2^T = T2^T (Y2^T A - (Y2^T Y1) W1^T), R rows   FP32 products
//   W11 = S11 R11^-1, B1 = S12 - W11 R12 (Eq. 3)    FP64
// The FP32 products run on the CUDA cores as a team-cooperative tiled GEMM
// (4 x 8 outputs per thread, 64 x 128 tiles, or 32 x 256 / 16 x 512 for
// products of few rows; split over K when there are fewer tiles than CTAs,
// partial sums added in a fixed order).
#include <algorithm>
#include <climits>

#include "kernels.cuh"
#include "panel.cuh"
#include "philox.cuh"
#include "sample_qrcp.cuh"

namespace rq {
namespace {

constexpr int NT = 256;
constexpr int MAXB = 128;
constexpr uint32_t kOmegaStreamId = 1;

// Loads of data that other CTAs of the launch wrote go through L2 (__ldcg):
// the L1 of an SM is not kept coherent with stores made on other SMs.
__device__ __forceinline__ int64_t ldg_i64(const int64_t* p) {
  return (int64_t)__ldcg(reinterpret_cast<const long long*>(p));
}

// ---------------------------------------------------------------- team GEMM
// C (M x N) = alpha op(A) op(B) + beta Cin, column-major.
//   op(A)(i, k) = at ? A[k + i lda] : A[i + k lda]
//   op(B)(k, j) = B[brow0 + k + col(j) ldb],  col(j) = bmap ? bmap[j] : j
//   Cin(i, j)   = Cin[crow0 + i + ccol(j) ldci], ccol(j) = cmap ? cmap[j] : j
// TC is the type of the products and sums.
template <typename TC, typename TA, typename TB, typename TI, typename TO>
struct TeamGemm {
  int64_t M, N, K;
  const TA* A;
  int64_t lda;
  int at;
  const TB* B;
  int64_t ldb;
  const int64_t* bmap;
  int64_t brow0;
  const TI* Cin;
  int64_t ldci;
  const int64_t* cmap;
  int64_t crow0;
  TO* C;
  int64_t ldc;
  TC alpha, beta;
};

template <typename TC, typename TA, typename TB, typename TI, typename TO>
__device__ __forceinline__ void tg_epilogue(const TeamGemm<TC, TA, TB, TI, TO>& op, int64_t i,
                                            int64_t j, TC acc) {
  TC v = op.alpha * acc;
  if (op.Cin != nullptr) {
    const int64_t cc = op.cmap ? ldg_i64(op.cmap + j) : j;
    v += op.beta * (TC)__ldcg(op.Cin + op.crow0 + i + cc * op.ldci);
  }
  op.C[i + j * op.ldc] = (TO)v;
}

// Four consecutive shared-memory values (16-byte aligned) in one or two
// vector loads.
__device__ __forceinline__ void ld4(const float* p, float (&v)[4]) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  v[0] = t.x;
  v[1] = t.y;
  v[2] = t.z;
  v[3] = t.w;
}
__device__ __forceinline__ void ld4(const double* p, double (&v)[4]) {
  const double2 t0 = *reinterpret_cast<const double2*>(p);
  const double2 t1 = *reinterpret_cast<const double2*>(p + 2);
  v[0] = t0.x;
  v[1] = t0.y;
  v[2] = t1.x;
  v[3] = t1.y;
}

// Output tile shapes of the team GEMM, chosen by the row count M: every
// thread computes 4 rows x 8 columns, 256 threads cover TM x TN =
// (TM / 4 row groups) x (TN / 8 column groups), and TK-deep slabs of both
// operands are staged in shared memory (rows padded by 4 to keep 16-byte
// alignment).  Short products (M = the block's b_J rows) get wide tiles, so
// that a partial last block does not pad its rows up to 64.
template <int TM_, int TN_, int TK_>
struct Tile {
  static constexpr int TM = TM_, TN = TN_, TK = TK_;
  static constexpr int RG = TM / 4, CG = TN / 8;     // row and column groups
  static constexpr int ACTIVE = RG * CG;             // threads that compute
  static constexpr int LDA = TM + 4, LDB = TN + 4;   // shared row lengths
  static constexpr int NLA = (TM * TK + NT - 1) / NT, NLB = (TN * TK + NT - 1) / NT;
  static_assert(ACTIVE <= NT && TM % 4 == 0 && TN % 8 == 0, "4 x 8 outputs per thread");
  static_assert(LDA % 4 == 0 && LDB % 4 == 0, "16-byte aligned shared rows");
};
using TileWide = Tile<16, 512, 8>;
using TileMid = Tile<32, 256, 16>;
using TileStd = Tile<64, 128, 16>;
// one tile over all rows of the sample B = Omega A (l <= 48, 80, 144 rows;
// a few threads idle)
using TileL48 = Tile<48, 160, 16>;
using TileL80 = Tile<80, 96, 16>;
using TileL144 = Tile<144, 56, 16>;

// One TM x TN output tile over k in [k0, k1), accumulated in acc (rows
// 4 ty.., columns 8 tx.. with ty = tid % RG, tx = tid / RG); the next slab of
// both operands is loaded into registers while the current one is multiplied
// from shared memory.
template <class TL, typename TC, typename TA, typename TB, typename TI, typename TO>
__device__ __forceinline__ void tg_tile(const TeamGemm<TC, TA, TB, TI, TO>& op, int64_t i0,
                                        int64_t j0, int64_t k0, int64_t k1, TC (&acc)[4][8],
                                        TC* As, TC* Bs, int64_t* Bcol) {
  const int tid = threadIdx.x;
  const int ty = tid % TL::RG, tx = tid / TL::RG;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = (TC)0;
  // the stored column of each of the tile's TN columns of op(B), read once
  // (a gather through bmap would otherwise put a dependent load in front of
  // every operand load)
  if (k0 < k1) {
    __syncthreads();  // the previous tile no longer reads Bcol
    for (int jj = tid; jj < TL::TN; jj += NT) {
      const int64_t gj = j0 + jj;
      Bcol[jj] = gj < op.N ? (op.bmap ? ldg_i64(op.bmap + gj) : gj) : 0;
    }
  }
  TC ra[TL::NLA], rb[TL::NLB];
  auto load = [&](int64_t kb) {
#pragma unroll
    for (int u = 0; u < TL::NLA; ++u) {
      const int e = tid + NT * u;
      // the fast index follows the stored layout of A
      const int ii = op.at ? e / TL::TK : e % TL::TM;
      const int kk = op.at ? e % TL::TK : e / TL::TM;
      const int64_t gi = i0 + ii, gk = kb + kk;
      ra[u] = (e < TL::TM * TL::TK && gi < op.M && gk < k1)
                  ? (TC)__ldcg(op.at ? op.A + gk + gi * op.lda : op.A + gi + gk * op.lda)
                  : (TC)0;
    }
#pragma unroll
    for (int u = 0; u < TL::NLB; ++u) {
      const int e = tid + NT * u;
      const int kk = e % TL::TK, jj = e / TL::TK;  // k fastest
      const int64_t gj = j0 + jj, gk = kb + kk;
      TC vb = (TC)0;
      if (e < TL::TN * TL::TK && gj < op.N && gk < k1)
        vb = (TC)__ldcg(op.B + op.brow0 + gk + Bcol[jj] * op.ldb);
      rb[u] = vb;
    }
  };
  auto store = [&]() {
#pragma unroll
    for (int u = 0; u < TL::NLA; ++u) {
      const int e = tid + NT * u;
      const int ii = op.at ? e / TL::TK : e % TL::TM;
      const int kk = op.at ? e % TL::TK : e / TL::TM;
      if (e < TL::TM * TL::TK) As[kk * TL::LDA + ii] = ra[u];
    }
#pragma unroll
    for (int u = 0; u < TL::NLB; ++u) {
      const int e = tid + NT * u;
      if (e < TL::TN * TL::TK) Bs[(e % TL::TK) * TL::LDB + e / TL::TK] = rb[u];
    }
  };
  if (k0 >= k1) return;
  __syncthreads();  // Bcol is complete
  load(k0);
  for (int64_t kb = k0; kb < k1; kb += TL::TK) {
    __syncthreads();  // the previous slab is no longer read
    store();
    __syncthreads();
    if (kb + TL::TK < k1) load(kb + TL::TK);
    if (TL::ACTIVE < NT && tid >= TL::ACTIVE) continue;
#pragma unroll
    for (int kk = 0; kk < TL::TK; ++kk) {
      TC a[4], b0[4], b1[4];
      ld4(As + kk * TL::LDA + 4 * ty, a);
      ld4(Bs + kk * TL::LDB + 8 * tx, b0);
      ld4(Bs + kk * TL::LDB + 8 * tx + 4, b1);
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) {
          acc[x][y] = fma(a[x], b0[y], acc[x][y]);
          acc[x][y + 4] = fma(a[x], b1[y], acc[x][y + 4]);
        }
    }
  }
}

// The whole product over the team (CTA g of G) with tile shape TL.  Tiles
// (and, when there are fewer tiles than CTAs and K is long, K splits) are
// dealt round-robin to the team's CTAs; split partial sums go to `part` and
// are added over the splits in order after a team barrier.
template <class TL, typename TC, typename TA, typename TB, typename TI, typename TO>
__device__ bool team_gemm_t(const TeamGemm<TC, TA, TB, TI, TO>& op, int g, int G, TC* part,
                            int64_t part_cap, GridBarrier* bar, int* status, unsigned char* smem) {
  constexpr int TE = TL::TM * TL::TN;  // elements of a tile
  TC* As = reinterpret_cast<TC*>(smem);
  TC* Bs = As + TL::TK * TL::LDA;
  int64_t* Bcol = reinterpret_cast<int64_t*>(Bs + TL::TK * TL::LDB);
  const int64_t tm = (op.M + TL::TM - 1) / TL::TM, tn = (op.N + TL::TN - 1) / TL::TN;
  const int64_t ntile = tm * tn;
  // K splits that balance the work items over the team.  The makespan, in
  // steps of k, is ceil(ntile s / G) (K / s + c [s > 1]): a split item also
  // writes its partial tile and the reduction reads it back, which costs
  // about as much as c = 128 steps of k (measured on GB300).  Each split keeps
  // at least 128 of K and the partial tiles fit in `part`.
  int64_t splits = 1;
  {
    constexpr double kPartialCost = 128.0;
    double best = (double)((ntile + G - 1) / G) * (double)op.K;
    const int64_t smax = std::min<int64_t>((int64_t)4 * G, op.K / 128);
    for (int64_t sp = 2; sp <= smax; ++sp) {
      if (ntile * sp * TE > part_cap) break;
      const double cost =
          (double)((ntile * sp + G - 1) / G) * ((double)op.K / (double)sp + kPartialCost);
      if (cost < best - 1e-9) {
        best = cost;
        splits = sp;
      }
    }
  }
  const int64_t kper = ((op.K + splits - 1) / splits + TL::TK - 1) / TL::TK * TL::TK;
  const int tid = threadIdx.x;
  const int ty = tid % TL::RG, tx = tid / TL::RG;
  const int64_t nitems = ntile * splits;
  for (int64_t w = g; w < nitems; w += G) {
    const int64_t tile = w % ntile, sp = w / ntile;
    const int64_t i0 = (tile % tm) * TL::TM, j0 = (tile / tm) * TL::TN;
    const int64_t k0 = sp * kper, k1 = std::min<int64_t>(op.K, k0 + kper);
    TC acc[4][8];
    tg_tile<TL>(op, i0, j0, k0, k1, acc, As, Bs, Bcol);
    if (TL::ACTIVE < NT && tid >= TL::ACTIVE) continue;
    if (splits == 1) {
#pragma unroll
      for (int y = 0; y < 8; ++y) {
        const int64_t j = j0 + 8 * tx + y;
        if (j >= op.N) continue;
#pragma unroll
        for (int x = 0; x < 4; ++x) {
          const int64_t i = i0 + 4 * ty + x;
          if (i < op.M) tg_epilogue(op, i, j, acc[x][y]);
        }
      }
    } else {
      TC* pw = part + w * TE;
#pragma unroll
      for (int y = 0; y < 8; ++y)
#pragma unroll
        for (int x = 0; x < 4; ++x) pw[(8 * tx + y) * TL::TM + 4 * ty + x] = acc[x][y];
    }
  }
  if (splits > 1) {
    if (!grid_barrier(bar, G, status)) return false;
    for (int64_t e = (int64_t)g * NT + tid; e < ntile * TE; e += (int64_t)G * NT) {
      const int64_t tile = e / TE, loc = e % TE;
      const int64_t i = (tile % tm) * TL::TM + loc % TL::TM;
      const int64_t j = (tile / tm) * TL::TN + loc / TL::TM;
      if (i >= op.M || j >= op.N) continue;
      TC s = (TC)0;
      for (int64_t sp = 0; sp < splits; ++sp) s += __ldcg(part + (sp * ntile + tile) * TE + loc);
      tg_epilogue(op, i, j, s);
    }
  }
  return true;
}

// The sample product B = Omega A (M = l rows): one tile spans every row, so
// the matrix is read once.
template <typename TC, typename TA, typename TB, typename TI, typename TO>
__device__ bool team_gemm_rows(const TeamGemm<TC, TA, TB, TI, TO>& op, int g, int G, TC* part,
                               int64_t part_cap, GridBarrier* bar, int* status,
                               unsigned char* smem) {
  if (op.M <= 0 || op.N <= 0) return true;
  if (op.M <= 48) return team_gemm_t<TileL48>(op, g, G, part, part_cap, bar, status, smem);
  if (op.M <= 80) return team_gemm_t<TileL80>(op, g, G, part, part_cap, bar, status, smem);
  if (op.M <= 144) return team_gemm_t<TileL144>(op, g, G, part, part_cap, bar, status, smem);
  return team_gemm_t<TileStd>(op, g, G, part, part_cap, bar, status, smem);
}

// Every CTA of the team calls it with the same arguments; returns false if a
// team barrier gave up.  The tile shape follows M (the same for every CTA).
template <typename TC, typename TA, typename TB, typename TI, typename TO>
__device__ bool team_gemm(const TeamGemm<TC, TA, TB, TI, TO>& op, int g, int G, TC* part,
                          int64_t part_cap, GridBarrier* bar, int* status, unsigned char* smem) {
  if (op.M <= 0 || op.N <= 0) return true;
  // the tile shape with the least padded area (ties: the taller tile)
  auto padded = [&](int64_t tm_, int64_t tn_) {
    return ((op.M + tm_ - 1) / tm_) * tm_ * ((op.N + tn_ - 1) / tn_) * tn_;
  };
  const int64_t aw = padded(TileWide::TM, TileWide::TN), am = padded(TileMid::TM, TileMid::TN),
                as = padded(TileStd::TM, TileStd::TN);
  if (as <= am && as <= aw)
    return team_gemm_t<TileStd>(op, g, G, part, part_cap, bar, status, smem);
  if (am <= aw) return team_gemm_t<TileMid>(op, g, G, part, part_cap, bar, status, smem);
  return team_gemm_t<TileWide>(op, g, G, part, part_cap, bar, status, smem);
}

// ---------------------------------------------------------------- the kernel
struct TeamCtl {
  rqrcp_problem prob;
  long long ticket;  // index of the claimed problem, -1 = none
  int status;        // the problem's status bits
  int singular;      // exactly singular R11 in the current block
};

struct BatchKernelArgs {
  const rqrcp_problem* table;  // batch mode: device table, nprob entries
  int nprob;
  RequestRing* ring;           // serving mode: mapped ring (table == nullptr)
  unsigned long long* next;    // claim counter (device)
  int* exited;                 // teams that have left the loop
  int G;                       // CTAs per team
  char* scratch;               // team t's scratch at scratch + t * team_bytes
  size_t team_bytes;
  BatchLayout L;
  GridBarrier* bars;           // one per team
  int* status;                 // the handle's status word (ORed)
  unsigned int idle_polls;     // serving mode: bound of an idle wait
  long long* trace;            // per team 8 phase times in ns (instrumentation), or null
};

template <typename T>
__device__ __forceinline__ T* at(char* base, size_t off) {
  return reinterpret_cast<T*>(base + off);
}

__device__ __forceinline__ long long ld_acquire_sys_s64(const long long* p) {
  long long v;
  asm volatile("ld.acquire.sys.global.s64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_acquire_sys_s32(const int* p) {
  int v;
  asm volatile("ld.acquire.sys.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Leader thread of a team: claim the next problem into ctl (ticket -1 when
// the source is exhausted, or, in serving mode, stopped or idle too long).
__device__ void claim(const BatchKernelArgs& a, TeamCtl* ctl) {
  if (a.table != nullptr) {
    const unsigned long long t = atomicAdd(a.next, 1ull);
    if (t < (unsigned long long)a.nprob) {
      ctl->prob = a.table[t];
      ctl->ticket = (long long)t;
    } else {
      ctl->ticket = -1;
    }
    return;
  }
  RequestRing* r = a.ring;
  unsigned int polls = 0;
  for (;;) {
    const unsigned long long cur = *(volatile unsigned long long*)a.next;
    const long long tail = ld_acquire_sys_s64(&r->tail);
    if ((long long)cur < tail) {
      if (atomicCAS(a.next, cur, cur + 1) == cur) {
        const int slot = (int)(cur % (unsigned long long)r->cap);
        const rqrcp_problem* src = reinterpret_cast<const rqrcp_problem*>(r + 1) + slot;
        ctl->prob = *src;
        ctl->ticket = (long long)cur;
        return;
      }
      continue;
    }
    if (ld_acquire_sys_s32(&r->stop) != 0 || ++polls > a.idle_polls) {
      ctl->ticket = -1;
      return;
    }
    __nanosleep(polls < 64 ? 100 : 1000);
  }
}

__device__ __forceinline__ long long global_ns() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Team wall time per phase (instrumentation): the team leader adds the time
// since the previous mark to acc[phase]; acc is null on every other thread
// and when tracing is off.  Phases follow the library's profile phases:
// 0 Omega and sketch, 1 sample QRCP, 2 permutation, 3 panel, T and write-back,
// 5 sample update, 6 products with A, Y and W^T, 7 other (outputs cleared,
// waiting for a problem).
struct Tracer {
  long long* acc;
  long long last;
  __device__ void mark(int phase) {
    if (acc != nullptr) {
      const long long now = global_ns();
      acc[phase] += now - last;
      last = now;
    }
  }
};

#define TEAM_SYNC()                                        \
  do {                                                     \
    if (!grid_barrier(bar, G, &ctl->status)) return false; \
  } while (0)

// Copy of the claimed problem, read through L2 (CTA 0 of the team wrote it).
__device__ __forceinline__ rqrcp_problem load_problem(const TeamCtl* ctl) {
  rqrcp_problem P;
  const long long* src = reinterpret_cast<const long long*>(&ctl->prob);
  long long* dst = reinterpret_cast<long long*>(&P);
#pragma unroll
  for (int i = 0; i < (int)(sizeof(rqrcp_problem) / 8); ++i) dst[i] = __ldcg(src + i);
  return P;
}

// Alg. 6 on ctl->prob by the team (CTA g of G).
__device__ bool run_problem(const BatchKernelArgs& a, char* ts, TeamCtl* ctl, GridBarrier* bar,
                            int g, int G, unsigned char* smem, Tracer& tr) {
  const rqrcp_problem P = load_problem(ctl);
  const BatchLayout& L = a.L;
  const int64_t m = P.m, n = P.n, k = P.k;
  const int b = P.b, ell = P.b + P.p;
  const int tid = threadIdx.x;
  const int64_t gt = (int64_t)g * NT + tid, gstride = (int64_t)G * NT;
  float* om = at<float>(ts, L.omega);    // ell x m, ld ell
  double* B = at<double>(ts, L.B);       // ell x n, ld ell
  float* Wt = at<float>(ts, L.Wt);       // k x n, ld k
  double* P64 = at<double>(ts, L.P64);   // m x b, ld m
  double* T = at<double>(ts, L.T);       // b x b
  float* T32 = at<float>(ts, L.T32);     // b x b
  float* Z32 = at<float>(ts, L.Z32);     // b x n, ld b
  float* YY = at<float>(ts, L.YY);       // b x k, ld b
  double* W11 = at<double>(ts, L.W11);   // b x b
  int64_t* swaps = at<int64_t>(ts, L.swaps);
  int* mp = at<int>(ts, L.map);          // [0] count, then (dst, src) pairs
  float* cbuf = at<float>(ts, L.cbuf);   // 2 x (2b) x k floats
  int64_t* jbuf = at<int64_t>(ts, L.jbuf);
  void* part = at<void>(ts, L.part);
  const int64_t part_elems = L.part_elems;
  int* st = &ctl->status;

  // ---- outputs start at zero / identity; Omega (FP32 Box-Muller)
  for (int64_t c = gt; c < n; c += gstride) P.d_jpvt[c] = c;
  for (int64_t e = gt; e < m * k; e += gstride) P.dY[e % m + (e / m) * P.ldy] = 0.0f;
  for (int64_t e = gt; e < k * n; e += gstride) {
    P.dR[e % k + (e / k) * P.ldr] = 0.0f;
    Wt[e] = 0.0f;
  }
  {
    const int64_t npairs = (ell + 1) / 2;
    const uint2 key = make_uint2((uint32_t)P.seed, (uint32_t)(P.seed >> 32));
    for (int64_t e = gt; e < npairs * m; e += gstride) {
      const int64_t q = e % npairs, r = e / npairs;
      const uint4 c = make_uint4((uint32_t)(uint64_t)r, (uint32_t)((uint64_t)r >> 32), (uint32_t)q,
                                 kOmegaStreamId);
      const uint4 x = px::philox10(c, key);
      const float u1 = (float)px::unit_open(x.x, x.y);
      const float u2 = (float)px::unit_open(x.z, x.w);
      const float rho = sqrtf(-2.0f * logf(u1));
      float s, co;
      sincospif(2.0f * u2, &s, &co);
      om[2 * q + r * ell] = rho * co;
      if (2 * q + 1 < ell) om[2 * q + 1 + r * ell] = rho * s;
    }
  }
  TEAM_SYNC();
  tr.mark(7);
  // ---- the sample B = Omega A (ell x n)
  {
    TeamGemm<float, float, float, float, double> op{ell, n, m, om, ell, 0, P.dA, P.lda, nullptr, 0,
                                                    nullptr, 0, nullptr, 0, B, ell, 1.0f, 0.0f};
    if (!team_gemm_rows(op, g, G, (float*)part, part_elems, bar, st, smem)) return false;
  }
  TEAM_SYNC();
  tr.mark(0);

  for (int64_t j0 = 0; j0 < k; j0 += b) {
    const int bJ = (int)std::min<int64_t>(b, k - j0);
    const int64_t nc = n - j0, n2 = nc - bJ, mJ = m - j0;
    double* Bblk = B + j0 * ell;
    // ---- b pivots from the sample (Alg. 1 halted); S left in B
    {
      SampleQrcpArgs sa{Bblk, ell, ell, nc, bJ, swaps, at<double>(ts, L.cand),
                        at<double>(ts, L.candcol), bar, st};
      sq::sample_qrcp_body<float>(sa, g, G, smem);
    }
    TEAM_SYNC();
    tr.mark(1);
    // ---- compose the swaps into (destination, source) position pairs
    if (g == 0 && tid < 32) {
      int* pos = reinterpret_cast<int*>(smem);
      int* src = pos + 2 * MAXB;
      int* sw = src + 2 * MAXB;
      int cnt = 0;
      const int lane = tid;
      // the whole swap list in one round of loads (the loop is sequential)
      for (int t = lane; t < bJ; t += 32) sw[t] = (int)__ldcg(swaps + t);
      __syncwarp();
      for (int i = 0; i < bJ; ++i) {
        const int s = sw[i];
        if (s == i) continue;
        // entries holding positions i and s (or -1)
        int ei = -1, es = -1;
        for (int q0 = 0; q0 < cnt; q0 += 32) {
          const int q = q0 + lane;
          const int p = q < cnt ? pos[q] : -1;
          const unsigned bi = __ballot_sync(0xffffffffu, p == i);
          const unsigned bs = __ballot_sync(0xffffffffu, p == s);
          if (bi && ei < 0) ei = q0 + __ffs(bi) - 1;
          if (bs && es < 0) es = q0 + __ffs(bs) - 1;
        }
        const int vi = ei >= 0 ? src[ei] : i;
        const int vs = es >= 0 ? src[es] : s;
        __syncwarp();
        if (lane == 0) {
          if (ei < 0) {
            ei = cnt++;
            pos[ei] = i;
          }
          if (es < 0) {
            es = cnt++;
            pos[es] = s;
          }
          src[ei] = vs;
          src[es] = vi;
        }
        ei = __shfl_sync(0xffffffffu, ei, 0);
        es = __shfl_sync(0xffffffffu, es, 0);
        cnt = __shfl_sync(0xffffffffu, cnt, 0);
        __syncwarp();
      }
      for (int q = lane; q < cnt; q += 32) {
        mp[1 + 2 * q] = pos[q];
        mp[2 + 2 * q] = src[q];
      }
      if (lane == 0) mp[0] = cnt;
    }
    TEAM_SYNC();
    // ---- move jpvt, the W^T rows and the R rows computed so far (gather, then scatter)
    {
      const int cnt = __ldcg(mp);
      const int64_t rows = j0;  // rows 0..j0-1 of W^T and R are filled
      for (int64_t e = gt; e < (int64_t)cnt * (2 * rows + 1); e += gstride) {
        const int q = (int)(e % cnt);
        const int64_t r = e / cnt;
        const int64_t from = j0 + __ldcg(mp + 2 + 2 * q);
        if (r == 2 * rows) {
          jbuf[q] = ldg_i64(P.d_jpvt + from);
        } else if (r < rows) {
          cbuf[r + (int64_t)q * rows] = __ldcg(Wt + r + from * k);
        } else {
          const int64_t rr = r - rows;
          cbuf[(int64_t)cnt * rows + rr + (int64_t)q * rows] = __ldcg(P.dR + rr + from * P.ldr);
        }
      }
      TEAM_SYNC();
      for (int64_t e = gt; e < (int64_t)cnt * (2 * rows + 1); e += gstride) {
        const int q = (int)(e % cnt);
        const int64_t r = e / cnt;
        const int64_t to = j0 + __ldcg(mp + 1 + 2 * q);
        if (r == 2 * rows) {
          P.d_jpvt[to] = ldg_i64(jbuf + q);
        } else if (r < rows) {
          Wt[r + to * k] = __ldcg(cbuf + r + (int64_t)q * rows);
        } else {
          const int64_t rr = r - rows;
          P.dR[rr + to * P.ldr] = __ldcg(cbuf + (int64_t)cnt * rows + rr + (int64_t)q * rows);
        }
      }
    }
    TEAM_SYNC();
    tr.mark(2);
    // ---- A_hat = A(j0:m, sel) - Y(j0:m, 0:j0) W^T(0:j0, sel), into the FP64 panel
    {
      TeamGemm<float, float, float, float, double> op{
          mJ, bJ, j0, P.dY + j0, P.ldy, 0, Wt + j0 * k, k, nullptr, 0,
          P.dA, P.lda, P.d_jpvt + j0, j0, P64, m, -1.0f, 1.0f};
      if (!team_gemm(op, g, G, (float*)part, part_elems, bar, st, smem)) return false;
    }
    TEAM_SYNC();
    tr.mark(6);
    // ---- panel QR and T (FP64), reflectors rounded to FP32
    {
      PanelArgs pa{P64, m, mJ, bJ, P.d_tau + j0, T, at<double>(ts, L.ppart),
                   at<double>(ts, L.rowj), bar, st, 1};
      pn::panel_body(pa, g, G, smem);
    }
    TEAM_SYNC();
    // ---- Y (explicit FP32), R11 (FP32, diagonal also FP64), T in FP32
    for (int64_t e = gt; e < mJ * bJ; e += gstride) {
      const int64_t i = e % mJ, c = e / mJ;
      const double v = __ldcg(P64 + i + c * m);
      P.dY[(j0 + i) + (j0 + c) * P.ldy] = i > c ? (float)v : (i == c ? 1.0f : 0.0f);
      if (i <= c) P.dR[(j0 + i) + (j0 + c) * P.ldr] = (float)v;
      if (i == c) P.d_rdiag[j0 + c] = v;
    }
    for (int64_t e = gt; e < (int64_t)bJ * bJ; e += gstride) T32[e] = (float)__ldcg(T + e);
    TEAM_SYNC();
    tr.mark(3);
    if (n2 > 0) {
      const int64_t* tcols = P.d_jpvt + j0 + bJ;
      const float* Y2 = P.dY + j0 + j0 * P.ldy;
      // Z = Y2^T A(j0:m, trailing)
      {
        TeamGemm<float, float, float, float, float> op{
            bJ, n2, mJ, Y2, P.ldy, 1, P.dA, P.lda, tcols, j0,
            nullptr, 0, nullptr, 0, Z32, bJ, 1.0f, 0.0f};
        if (!team_gemm(op, g, G, (float*)part, part_elems, bar, st, smem)) return false;
      }
      if (j0 > 0) {
        // YY = Y2^T Y1, then Z -= YY W1^T(:, trailing)
        TeamGemm<float, float, float, float, float> op1{
            bJ, j0, mJ, Y2, P.ldy, 1, P.dY + j0, P.ldy, nullptr, 0,
            nullptr, 0, nullptr, 0, YY, bJ, 1.0f, 0.0f};
        if (!team_gemm(op1, g, G, (float*)part, part_elems, bar, st, smem)) return false;
        TEAM_SYNC();
        TeamGemm<float, float, float, float, float> op2{
            bJ, n2, j0, YY, bJ, 0, Wt + (j0 + bJ) * k, k, nullptr, 0,
            Z32, bJ, nullptr, 0, Z32, bJ, -1.0f, 1.0f};
        if (!team_gemm(op2, g, G, (float*)part, part_elems, bar, st, smem)) return false;
      }
      TEAM_SYNC();
      // W2^T(:, trailing) = T2^T Z
      {
        TeamGemm<float, float, float, float, float> op{
            bJ, n2, bJ, T32, bJ, 1, Z32, bJ, nullptr, 0,
            nullptr, 0, nullptr, 0, Wt + j0 + (j0 + bJ) * k, k, 1.0f, 0.0f};
        if (!team_gemm(op, g, G, (float*)part, part_elems, bar, st, smem)) return false;
      }
      TEAM_SYNC();
      // R(j0:j0+bJ, trailing) = A(j0:j0+bJ, trailing) - Y(j0:j0+bJ, 0:j0+bJ) W^T(0:j0+bJ, trailing)
      {
        TeamGemm<float, float, float, float, float> op{
            bJ, n2, j0 + bJ, P.dY + j0, P.ldy, 0, Wt + (j0 + bJ) * k, k, nullptr, 0,
            P.dA, P.lda, tcols, j0, P.dR + j0 + (j0 + bJ) * P.ldr, P.ldr, -1.0f, 1.0f};
        if (!team_gemm(op, g, G, (float*)part, part_elems, bar, st, smem)) return false;
      }
      TEAM_SYNC();
      tr.mark(6);
    }
    if (j0 + bJ < k) {
      // ---- Eq. (3): W11 = S11 R11^-1 (FP64), one warp per row of W11
      double* Rs = reinterpret_cast<double*>(smem);  // bJ x bJ upper, ld bJ
      double* rinv = Rs + (size_t)bJ * bJ;
      __shared__ int s_sing;
      if (tid == 0) s_sing = 0;
      __syncthreads();
      for (int e = tid; e < bJ * bJ; e += NT) {
        const int r = e % bJ, c = e / bJ;
        Rs[e] = r <= c ? __ldcg(P64 + r + (int64_t)c * m) : 0.0;
      }
      for (int j = tid; j < bJ; j += NT) {
        const double d = __ldcg(P64 + j + (int64_t)j * m);
        if (d == 0.0) s_sing = 1;
        rinv[j] = 1.0 / d;
      }
      __syncthreads();
      const int sing = s_sing;
      const int lane = tid & 31, warp = tid >> 5;
      if (!sing) {
        for (int r = g * (NT / 32) + warp; r < bJ; r += G * (NT / 32)) {
          double acc[MAXB / 32];
#pragma unroll
          for (int q = 0; q < MAXB / 32; ++q) {
            const int c = lane + 32 * q;
            acc[q] = (c < bJ && c >= r) ? __ldcg(Bblk + r + (int64_t)c * ell) : 0.0;
          }
          for (int j = r; j < bJ; ++j) {
            double mine = 0.0;
#pragma unroll
            for (int q = 0; q < MAXB / 32; ++q)
              if (q == (j >> 5)) mine = acc[q];
            const double wj = __shfl_sync(0xffffffffu, mine * rinv[j], j & 31);
#pragma unroll
            for (int q = 0; q < MAXB / 32; ++q) {
              const int c = lane + 32 * q;
              if (c > j && c < bJ) acc[q] = fma(-wj, Rs[j + c * bJ], acc[q]);
              if (c == j) acc[q] = wj;
            }
          }
#pragma unroll
          for (int q = 0; q < MAXB / 32; ++q) {
            const int c = lane + 32 * q;
            if (c < bJ) W11[r + (int64_t)c * bJ] = c >= r ? acc[q] : 0.0;
          }
        }
      } else if (g == 0 && tid == 0) {
        atomicOr(st, RQRCP_INFO_RESAMPLED);
      }
      TEAM_SYNC();
      if (!sing && n2 > 0) {
        // B1 = S12 - W11 R12 in place (rows 0..bJ-1 of the next sample); B2 = S22 stays
        double* Bnext = Bblk + (int64_t)bJ * ell;
        TeamGemm<double, double, float, double, double> op{
            bJ, n2, bJ, W11, bJ, 0, P.dR + j0 + (j0 + bJ) * P.ldr, P.ldr, nullptr, 0,
            Bnext, ell, nullptr, 0, Bnext, ell, -1.0, 1.0};
        if (!team_gemm(op, g, G, (double*)part, part_elems / 2, bar, st, smem)) return false;
      }
      TEAM_SYNC();
      tr.mark(5);
    }
  }
  return true;
}

__global__ void __launch_bounds__(NT, 1) batch_trqrcp_kernel(BatchKernelArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int G = a.G;
  const int team = blockIdx.x / G, g = blockIdx.x % G;
  char* ts = a.scratch + (size_t)team * a.team_bytes;
  TeamCtl* ctl = at<TeamCtl>(ts, a.L.ctl);
  GridBarrier* bar = a.bars + team;
  Tracer tr{(a.trace != nullptr && g == 0 && threadIdx.x == 0) ? a.trace + 8 * team : nullptr,
            global_ns()};
  for (;;) {
    if (g == 0 && threadIdx.x == 0) {
      claim(a, ctl);
      ctl->status = 0;
    }
    if (!grid_barrier(bar, G, a.status)) break;
    tr.mark(7);
    const long long ticket = __ldcg(&ctl->ticket);
    if (ticket < 0) break;
    const bool ok = run_problem(a, ts, ctl, bar, g, G, smem_raw, tr);
    if (g == 0 && threadIdx.x == 0) {
      const int s = __ldcg(&ctl->status);
      if (s) atomicOr(a.status, s);
      if (a.ring != nullptr) {
        // publish the result: info word, then the completion word (the
        // ticket + 1) with release semantics at system scope
        RequestRing* r = a.ring;
        const int slot = (int)(ticket % r->cap);
        int* info = reinterpret_cast<int*>(reinterpret_cast<rqrcp_problem*>(r + 1) + r->cap);
        long long* done = reinterpret_cast<long long*>(info + ((r->cap + 1) & ~1));
        info[slot] = s;
        __threadfence_system();
        asm volatile("st.release.sys.global.s64 [%0], %1;" ::"l"(done + slot), "l"(ticket + 1)
                     : "memory");
      }
    }
    if (!ok) {
      atomicOr(a.status, RQRCP_INFO_TIMEOUT);
      break;
    }
  }
  // serving: the last team to leave tells the host that nothing runs any more
  if (a.ring != nullptr && g == 0 && threadIdx.x == 0) {
    const int teams = (int)(gridDim.x / G);
    if (atomicAdd(a.exited, 1) == teams - 1) {
      __threadfence_system();
      asm volatile("st.release.sys.global.s32 [%0], %1;" ::"l"(&a.ring->running), "r"(0)
                   : "memory");
    }
  }
}

}  // namespace

size_t batch_team_bytes(const BatchLimits& lim, int G, BatchLayout* L) {
  BatchLayout l{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    off = (off + 255) & ~(size_t)255;
    const size_t o = off;
    off += bytes;
    return o;
  };
  const size_t ell = lim.ell, b = lim.b, m = lim.m, n = lim.n, k = lim.k;
  l.ctl = take(sizeof(TeamCtl));
  l.omega = take(sizeof(float) * ell * m);
  l.B = take(sizeof(double) * ell * n);
  l.Wt = take(sizeof(float) * k * n);
  l.P64 = take(sizeof(double) * m * b);
  l.T = take(sizeof(double) * b * b);
  l.T32 = take(sizeof(float) * b * b);
  l.Z32 = take(sizeof(float) * b * n);
  l.YY = take(sizeof(float) * b * k);
  l.W11 = take(sizeof(double) * b * b);
  l.swaps = take(sizeof(int64_t) * b);
  l.map = take(sizeof(int) * (1 + 4 * b));
  l.cbuf = take(sizeof(float) * 2 * (2 * b) * k);
  l.jbuf = take(sizeof(int64_t) * 2 * b);
  l.cand = take(sizeof(double) * 2 * G * 4);
  l.candcol = take(sizeof(double) * 2 * G * ell);
  l.ppart = take(sizeof(double) * panel_partial_doubles(G, (int)b));
  l.rowj = take(sizeof(double) * 2 * b);
  l.part_elems = (int64_t)4 * G * 8192 * 2;  // floats (half as many doubles): 4G tiles of 8192
  l.part = take(sizeof(float) * (size_t)l.part_elems);
  if (L) *L = l;
  return (off + 255) & ~(size_t)255;
}

// the kernel's dynamic shared memory: its static arrays (the panel's partial
// sums and a few words) stay within the 227 KB per CTA
constexpr size_t kBatchSmem = 200 * 1024;

bool batch_fits(int64_t m, int64_t n, int b, int ell, int G) {
  if (b < 1 || b > MAXB || ell > 192 || G < 1) return false;
  const int64_t cs = (n + G - 1) / G, cp = (m + G - 1) / G;
  if (sq::sample_qrcp_smem_bytes(ell, cs, sizeof(float)) > kBatchSmem) return false;
  if (pn::panel_smem_bytes(cp, b) > kBatchSmem) return false;
  if (((size_t)b * b + b) * 8 > kBatchSmem) return false;
  return true;
}

cudaError_t launch_batch_trqrcp(const BatchLaunch& bl, cudaStream_t st) {
  static std::atomic<uint64_t> attr_done{0};
  cudaError_t e = ensure_smem_attr(batch_trqrcp_kernel, (int)kBatchSmem, attr_done);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(bl.bars, 0, sizeof(GridBarrier) * bl.teams, st);
  if (e != cudaSuccess) return e;
  if (!bl.keep_next) {
    e = cudaMemsetAsync(bl.next, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
  }
  e = cudaMemsetAsync(bl.exited, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  BatchKernelArgs a{bl.table, bl.nprob, bl.ring, bl.next,   bl.exited,     bl.G,
                    bl.scratch, bl.team_bytes, bl.L, bl.bars, bl.status, bl.idle_polls,
                    bl.trace};
  void* params[] = {&a};
  return cudaLaunchCooperativeKernel((const void*)batch_trqrcp_kernel,
                                     dim3((unsigned)(bl.teams * bl.G)), dim3(NT), params,
                                     kBatchSmem, st);
}

}  // namespace rq

namespace rq {
size_t request_ring_bytes(int cap) {
  return sizeof(RequestRing) + sizeof(rqrcp_problem) * (size_t)cap +
         sizeof(int) * (size_t)((cap + 1) & ~1) + sizeof(long long) * (size_t)cap;
}
}  // namespace rq
