// FP64-accurate GEMM on the BF16 tensor cores (tcgen05, sm_103a) by exact
// operand slicing -- the FP64 form of the trailing update of Alg. 4
// (W = T^T Y^T A2, A2 -= Y W) when the GPU's FP64 pipe (~1.25 TFLOP/s on a
// GB300) is the bottleneck.
//
// Slicing (launch_oz_slice, a memory-bound pass per operand).  Row r of an operand
// (K values x_k) gets the power-of-two scale 2^e_r with max_k |x_k| < 2^e_r;
// t = x 2^-e_r lies in (-1, 1) and is cut into S = 7 slices of 8 bits,
//   t = sum_s y_s 2^{-8s} + (|rest| < 2^-56),  y_s integer in [-255, 255],
// each slice value y_s 2^{-8s} exactly representable in BF16.  The slices are
// stored in pairs: for pair q (slices 2q+1, 2q+2) and each 32-wide k chunk a
// row holds 64 values [slice 2q+1, k 0..31 | slice 2q+2, k 0..31], so one
// 128-byte swizzled shared-memory row feeds the MMA with two slices.
//
// Products.  C_ij = 2^{e_i + f_j} sum_{s,t} sum_k a_s(i,k) b_t(k,j).  The pairs
// with s + t = d carry the common grid 2^{-8d}; with K <= 64 per accumulation
// their sum is an integer multiple of that grid below (d-1) 64 255^2 < 2^24
// units for d <= 5, hence EXACT in an FP32 accumulator whatever the tensor
// core's rounding (it truncates).  d = 2..5 get one accumulator each; d = 6
// gets one (its terms are below 2^-32 of the leading ones, so the truncation
// of its 20 MMA additions per accumulation stays below 2^-42 of the leading
// scale); d = 7, 8 share one (below 2^-40); pairs with s + t > 8 are dropped
// (below 2^-56).  28 BF16 MMAs per 16-wide k step.
//
// Kernel (oz_gemm_kernel): persistent, one CTA per SM, 128 x 64 output tiles,
// split-K units, 10 warps:
//   warp 0      one thread issues the TMA copies (per 32-k stage one 3-D box
//               per operand: 64 values x rows x 4 pairs) into a two-stage
//               shared-memory ring, refilling a slot as soon as its MMAs end;
//   warp 1      allocates tensor memory; one thread issues the 56 MMAs of a
//               stage into the six accumulators (6 x 64 tensor-memory
//               columns), which accumulate over two stages (64 k);
//   warps 2-9   drain: after every two stages, warp w adds the six group sums
//               of lanes 32 (w % 4).. (one output row per thread, 32 of the 64
//               columns) into running double-FP32 sums (error-free TwoSum),
//               smallest first; at the end of a unit it writes
//               C = alpha 2^{e_i + f_j} (hi + lo) + beta C (or the split's hi
//               and lo to the partial-sum buffer).  With alpha = +-1 and
//               beta in {0, 1} the scaled hi and lo are built as FP64 bit
//               fields with integer operations, so an output element costs
//               two FP64 additions.
// Every mbarrier wait is bounded; on timeout the status word gets
// RQRCP_INFO_TIMEOUT, each role stops, in-flight copies and MMAs are waited
// for (bounded) and the tensor memory is freed.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "kernels.cuh"
#include "tcgen05.cuh"

namespace rq {
namespace {

using namespace tc;

constexpr int OZ_S = 7;        // slices per operand
constexpr int OZ_PAIRS = 4;    // slice pairs per operand (the eighth slot is zero)
constexpr int OZ_BITS = 8;     // bits per slice
constexpr int OZ_NG = 6;       // accumulators: d = 2, 3, 4, 5, 6 and d >= 7
constexpr int OZ_BM = 128;     // tile rows (A role), UMMA M
constexpr int OZ_BN = 64;      // tile columns (B role), UMMA N
constexpr int OZ_BK = 32;      // k per stage
constexpr int OZ_DR = 2;       // stages per accumulation (drain every 64 k)
constexpr int OZ_KP = 64;      // K padding of the slice buffers
constexpr int OZ_NST = 2;      // shared-memory ring stages
constexpr int OZ_NT = 320;     // warp 0 TMA, warp 1 MMA issue, warps 2..9 drain
constexpr int OZ_CPT = 32;     // output columns per drain thread (two warps per lane quadrant)
constexpr int OZ_PT_A = OZ_BM * 128;          // bytes of one A pair tile
constexpr int OZ_PT_B = OZ_BN * 128;          // bytes of one B pair tile
constexpr int OZ_STAGE_A = OZ_PAIRS * OZ_PT_A;
constexpr int OZ_STAGE = OZ_PAIRS * (OZ_PT_A + OZ_PT_B);
constexpr uint32_t OZ_IDESC = idesc_bf16_f32(OZ_BM, OZ_BN);
constexpr uint32_t OZ_TCOLS = 512;  // power of two >= 6 x 64

// group of the diagonal d = s + t (s, t >= 1)
__host__ __device__ constexpr int oz_group(int d) { return d - 2 < OZ_NG - 1 ? d - 2 : OZ_NG - 1; }

int64_t rpad128(int64_t R) { return (R + OZ_BM - 1) / OZ_BM * OZ_BM; }

// Split-K factor for `tiles` output tiles of KT stages on nsm persistent CTAs:
// the smallest busiest-CTA stage count (rounds of units x stages per unit),
// counting a split's partial-sum pass as two stages; at most `smax` splits.
int pick_splits(int64_t tiles, int KT, int nsm, int smax) {
  int best = 1;
  int64_t best_cost = -1;
  for (int sp = 1; sp <= smax && sp <= KT; ++sp) {
    const int64_t rounds = (tiles * sp + nsm - 1) / nsm;
    const int64_t per = (KT + sp - 1) / sp;
    const int64_t cost = rounds * per + (sp > 1 ? 2 : 0);
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      best = sp;
    }
  }
  return best;
}

// ---------------------------------------------------------------- slicing
// Rows of op(X): KC -> element (r, k) at X[r * ld + k] (a stored column per
// row); otherwise at X[r + k * ld].  amode 1: X is a unit-lower reflector
// block stored in place (above the diagonal 0, diagonal 1; the diagonal is
// the stored (row, col) with row == col).
template <bool KC, int AMODE>
__device__ __forceinline__ double oz_elem(const double* __restrict__ X, int64_t ld, int64_t r,
                                          int64_t k) {
  const int64_t sr = KC ? k : r, sc = KC ? r : k;  // stored (row, col)
  if (AMODE == 1) {
    if (sr < sc) return 0.0;
    if (sr == sc) return 1.0;
  }
  return X[sr + sc * ld];
}

// The slicing runs on integer bit fields only (the GPU's FP64 pipe is too
// slow for a per-element pass): |x| = m 2^(E - 1075) with a 53-bit integer
// m, T = |t| 2^56 = m 2^(E - 1075 + 56 - e) < 2^56, and slice s (1-based) is
// the byte (T >> (56 - 8s)) & 255 with the sign of x.
// exps[r] holds F_r, the biased FP64 exponent field of max_k |x_rk| (0 when
// the row is zero or subnormal); the scale is e_r = max(F_r, 1) - 1022, so
// that max |x| < 2^e_r.
__device__ __forceinline__ int oz_scale_exp(int field) { return (field > 1 ? field : 1) - 1022; }

__device__ __forceinline__ int oz_field(double x) {
  return (int)(((unsigned long long)__double_as_longlong(x) >> 52) & 0x7FFull);
}

// Output (Rp rows, Kp multiple of 64): pair q, row r, k chunk c (32 wide):
// out[((q * Rp + r) * (Kp / 32) + c) * 64 + h * 32 + kk] = slice 2q + h + 1 at
// k = 32 c + kk; rows r >= R and the eighth slot are zero.
template <bool KC, int AMODE>
__device__ __forceinline__ unsigned long long oz_fixed(const double* __restrict__ X, int64_t ld,
                                                       int64_t R, int64_t K, int64_t r, int64_t k,
                                                       int e, bool& neg) {
  unsigned long long T = 0;
  neg = false;
  if (r < R && k < K) {
    const unsigned long long b =
        (unsigned long long)__double_as_longlong(oz_elem<KC, AMODE>(X, ld, r, k));
    neg = (b >> 63) != 0;
    const int E = (int)((b >> 52) & 0x7FF);
    unsigned long long m = b & 0x000FFFFFFFFFFFFFull;
    int Eu = E;
    if (E != 0) m |= 0x0010000000000000ull;
    else Eu = 1;
    const int sh = Eu - 1075 + 56 - e;  // <= 3
    if (sh >= 0) T = m << sh;
    else if (sh > -64) T = m >> (-sh);
  }
  return T;
}

__device__ __forceinline__ float oz_slice_val(unsigned long long T, bool neg, int s) {
  const float y = (float)(unsigned)((T >> (8 * (OZ_S - 1 - s))) & 0xFFull);
  return ldexpf(neg ? -y : y, -OZ_BITS * (s + 1));  // exact
}

// Slices of elements k and k + 1 (k even) of row r: one 4-byte store per
// slice (the eighth slot of the last pair is never read and not written).
template <bool KC, int AMODE>
__device__ __forceinline__ void oz_slice_two(const double* __restrict__ X, int64_t ld, int64_t R,
                                             int64_t K, int64_t Rp, int64_t Kp, int64_t r,
                                             int64_t k, int e, __nv_bfloat16* __restrict__ out) {
  bool n0, n1;
  const unsigned long long T0 = oz_fixed<KC, AMODE>(X, ld, R, K, r, k, e, n0);
  const unsigned long long T1 = oz_fixed<KC, AMODE>(X, ld, R, K, r, k + 1, e, n1);
  const size_t pstride = (size_t)Rp * Kp * 2;  // elements per pair plane
  __nv_bfloat16* p = out + (size_t)r * (Kp / 32) * 64 + (k >> 5) * 64 + (k & 31);
#pragma unroll
  for (int s = 0; s < OZ_S; ++s) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(oz_slice_val(T0, n0, s), oz_slice_val(T1, n1, s));
    *reinterpret_cast<__nv_bfloat162*>(p + (size_t)(s >> 1) * pstride + (s & 1) * 32) = v;
  }
}

// Row-contiguous source (element (r, k) at X[r + k ld], small K): one warp per
// row finds the maximum and slices the row.
template <int AMODE>
__global__ void oz_slice_rows(const double* __restrict__ X, int64_t ld, int64_t R, int64_t K,
                              int64_t Rp, int64_t Kp, __nv_bfloat16* __restrict__ out,
                              int* __restrict__ exps) {
  const int lane = threadIdx.x & 31;
  const int64_t r = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  if (r >= Rp) return;
  int f = 0;
  if (r < R)
    for (int64_t k = lane; k < K; k += 32) f = max(f, oz_field(oz_elem<false, AMODE>(X, ld, r, k)));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) f = max(f, __shfl_xor_sync(0xffffffffu, f, o));
  if (lane == 0 && r < R) exps[r] = f;
  const int e = oz_scale_exp(f);
  for (int64_t k = 2 * lane; k < Kp; k += 64)
    oz_slice_two<false, AMODE>(X, ld, R, K, Rp, Kp, r, k, e, out);
}

// Column-contiguous source (element (r, k) at X[r ld + k], K may be long):
// pass 1 takes the maximum exponent field of each (row, 1024-wide k chunk)
// into exps[r] (zeroed before) with an integer atomic maximum; pass 2 slices
// each (row, k chunk) with the row's scale.  One warp per (row, chunk).
constexpr int OZ_KCH = 1024;

template <int AMODE>
__global__ void oz_rowmax_cols(const double* __restrict__ X, int64_t ld, int64_t R, int64_t K,
                               int* __restrict__ exps) {
  const int lane = threadIdx.x & 31;
  const int64_t r = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  if (r >= R) return;
  const int64_t k0 = (int64_t)blockIdx.y * OZ_KCH, k1 = imin64(K, k0 + OZ_KCH);
  int f = 0;
  for (int64_t k = k0 + lane; k < k1; k += 32) f = max(f, oz_field(oz_elem<true, AMODE>(X, ld, r, k)));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) f = max(f, __shfl_xor_sync(0xffffffffu, f, o));
  if (lane == 0 && f > 0) atomicMax(exps + r, f);
}

template <int AMODE>
__global__ void oz_slice_cols(const double* __restrict__ X, int64_t ld, int64_t R, int64_t K,
                              int64_t Rp, int64_t Kp, __nv_bfloat16* __restrict__ out,
                              const int* __restrict__ exps) {
  const int lane = threadIdx.x & 31;
  const int64_t r = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  if (r >= Rp) return;
  const int e = oz_scale_exp(r < R ? exps[r] : 0);
  const int64_t k0 = (int64_t)blockIdx.y * OZ_KCH, k1 = imin64(Kp, k0 + OZ_KCH);
  for (int64_t k = k0 + 2 * lane; k < k1; k += 64)
    oz_slice_two<true, AMODE>(X, ld, R, K, Rp, Kp, r, k, e, out);
}

// ---------------------------------------------------------------- GEMM
struct OzArgs {
  int64_t M, N;
  int KT;             // 32-k stages
  int kt_per_split;
  int tiles_m, tiles_n, units;
  double alpha, beta;
  double* C;
  int64_t ldc;
  const int* expA;
  const int* expB;
  float* part;        // splits > 1: hi at part[2z MN + r + c M], lo at part[(2z+1) MN + ...]
  int* status;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& err) {
  s = a + b;
  const float bb = s - a;
  err = (a - (s - bb)) + (b - bb);
}

// x 2^e as an FP64 value (sign flipped by neg = 0x80000000), built from the
// FP32 bit fields with integer operations; exact.  FP32 subnormals and
// results outside the normal FP64 range take the (rare) FP64 path.
__device__ __forceinline__ double scaled_f64(float x, int e, uint32_t neg) {
  const uint32_t b = __float_as_uint(x) ^ neg;
  const uint32_t ex = (b >> 23) & 0xFFu;
  if ((b & 0x7FFFFFFFu) == 0u) return 0.0;
  const int e64 = (int)ex - 127 + 1023 + e;
  if (ex == 0u || e64 <= 0 || e64 >= 2047) return ldexp((double)__uint_as_float(b), e);
  const uint32_t hiw = (b & 0x80000000u) | ((uint32_t)e64 << 20) | ((b >> 3) & 0xFFFFFu);
  const uint32_t low = (b & 7u) << 29;
  return __hiloint2double((int)hiw, (int)low);
}

__device__ __forceinline__ double pow2(int e) {
  return (e >= -1022 && e <= 1023) ? __longlong_as_double((long long)(e + 1023) << 52)
                                   : ldexp(1.0, e);
}

__global__ void __launch_bounds__(OZ_NT, 1)
    oz_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   OzArgs g) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full[OZ_NST], empty[OZ_NST], tfull, tempty, done;
  __shared__ uint32_t s_tmem;
  __shared__ volatile int s_fail;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int i = 0; i < OZ_NST; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    mbar_init(&tfull, 1);
    mbar_init(&tempty, 8);
    mbar_init(&done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_fail = 0;
  }
  if (warp == 1) tmem_alloc(&s_tmem, OZ_TCOLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;

  auto stage_a = [&](int st) { return smem + (size_t)st * OZ_STAGE; };
  auto stage_b = [&](int st) { return smem + (size_t)st * OZ_STAGE + OZ_STAGE_A; };

  if (warp == 0) {
    // ------------------------------------------------ TMA producer
    // refills each ring slot as soon as the MMAs that read it have completed
    if (lane == 0) {
      int lst = 0;
      uint32_t lpar = 0u, lused = 0u;
      bool ok = true;
      for (int u = blockIdx.x; u < g.units && ok; u += gridDim.x) {
        const int tm = u % g.tiles_m, rest = u / g.tiles_m;
        const int tn = rest % g.tiles_n;
        const int kb = (rest / g.tiles_n) * g.kt_per_split, ke = min(g.KT, kb + g.kt_per_split);
        for (int kt = kb; kt < ke; ++kt) {
          if (!mbar_wait(&empty[lst], ((lpar >> lst) & 1u) ^ 1u) || s_fail) {
            ok = false;
            break;
          }
          mbar_expect_tx(&full[lst], OZ_STAGE);
          tma_load_3d(stage_a(lst), &tmA, kt * 64, tm * OZ_BM, 0, &full[lst]);
          tma_load_3d(stage_b(lst), &tmB, kt * 64, tn * OZ_BN, 0, &full[lst]);
          lpar ^= 1u << lst;
          lused |= 1u << lst;
          lst = (lst + 1 == OZ_NST) ? 0 : lst + 1;
        }
      }
      if (!ok) {
        s_fail = 1;
        // wait (bounded) for the last copy issued on each slot
        for (int i = 0; i < OZ_NST; ++i)
          if ((lused >> i) & 1u) mbar_wait(&full[i], ((lpar >> i) & 1u) ^ 1u);
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ------------------------------------------------ MMA issue
    if (lane == 0) {
      int st = 0;
      uint32_t fpar = 0u, tpar = 0u;
      bool ok = true, any = false;
      for (int u = blockIdx.x; u < g.units && ok; u += gridDim.x) {
        const int z = u / (g.tiles_m * g.tiles_n);
        const int kb = z * g.kt_per_split, ke = min(g.KT, kb + g.kt_per_split);
        uint32_t started = 0;  // bit grp: accumulator grp written in this accumulation
        for (int kt = kb; kt < ke; ++kt) {
          const bool cstart = ((kt - kb) % OZ_DR) == 0;
          const bool cend = ((kt - kb) % OZ_DR) == OZ_DR - 1 || kt == ke - 1;
          if (!mbar_wait(&full[st], (fpar >> st) & 1u) || s_fail) {
            ok = false;
            break;
          }
          if (cstart) {
            // the accumulators are free once the previous drain has read them
            if (!mbar_wait(&tempty, (tpar & 1u) ^ 1u) || s_fail) {
              ok = false;
              break;
            }
            started = 0;
          }
          tc_fence_after();
          const uint32_t a0 = smem_u32(stage_a(st)), b0 = smem_u32(stage_b(st));
#pragma unroll
          for (int d = OZ_S + 1; d >= 2; --d) {
            const int grp = oz_group(d);
#pragma unroll
            for (int s = 1; s <= OZ_S; ++s) {
              const int t = d - s;
              if (t < 1 || t > OZ_S) continue;
              // slice s (1-based) sits in pair (s-1)/2 at byte offset ((s-1)&1)*64
              const uint32_t ao = (uint32_t)(((s - 1) >> 1) * OZ_PT_A + ((s - 1) & 1) * 64);
              const uint32_t bo = (uint32_t)(((t - 1) >> 1) * OZ_PT_B + ((t - 1) & 1) * 64);
#pragma unroll
              for (int kk = 0; kk < OZ_BK / 16; ++kk) {
                const uint32_t acc = (started >> grp) & 1u;
                mma_bf16(tmem + (uint32_t)(grp * OZ_BN), sw128_desc(a0 + ao + kk * 32),
                         sw128_desc(b0 + bo + kk * 32), OZ_IDESC, acc);
                started |= 1u << grp;
              }
            }
          }
          any = true;
          mma_commit(&empty[st]);
          fpar ^= 1u << st;
          st = (st + 1 == OZ_NST) ? 0 : st + 1;
          if (cend) {
            mma_commit(&tfull);
            tpar ^= 1u;
          }
        }
      }
      if (!ok) s_fail = 1;
      if (any) {
        // every MMA of this thread has completed once this commit arrives
        mma_commit(&done);
        mbar_wait(&done, 0u);
      }
    }
    __syncwarp();
  } else {
    // ------------------------------------------------ drain and epilogue
    const int quad = warp & 3, half = (warp - 2) >> 2;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)(half * OZ_CPT);
    const int64_t MN = g.M * g.N;
    uint32_t tpar = 0u;
    bool ok = true;
    for (int u = blockIdx.x; u < g.units && ok; u += gridDim.x) {
      const int tm = u % g.tiles_m, rest = u / g.tiles_m;
      const int tn = rest % g.tiles_n, z = rest / g.tiles_n;
      const int kb = z * g.kt_per_split, ke = min(g.KT, kb + g.kt_per_split);
      float hi[OZ_CPT], lo[OZ_CPT];
#pragma unroll
      for (int c = 0; c < OZ_CPT; ++c) hi[c] = lo[c] = 0.0f;
      for (int kt = kb; kt < ke; kt += OZ_DR) {
        if (!mbar_wait(&tfull, tpar & 1u) || s_fail) {
          ok = false;
          break;
        }
        tc_fence_after();
        // smallest groups first; each group sum goes into (hi, lo)
#pragma unroll 1
        for (int gp = OZ_NG - 1; gp >= 1; gp -= 2) {
          float v[OZ_CPT], w[OZ_CPT];
          tmem_ld32x2(lane_base + (uint32_t)(gp * OZ_BN), lane_base + (uint32_t)((gp - 1) * OZ_BN),
                      v, w);
#pragma unroll
          for (int e = 0; e < OZ_CPT; ++e) {
            float sm, err, sm2, err2;
            two_sum(hi[e], v[e], sm, err);
            two_sum(sm, w[e], sm2, err2);
            hi[e] = sm2;
            lo[e] += err + err2;
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty);
        tpar ^= 1u;
      }
      if (!ok) break;
      const int64_t r = (int64_t)tm * OZ_BM + 32 * quad + lane;
      const int64_t c0 = (int64_t)tn * OZ_BN + half * OZ_CPT;
      const int nval = (int)imin64(OZ_CPT, g.N - c0);
      if (r < g.M && nval > 0) {
        if (g.part != nullptr) {
          float* ph = g.part + (int64_t)(2 * z) * MN + r + c0 * g.M;
#pragma unroll
          for (int c = 0; c < OZ_CPT; ++c) {
            if (c < nval) {
              ph[0] = hi[c];
              ph[MN] = lo[c];
            }
            ph += g.M;
          }
        } else {
          const int ea = oz_scale_exp(g.expA[r]);
          double* cp = g.C + r + c0 * g.ldc;
          const int64_t ldc = g.ldc;
          const double alpha = g.alpha, beta = g.beta;
          const bool fast = (alpha == 1.0 || alpha == -1.0) && (beta == 0.0 || beta == 1.0);
          const bool use_c = beta != 0.0;
          const uint32_t neg = alpha < 0.0 ? 0x80000000u : 0u;
#pragma unroll
          for (int cb = 0; cb < OZ_CPT; cb += 16) {
            double cv[16];
#pragma unroll
            for (int e = 0; e < 16; ++e)
              cv[e] = (use_c && cb + e < nval) ? __ldcs(cp + (cb + e) * ldc) : 0.0;
#pragma unroll
            for (int e = 0; e < 16; ++e) {
              const int c = cb + e;
              if (c < nval) {
                const int sc = ea + oz_scale_exp(__ldg(g.expB + c0 + c));
                double out;
                if (fast) {
                  out = cv[e] + scaled_f64(hi[c], sc, neg);
                  out = out + scaled_f64(lo[c], sc, neg);
                } else {
                  const double f = alpha * pow2(sc);
                  out = fma(f, (double)hi[c], fma(f, (double)lo[c], use_c ? beta * cv[e] : 0.0));
                }
                __stcs(cp + c * ldc, out);
              }
            }
          }
        }
      }
    }
    if (!ok) s_fail = 1;
  }

  if (tid == 0 && s_fail) atomicOr(g.status, RQRCP_INFO_TIMEOUT);
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, OZ_TCOLS);
  }
}

// C = alpha 2^(e_i + f_j) sum_z (hi_z + lo_z) + beta C, the sum in FP64 in a
// fixed order; splits = 0 gives C = beta C.
__global__ void oz_reduce(const float* __restrict__ part, int splits, int64_t M, int64_t N,
                          const int* __restrict__ expA, const int* __restrict__ expB, double alpha,
                          double beta, double* __restrict__ C, int64_t ldc) {
  const int64_t MN = M * N;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < MN;
       e += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int z = 0; z < splits; ++z)
      s += (double)part[(int64_t)(2 * z) * MN + e] + (double)part[(int64_t)(2 * z + 1) * MN + e];
    const int64_t i = e % M, j = e / M;
    double* cp = C + i + j * ldc;
    const double v =
        splits > 0 ? alpha * s * pow2(oz_scale_exp(expA[i]) + oz_scale_exp(expB[j])) : 0.0;
    *cp = beta != 0.0 ? fma(beta, *cp, v) : v;
  }
}

}  // namespace

int64_t oz_kpad(int64_t K) { return (K + OZ_KP - 1) / OZ_KP * OZ_KP; }

size_t oz_slice_elems(int64_t rows, int64_t K) {
  return (size_t)2 * OZ_PAIRS * rpad128(rows) * oz_kpad(K);
}

cudaError_t launch_oz_slice(const double* X, int64_t ld, bool kc, int amode, int64_t R, int64_t K,
                            __nv_bfloat16* slices, int* exps, cudaStream_t st) {
  if (R <= 0) return cudaSuccess;
  const int64_t Rp = rpad128(R), Kp = oz_kpad(K);
  const int warps = 8;
  const unsigned gx = (unsigned)((Rp + warps - 1) / warps);
  if (!kc) {
    if (amode == 1)
      oz_slice_rows<1><<<gx, 32 * warps, 0, st>>>(X, ld, R, K, Rp, Kp, slices, exps);
    else
      oz_slice_rows<0><<<gx, 32 * warps, 0, st>>>(X, ld, R, K, Rp, Kp, slices, exps);
    return cudaGetLastError();
  }
  cudaError_t e = cudaMemsetAsync(exps, 0, sizeof(int) * (size_t)R, st);
  if (e != cudaSuccess) return e;
  const dim3 g1((unsigned)((R + warps - 1) / warps), (unsigned)((K + OZ_KCH - 1) / OZ_KCH));
  const dim3 g2(gx, (unsigned)((Kp + OZ_KCH - 1) / OZ_KCH));
  if (K > 0) {
    if (amode == 1)
      oz_rowmax_cols<1><<<g1, 32 * warps, 0, st>>>(X, ld, R, K, exps);
    else
      oz_rowmax_cols<0><<<g1, 32 * warps, 0, st>>>(X, ld, R, K, exps);
  }
  if (amode == 1)
    oz_slice_cols<1><<<g2, 32 * warps, 0, st>>>(X, ld, R, K, Rp, Kp, slices, exps);
  else
    oz_slice_cols<0><<<g2, 32 * warps, 0, st>>>(X, ld, R, K, Rp, Kp, slices, exps);
  return cudaGetLastError();
}

int oz_slice_launches(bool kc, int64_t K) { return kc ? (K > 0 ? 2 : 1) : 1; }

int oz_launches(int64_t M, int64_t N, int64_t Kp, int num_sms, size_t partial_cap) {
  if (M <= 0 || N <= 0) return 0;
  const int KT = (int)(Kp / OZ_BK);
  if (KT == 0) return 1;
  const int64_t tiles = (rpad128(M) / OZ_BM) * ((N + OZ_BN - 1) / OZ_BN);
  int splits = 1;
  if (partial_cap > 0 && tiles < num_sms && KT > 1)
    splits = pick_splits(tiles, KT, num_sms,
                         (int)std::min<size_t>(64, partial_cap / (2 * (size_t)M * N)));
  const int per = (KT + splits - 1) / splits;
  splits = (KT + per - 1) / per;
  return splits > 1 ? 2 : 1;
}

cudaError_t launch_oz_gemm(const OzGemmArgs& a, cudaStream_t st) {
  if (a.M <= 0 || a.N <= 0) return cudaSuccess;
  const int nsm = a.num_sms > 0 ? a.num_sms : 1;
  const int KT = (int)(a.Kp / OZ_BK);
  if (KT == 0) {
    int64_t blocks = (a.M * a.N + 255) / 256;
    if (blocks > (int64_t)nsm * 16) blocks = (int64_t)nsm * 16;
    oz_reduce<<<(unsigned)blocks, 256, 0, st>>>(nullptr, 0, a.M, a.N, a.expA, a.expB, a.alpha,
                                                a.beta, a.C, a.ldc);
    return cudaGetLastError();
  }
  // both operands are stored with rows padded to 128 (see launch_oz_slice)
  const int64_t RpA = rpad128(a.M), RpB = rpad128(a.N);
  CUtensorMap ma, mb;
  cudaError_t e = make_map_bf16_3d(&ma, a.As, (uint64_t)(2 * a.Kp), (uint64_t)RpA, OZ_PAIRS,
                                   OZ_BM, OZ_PAIRS);
  if (e != cudaSuccess) return e;
  e = make_map_bf16_3d(&mb, a.Bs, (uint64_t)(2 * a.Kp), (uint64_t)RpB, OZ_PAIRS, OZ_BN, OZ_PAIRS);
  if (e != cudaSuccess) return e;

  OzArgs x{};
  x.M = a.M;
  x.N = a.N;
  x.KT = KT;
  x.tiles_m = (int)(RpA / OZ_BM);
  x.tiles_n = (int)((a.N + OZ_BN - 1) / OZ_BN);
  const int64_t tiles = (int64_t)x.tiles_m * x.tiles_n;
  int splits = 1;
  if (a.partial != nullptr && tiles < nsm && KT > 1)
    splits = pick_splits(tiles, KT, nsm,
                         (int)std::min<size_t>(64, a.partial_cap / (2 * (size_t)a.M * a.N)));
  x.kt_per_split = (KT + splits - 1) / splits;
  splits = (KT + x.kt_per_split - 1) / x.kt_per_split;
  x.units = (int)(tiles * splits);
  x.alpha = a.alpha;
  x.beta = a.beta;
  x.C = a.C;
  x.ldc = a.ldc;
  x.expA = a.expA;
  x.expB = a.expB;
  x.part = splits > 1 ? a.partial : nullptr;
  x.status = a.status;

  const size_t smem = (size_t)OZ_NST * OZ_STAGE + 1024;
  e = cudaFuncSetAttribute(oz_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = (int)std::min<int64_t>(x.units, nsm);
  oz_gemm_kernel<<<grid, OZ_NT, smem, st>>>(ma, mb, x);
  e = cudaGetLastError();
  if (e != cudaSuccess || splits == 1) return e;
  int64_t blocks = (a.M * a.N + 255) / 256;
  if (blocks > (int64_t)nsm * 16) blocks = (int64_t)nsm * 16;
  oz_reduce<<<(unsigned)blocks, 256, 0, st>>>(a.partial, splits, a.M, a.N, a.expA, a.expB, a.alpha,
                                              a.beta, a.C, a.ldc);
  return cudaGetLastError();
}

}  // namespace rq
