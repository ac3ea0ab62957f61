// FP64-accurate GEMM on the BF16 tensor cores (tcgen05, sm_103a) by exact
// operand slicing -- the FP64 form of the trailing update of Alg. 4
// (W = T^T Y^T A2, A2 -= Y W) when the GPU's FP64 pipe (~1.25 TFLOP/s on a
// GB300) is the bottleneck.
//
// Slicing (one pass per operand, oz_slice_kernel).  Row r of an operand
// (K values x_k) gets the power-of-two scale 2^e_r with max_k |x_k| < 2^e_r;
// t = x 2^-e_r lies in (-1, 1) and is cut into S = 7 slices of 8 bits,
//   t = sum_s y_s 2^{-8s} + (|rest| < 2^-56),  y_s integer in [-255, 255],
// each slice value y_s 2^{-8s} exactly representable in BF16.
//
// Products.  C_ij = 2^{e_i + f_j} sum_{s,t} sum_k a_s(i,k) b_t(k,j).  The pairs
// with s + t = d carry the common grid 2^{-8d}; with K <= 32 per accumulation
// their sum is an integer multiple of that grid below (d-1) 32 255^2 < 2^24
// units for d <= 6, hence EXACT in an FP32 accumulator whatever the tensor
// core's rounding (it truncates).  d = 2..6 get one accumulator each; d = 7, 8
// share one (at most 2^-40 of the leading term, so even a truncating FP32 sum
// of its 416 products errs below 2^-54); pairs with s + t > 8 are dropped
// (below 2^-56).  28 BF16 MMAs per k-step.
//
// Kernel (oz_gemm_kernel): one 128 x 64 output tile per CTA, 256 threads.
// Per 64-wide k-stage the slices are copied (16-byte chunks) into the
// 128-byte-swizzled K-major layout; for each 32-wide half of the stage,
// thread 0 issues the 28 x 2 tcgen05.mma into the six tensor-memory
// accumulators (6 x 64 columns), commits to an mbarrier, and the eight warps
// (two per accumulator lane quadrant, one per 32-column half) drain the
// accumulators into running double-FP32 sums (error-free TwoSum), so the
// exactness bound never needs K > 32.  The epilogue forms
// 2^{e_i + f_j} (hi + lo) in FP64 and writes C = alpha * that + beta * C.
#include <cuda_bf16.h>

#include "kernels.cuh"

namespace rq {
namespace {

constexpr int OZ_S = 7;        // slices per operand
constexpr int OZ_BITS = 8;     // bits per slice
constexpr int OZ_NG = 6;       // accumulators: d = 2, 3, 4, 5, 6 and d >= 7
constexpr int OZ_KH = 32;      // k per exact accumulation (one drain)
constexpr int OZ_BM = 128;
constexpr int OZ_BN = 64;
constexpr int OZ_BK = 64;
constexpr int OZ_NT = 256;  // warp w: accumulator lanes 32 (w % 4).., columns 32 (w / 4)..
constexpr unsigned kOzPolls = 1u << 26;

__device__ __forceinline__ uint32_t su32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// ---------------------------------------------------------------- slicing
// Rows of op(X): KC -> element (r, k) at X[r * ld + k] (a stored column per
// row); otherwise at X[r + k * ld].  amode 1: X is a unit-lower reflector
// block stored in place (above the diagonal 0, diagonal 1; the diagonal is
// the stored (row, col) with row == col).  Output: slices s = 0..6 at
// out + s * R * Kp, row r at [r * Kp, r * Kp + Kp), K padded with zeros;
// exps[r] = e_r.
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
// m, T = |t| 2^56 = m 2^(E - 1075 + 56 - e) < 2^56, and slice s is the byte
// (T >> (56 - 8s)) & 255 with the sign of x.
template <bool KC, int AMODE>
__global__ void oz_slice_kernel(const double* __restrict__ X, int64_t ld, int64_t R, int64_t K,
                                int64_t Kp, __nv_bfloat16* __restrict__ out, int* __restrict__ exps) {
  // one warp per row
  const int lane = threadIdx.x & 31;
  const int64_t r = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  if (r >= R) return;
  unsigned long long mb = 0;  // max |x| as bits (monotone for non-negative doubles)
  for (int64_t k = lane; k < K; k += 32) {
    const unsigned long long b =
        (unsigned long long)__double_as_longlong(oz_elem<KC, AMODE>(X, ld, r, k)) & 0x7FFFFFFFFFFFFFFFull;
    mb = b > mb ? b : mb;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long other = __shfl_xor_sync(0xffffffffu, mb, o);
    mb = other > mb ? other : mb;
  }
  // e with max|x| < 2^e: biased exponent - 1022 (subnormals: -1022)
  const int e = (mb == 0) ? 0 : (int)((mb >> 52) & 0x7FF) - 1022;
  if (lane == 0) exps[r] = e;
  for (int64_t k = lane; k < Kp; k += 32) {
    unsigned long long T = 0;
    bool neg = false;
    if (k < K) {
      const unsigned long long b = (unsigned long long)__double_as_longlong(oz_elem<KC, AMODE>(X, ld, r, k));
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
#pragma unroll
    for (int s = 0; s < OZ_S; ++s) {
      const float y = (float)(unsigned)((T >> (8 * (OZ_S - 1 - s))) & 0xFFull);
      const float v = ldexpf(neg ? -y : y, -OZ_BITS * (s + 1));  // exact
      out[(int64_t)s * R * Kp + r * Kp + k] = __float2bfloat16_rn(v);
    }
  }
}

// ---------------------------------------------------------------- tcgen05
__device__ __forceinline__ void oz_mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(bar)) : "memory");
}

__device__ __forceinline__ bool oz_mbar_wait(uint64_t* bar, uint32_t parity) {
  for (unsigned i = 0; i < kOzPolls; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(su32(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
    if (i > 32) __nanosleep(32);
  }
  return false;
}

__device__ __forceinline__ uint64_t oz_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// kind::f16, FP32 accumulate, BF16 A and B, K-major, M = 128, N = 64
constexpr uint32_t OZ_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(OZ_BN >> 3) << 17) |
                              ((uint32_t)(OZ_BM >> 4) << 24);

__device__ __forceinline__ void oz_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(OZ_IDESC), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void oz_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// error-free transformation: s + err = a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& err) {
  s = a + b;
  const float bb = s - a;
  err = (a - (s - bb)) + (b - bb);
}

// group of the diagonal d = s + t (s, t >= 1)
__host__ __device__ constexpr int oz_group(int d) { return d - 2 < OZ_NG - 1 ? d - 2 : OZ_NG - 1; }

__global__ void __launch_bounds__(OZ_NT, 1) oz_gemm_kernel(OzGemmArgs g) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  constexpr size_t A_SL = (size_t)OZ_BM * 128;  // one slice tile, 64 k x 2 bytes per row
  constexpr size_t B_SL = (size_t)OZ_BN * 128;
  unsigned char* As = smem;
  unsigned char* Bs = smem + OZ_S * A_SL;
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t i0 = (int64_t)blockIdx.x * OZ_BM, j0 = (int64_t)blockIdx.y * OZ_BN;
  const int KT = (int)(g.Kp / OZ_BK);

  if (tid == 0) {
    oz_mbar_init(&mbar);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_fail = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(&s_tmem)),
                 "r"(512u)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;

  // running double-FP32 sums for this thread's row, 32 columns
  constexpr int CPT = OZ_BN / 2;
  const int quad = warp & 3, cbase = (warp >> 2) * CPT;
  float hi[CPT], lo[CPT];
#pragma unroll
  for (int c = 0; c < CPT; ++c) hi[c] = lo[c] = 0.0f;

  for (int kt = 0; kt < KT; ++kt) {
    // ---- copy the stage's slices into swizzled shared memory
    const int64_t k0 = (int64_t)kt * OZ_BK;
    for (int item = tid; item < OZ_S * OZ_BM * 8; item += OZ_NT) {
      const int s = item / (OZ_BM * 8), rem = item % (OZ_BM * 8), r = rem >> 3, c = rem & 7;
      const int64_t gr = i0 + r;
      uint4 v = make_uint4(0, 0, 0, 0);
      if (gr < g.M)
        v = *reinterpret_cast<const uint4*>(g.As + (int64_t)s * g.M * g.Kp + gr * g.Kp + k0 + 8 * c);
      *reinterpret_cast<uint4*>(As + s * A_SL + r * 128 + ((c ^ (r & 7)) << 4)) = v;
    }
    for (int item = tid; item < OZ_S * OZ_BN * 8; item += OZ_NT) {
      const int s = item / (OZ_BN * 8), rem = item % (OZ_BN * 8), r = rem >> 3, c = rem & 7;
      const int64_t gr = j0 + r;
      uint4 v = make_uint4(0, 0, 0, 0);
      if (gr < g.N)
        v = *reinterpret_cast<const uint4*>(g.Bs + (int64_t)s * g.N * g.Kp + gr * g.Kp + k0 + 8 * c);
      *reinterpret_cast<uint4*>(Bs + s * B_SL + r * 128 + ((c ^ (r & 7)) << 4)) = v;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    for (int half = 0; half < OZ_BK / OZ_KH; ++half) {
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t a0 = su32(As), b0 = su32(Bs);
        uint32_t started = 0;  // bit g: accumulator g written in this half
#pragma unroll
        for (int d = OZ_S + 1; d >= 2; --d) {
          const int grp = oz_group(d);
#pragma unroll
          for (int s = 1; s <= OZ_S; ++s) {
            const int t = d - s;
            if (t < 1 || t > OZ_S) continue;
#pragma unroll
            for (int kq = 0; kq < OZ_KH / 16; ++kq) {
              const int kk = half * (OZ_KH / 16) + kq;
              const uint32_t acc = (started >> grp) & 1u;
              oz_mma(tmem + (uint32_t)(grp * OZ_BN),
                     oz_desc(a0 + (uint32_t)((s - 1) * A_SL) + kk * 32),
                     oz_desc(b0 + (uint32_t)((t - 1) * B_SL) + kk * 32), acc);
              started |= 1u << grp;
            }
          }
        }
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                su32(&mbar))
            : "memory");
        if (!oz_mbar_wait(&mbar, (uint32_t)((kt * (OZ_BK / OZ_KH) + half) & 1))) s_fail = 1;
      }
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (s_fail) break;
      // ---- drain: add the exact group sums (smallest first) into the
      // running double-FP32 sums of row 32 quad + lane, columns cbase..
      const uint32_t lane_base = tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)cbase;
#pragma unroll
      for (int c0 = 0; c0 < CPT; c0 += 16) {
        float v[16], part_hi[16], part_lo[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) part_hi[e] = part_lo[e] = 0.0f;
#pragma unroll
        for (int grp = OZ_NG - 1; grp >= 0; --grp) {
          oz_ld16(lane_base + (uint32_t)(grp * OZ_BN + c0), v);
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            float sm, err;
            two_sum(part_hi[e], v[e], sm, err);
            part_hi[e] = sm;
            part_lo[e] += err;
          }
        }
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          float sm, err;
          two_sum(hi[c0 + e], part_hi[e], sm, err);
          hi[c0 + e] = sm;
          lo[c0 + e] += err + part_lo[e];
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();  // accumulators read before the next MMAs overwrite them
    }
    if (s_fail) break;
  }

  if (s_fail) {
    if (tid == 0) atomicOr(g.status, RQRCP_INFO_TIMEOUT);
  } else {
    const int64_t i = i0 + 32 * quad + lane;
    if (i < g.M) {
      const int ei = g.expA[i];
#pragma unroll
      for (int c = 0; c < CPT; ++c) {
        const int64_t j = j0 + cbase + c;
        if (j < g.N) {
          const int sc = ei + g.expB[j];
          const double x = ldexp((double)hi[c] + (double)lo[c], sc);
          double* cp = g.C + i + j * g.ldc;
          *cp = (g.beta != 0.0) ? fma(g.alpha, x, g.beta * *cp) : g.alpha * x;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u)
                 : "memory");
}

}  // namespace

size_t oz_slice_bytes(int64_t rows, int64_t K) {
  const int64_t Kp = (K + OZ_BK - 1) / OZ_BK * OZ_BK;
  return (size_t)OZ_S * rows * Kp * 2 + (size_t)rows * 4 + 512;
}

int64_t oz_kpad(int64_t K) { return (K + OZ_BK - 1) / OZ_BK * OZ_BK; }

cudaError_t launch_oz_slice(const double* X, int64_t ld, bool kc, int amode, int64_t R, int64_t K,
                            __nv_bfloat16* slices, int* exps, cudaStream_t st) {
  if (R <= 0) return cudaSuccess;
  const int64_t Kp = oz_kpad(K);
  const int warps = 8;
  const unsigned grid = (unsigned)((R + warps - 1) / warps);
  if (kc && amode == 1) oz_slice_kernel<true, 1><<<grid, 32 * warps, 0, st>>>(X, ld, R, K, Kp, slices, exps);
  else if (kc) oz_slice_kernel<true, 0><<<grid, 32 * warps, 0, st>>>(X, ld, R, K, Kp, slices, exps);
  else if (amode == 1) oz_slice_kernel<false, 1><<<grid, 32 * warps, 0, st>>>(X, ld, R, K, Kp, slices, exps);
  else oz_slice_kernel<false, 0><<<grid, 32 * warps, 0, st>>>(X, ld, R, K, Kp, slices, exps);
  return cudaGetLastError();
}

cudaError_t launch_oz_gemm(const OzGemmArgs& g, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0) return cudaSuccess;
  const size_t smem = (size_t)OZ_S * ((size_t)OZ_BM + OZ_BN) * 128 + 1024;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(oz_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  dim3 grid((unsigned)((g.M + OZ_BM - 1) / OZ_BM), (unsigned)((g.N + OZ_BN - 1) / OZ_BN));
  oz_gemm_kernel<<<grid, OZ_NT, smem, st>>>(g);
  return cudaGetLastError();
}

}  // namespace rq
