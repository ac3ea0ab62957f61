// Split-BF16 GEMM on the 5th-generation tensor cores (tcgen05, sm_103a):
//   C = alpha op(A) op(B) + beta C, FP32 operands and result, column-major.
//
// Splitting (tcx_split_kernel, one memory-bound pass per operand).  Each FP32
// element x becomes S bfloat16 slices
//   x1 = bf16(x), x2 = bf16(x - x1), x3 = bf16(x - x1 - x2)
// (every subtraction is exact in FP32 and x1 + x2 + x3 = x).  The rows of
// op(A) and the columns of op(B) are written k-contiguous, S slices after one
// another, rows padded to 128 and k to 64 with zeros, so that one TMA box is
// one slice tile in the layout the MMA reads.
//
// Products.  S = 3 is the mixed-precision form of the trailing update of
// Alg. 4 (FP32-level accuracy): the six slice products with s + t <= 4.  The
// tensor core rounds its FP32 accumulator toward zero, which over a long k
// loop gives an error that grows with K; so the leading product x1 y1 and the
// five correction products go to two separate tensor-memory accumulators that
// are drained every 32 k (two MMA k-steps) into running sums in registers
// with Kahan compensation (error below 2u of the sum, independent of K).
// S = 1 (the sketch B = Omega A, which only steers pivots) is one product
// accumulated over the whole k range.
//
// Kernel (tcx_gemm_kernel): persistent, one CTA per SM, 128 x 128 output
// tiles, split-K units; 10 warps with fixed roles:
//   warp 0      one thread issues the TMA copies (per 64-k stage one 3-D box
//               per operand: 64 k x 128 rows x S slices, 128-byte swizzle) into
//               a shared-memory ring (2 stages of 96 KB for S = 3, 4 of 32 KB
//               for S = 1; mbarrier expect-tx), refilling a slot as soon as
//               the MMAs that read it have completed;
//   warp 1      allocates tensor memory; one thread issues the tcgen05.mma
//               (M = 128, N = 128, K = 16) and the tcgen05.commit;
//   warps 2-9   drain: warp w reads accumulator lanes 32 (w % 4).. (one row
//               per thread) and columns 64 ((w - 2) / 4).. (64 columns), adds
//               into the compensated sums and, at the end of a unit, writes C
//               (or its split-K partial sums).
// The accumulators are double-buffered in tensor memory (2 x 2 x 128
// columns, all 512), so the drain of one chunk overlaps the MMAs of the next.
// The 128-column tile halves the operand bytes per flop of the earlier
// 128 x 64 tile, whose reads from L2 and HBM bounded it.
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

constexpr int XBM = 128;          // tile rows (A role), UMMA M
constexpr int XBN = 128;          // tile columns (B role), UMMA N
constexpr int XBK = 64;           // k per pipeline stage: one 128-byte swizzle row
constexpr int XNDW = 8;           // drain warps: two per tensor-memory lane quadrant
constexpr int XDC = XBN / 2;      // columns a drain thread owns
constexpr int XNT = 64 + 32 * XNDW;  // warp 0 TMA, warp 1 MMA issue, warps 2.. drain
constexpr int XCH = 2;            // MMA k-steps per drained chunk (S = 3): 32 k
constexpr int XTILE_A = XBM * 128;  // bytes of one A slice tile (128 rows x 64 k)
constexpr int XTILE_B = XBN * 128;  // bytes of one B slice tile (128 rows x 64 k)
// shared-memory ring stages: 2 x 96 KB for S = 3, 4 x 32 KB for S = 1
__host__ __device__ constexpr int xnst(int S) { return S == 3 ? 2 : 4; }
constexpr uint32_t XIDESC = idesc_bf16_f32(XBM, XBN);
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&h);
}

// Split 8 consecutive-k values into S slices; slice s goes to dst[s * sstride].
template <int S>
__device__ __forceinline__ void split8_store(const float* x, __nv_bfloat16* dst, size_t sstride) {
  float rem[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) rem[e] = x[e];
#pragma unroll
  for (int s = 0; s < S; ++s) {
    float h[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      h[e] = __bfloat162float(__float2bfloat16_rn(rem[e]));
      rem[e] = rem[e] - h[e];
    }
    *reinterpret_cast<uint4*>(dst + (size_t)s * sstride) =
        make_uint4(pack_bf16(h[0], h[1]), pack_bf16(h[2], h[3]), pack_bf16(h[4], h[5]),
                   pack_bf16(h[6], h[7]));
  }
}

// ---------------------------------------------------------------- splitting
// Rows r < Rp of op(X), K values each (k-contiguous source: element (r, k) at
// X[row(r) * ld + k], row(r) = rmap ? rmap[r] : r).  Output slice s of row r
// at out[s * Rp * Kp + r * Kp + k]; zeros for r >= R or k >= K.
template <int S>
__global__ void tcx_split_kc(const float* __restrict__ X, int64_t ld, int64_t R, int64_t K,
                             int64_t Rp, int64_t Kp, const int64_t* __restrict__ rmap, bool vec,
                             __nv_bfloat16* __restrict__ out) {
  const int64_t chunks = Kp / 8, items = Rp * chunks;
  const size_t sstride = (size_t)Rp * Kp;
  for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < items;
       it += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = it / chunks, k0 = (it % chunks) * 8;
    float x[8];
    if (r < R && k0 < K) {
      const float* src = X + (rmap ? rmap[r] : r) * ld + k0;
      if (vec && k0 + 8 <= K) {
        const float4 a = __ldg(reinterpret_cast<const float4*>(src));
        const float4 b = __ldg(reinterpret_cast<const float4*>(src) + 1);
        x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
        x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
      } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) x[e] = (k0 + e < K) ? __ldg(src + e) : 0.0f;
      }
    } else {
#pragma unroll
      for (int e = 0; e < 8; ++e) x[e] = 0.0f;
    }
    split8_store<S>(x, out + r * Kp + k0, sstride);
  }
}

// Same output from a row-contiguous source: element (r, k) at X[r + k * ld].
// A 32-row x 64-k tile is transposed through shared memory (256 threads).
template <int S>
__global__ void tcx_split_rc(const float* __restrict__ X, int64_t ld, int64_t R, int64_t K,
                             int64_t Rp, int64_t Kp, __nv_bfloat16* __restrict__ out) {
  __shared__ float tile[64][33];
  const int t = threadIdx.x, tx = t & 31, ty = t >> 5;
  const int64_t r0 = (int64_t)blockIdx.x * 32, k0 = (int64_t)blockIdx.y * 64;
#pragma unroll
  for (int kk = 0; kk < 64; kk += 8) {
    const int64_t r = r0 + tx, k = k0 + kk + ty;
    tile[kk + ty][tx] = (r < R && k < K) ? __ldg(X + r + k * ld) : 0.0f;
  }
  __syncthreads();
  const int row = t >> 3, c = t & 7;
  const int64_t r = r0 + row;
  if (r >= Rp) return;
  float x[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) x[e] = tile[8 * c + e][row];
  split8_store<S>(x, out + r * Kp + k0 + 8 * c, (size_t)Rp * Kp);
}

// ---------------------------------------------------------------- GEMM
struct TcxArgs {
  int64_t M, N;       // rows of the A-role and B-role operands (C is M x N)
  int KT;             // 64-k stages
  int kt_per_split;   // stages per split-K unit
  int tiles_m, tiles_n, units;
  float alpha, beta;
  float* C;
  int64_t ldc;
  float* part;        // splits > 1: hi at part[2z MN + r + c M], lo at part[(2z+1) MN + ...]
  int* status;
};

template <int S>
__global__ void __launch_bounds__(XNT, 1)
    tcx_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                    TcxArgs g) {
  constexpr int NACC = (S == 3) ? 2 : 1;
  constexpr int XNST = xnst(S);
  constexpr uint32_t TCOLS = (uint32_t)(2 * NACC * XBN);  // two buffers of NACC accumulators
  constexpr uint32_t STAGE_A = (uint32_t)S * XTILE_A;
  constexpr uint32_t STAGE_TX = (uint32_t)S * (XTILE_A + XTILE_B);
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full[XNST], empty[XNST], tfull[2], tempty[2], done;
  __shared__ uint32_t s_tmem;
  __shared__ volatile int s_fail;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int i = 0; i < XNST; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&tfull[i], 1);
      mbar_init(&tempty[i], XNDW);
    }
    mbar_init(&done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_fail = 0;
  }
  if (warp == 1) tmem_alloc(&s_tmem, TCOLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;

  auto stage_a = [&](int st) { return smem + (size_t)st * STAGE_TX; };
  auto stage_b = [&](int st) { return smem + (size_t)st * STAGE_TX + STAGE_A; };

  if (warp == 0) {
    // ------------------------------------------------ TMA producer
    // refills each ring slot as soon as the MMAs that read it have completed
    if (lane == 0) {
      int lst = 0;
      uint32_t lpar = 0u, lused = 0u;  // per slot: parity of its uses, used at all
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
          mbar_expect_tx(&full[lst], STAGE_TX);
          tma_load_3d(stage_a(lst), &tmA, kt * XBK, tm * XBM, 0, &full[lst]);
          tma_load_3d(stage_b(lst), &tmB, kt * XBK, tn * XBN, 0, &full[lst]);
          lpar ^= 1u << lst;
          lused |= 1u << lst;
          lst = (lst + 1 == XNST) ? 0 : lst + 1;
        }
      }
      if (!ok) {
        s_fail = 1;
        // wait (bounded) for the last copy issued on each slot
        for (int i = 0; i < XNST; ++i)
          if ((lused >> i) & 1u) mbar_wait(&full[i], ((lpar >> i) & 1u) ^ 1u);
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ------------------------------------------------ MMA issue
    if (lane == 0) {
      bool ok = true;
      int st = 0, buf = 0;
      uint32_t fpar = 0u, tpar = 0u;  // parities of the full[] and tempty[] uses
      bool any = false;
      for (int u = blockIdx.x; u < g.units && ok; u += gridDim.x) {
        const int z = u / (g.tiles_m * g.tiles_n);
        const int kb = z * g.kt_per_split, ke = min(g.KT, kb + g.kt_per_split);
        const int nks = (ke - kb) * (XBK / 16);
        for (int q = 0; q < nks; ++q) {
          const int sq = q & 3;
          if (sq == 0) {
            if (!mbar_wait(&full[st], (fpar >> st) & 1u) || s_fail) {
              ok = false;
              break;
            }
            tc_fence_after();
          }
          const bool cstart = (S == 3) ? (q % XCH == 0) : (q == 0);
          const bool cend = (S == 3) ? (q % XCH == XCH - 1) : (q == nks - 1);
          if (cstart) {
            if (!mbar_wait(&tempty[buf], ((tpar >> buf) & 1u) ^ 1u) || s_fail) {
              ok = false;
              break;
            }
            tc_fence_after();
          }
          const uint32_t acc = cstart ? 0u : 1u;
          const uint32_t a0 = smem_u32(stage_a(st)) + (uint32_t)sq * 32u;
          const uint32_t b0 = smem_u32(stage_b(st)) + (uint32_t)sq * 32u;
          const uint32_t d_big = tmem + (uint32_t)(buf * NACC * XBN);
          mma_bf16(d_big, sw128_desc(a0), sw128_desc(b0), XIDESC, acc);  // x1 y1
          if (S == 3) {
            const uint32_t d_small = d_big + XBN;
            // correction products (s, t) with 2 < s + t <= 4
            mma_bf16(d_small, sw128_desc(a0 + 2 * XTILE_A), sw128_desc(b0), XIDESC, acc);        // x3 y1
            mma_bf16(d_small, sw128_desc(a0 + XTILE_A), sw128_desc(b0 + XTILE_B), XIDESC, 1u);   // x2 y2
            mma_bf16(d_small, sw128_desc(a0), sw128_desc(b0 + 2 * XTILE_B), XIDESC, 1u);         // x1 y3
            mma_bf16(d_small, sw128_desc(a0 + XTILE_A), sw128_desc(b0), XIDESC, 1u);             // x2 y1
            mma_bf16(d_small, sw128_desc(a0), sw128_desc(b0 + XTILE_B), XIDESC, 1u);             // x1 y2
          }
          any = true;
          if (cend) {
            mma_commit(&tfull[buf]);
            tpar ^= 1u << buf;
            buf ^= 1;
          }
          if (sq == 3) {
            mma_commit(&empty[st]);
            fpar ^= 1u << st;
            st = (st + 1 == XNST) ? 0 : st + 1;
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
    // warp w reads tensor-memory lanes 32 (w % 4).. (its quadrant); the two
    // warps of a quadrant take columns 0..63 and 64..127 of the tile
    const int quad = warp & 3;
    const int half = (warp - 2) / 4;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)(XDC * half);
    const int64_t MN = g.M * g.N;
    int buf = 0;
    uint32_t tpar = 0u;  // parity of the tfull[] uses
    bool ok = true;
    for (int u = blockIdx.x; u < g.units && ok; u += gridDim.x) {
      const int tm = u % g.tiles_m, rest = u / g.tiles_m;
      const int tn = rest % g.tiles_n, z = rest / g.tiles_n;
      const int kb = z * g.kt_per_split, ke = min(g.KT, kb + g.kt_per_split);
      const int nch = (S == 3) ? (ke - kb) * (XBK / 16) / XCH : (ke > kb ? 1 : 0);
      // compensated sums: value = hi - cc.  The compensation cc is below half
      // an ulp of hi, so it is kept as bfloat16 (8 bits of it are plenty: the
      // error of the stored compensation is below 2^-10 ulp of the sum per
      // chunk), two per register, which keeps the drain thread's state within
      // the register budget of a 320-thread CTA.
      float hi[XDC];
      __nv_bfloat162 ccp[XDC / 2];
#pragma unroll
      for (int c = 0; c < XDC; ++c) hi[c] = 0.0f;
#pragma unroll
      for (int c = 0; c < XDC / 2; ++c) ccp[c] = __floats2bfloat162_rn(0.0f, 0.0f);
      for (int ch = 0; ch < nch; ++ch) {
        if (!mbar_wait(&tfull[buf], (tpar >> buf) & 1u) || s_fail) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t tb = lane_base + (uint32_t)(buf * NACC * XBN);
        if (S == 3) {
#pragma unroll
          for (int c0 = 0; c0 < XDC; c0 += 16) {
            float v[16], w[16];
            tmem_ld16x2(tb + c0, tb + XBN + c0, v, w);
#pragma unroll
            for (int e = 0; e < 16; e += 2) {
              // Kahan steps with the chunk's leading and correction parts
              const float2 cf = __bfloat1622float2(ccp[(c0 + e) / 2]);
              const float y0 = (v[e] - cf.x) + w[e];
              const float t0 = hi[c0 + e] + y0;
              const float n0 = (t0 - hi[c0 + e]) - y0;
              hi[c0 + e] = t0;
              const float y1 = (v[e + 1] - cf.y) + w[e + 1];
              const float t1 = hi[c0 + e + 1] + y1;
              const float n1 = (t1 - hi[c0 + e + 1]) - y1;
              hi[c0 + e + 1] = t1;
              ccp[(c0 + e) / 2] = __floats2bfloat162_rn(n0, n1);
            }
          }
        } else {
#pragma unroll
          for (int c0 = 0; c0 < XDC; c0 += 16) {
            float v[16];
            tmem_ld16(tb + c0, v);
#pragma unroll
            for (int e = 0; e < 16; ++e) hi[c0 + e] = v[e];
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[buf]);
        tpar ^= 1u << buf;
        buf ^= 1;
      }
      if (!ok) break;
      const int64_t r = (int64_t)tm * XBM + 32 * quad + lane;
      const int64_t c0 = (int64_t)tn * XBN + XDC * half;
      const int nval = (int)imax64(0, imin64(XDC, g.N - c0));
      if (r < g.M) {
        if (g.part != nullptr) {
          float* ph = g.part + (int64_t)(2 * z) * MN + r + c0 * g.M;
#pragma unroll
          for (int c = 0; c < XDC; ++c) {
            if (c < nval) {
              const float2 cf = __bfloat1622float2(ccp[c / 2]);
              ph[0] = hi[c];
              ph[MN] = -((c & 1) ? cf.y : cf.x);
            }
            ph += g.M;
          }
        } else {
          // C read in batches of 16 independent loads, then written
          float* cp = g.C + r + c0 * g.ldc;
          const int64_t ldc = g.ldc;
          const float alpha = g.alpha, beta = g.beta;
#pragma unroll
          for (int cb = 0; cb < XDC; cb += 16) {
            float cv[16];
#pragma unroll
            for (int e = 0; e < 16; ++e)
              cv[e] = (beta != 0.0f && cb + e < nval) ? __ldcs(cp + (cb + e) * ldc) : 0.0f;
#pragma unroll
            for (int e = 0; e < 16; ++e) {
              const int c = cb + e;
              if (c < nval) {
                const float out = fmaf(alpha, hi[c], beta * cv[e]);
                const float2 cf = __bfloat1622float2(ccp[c / 2]);
                __stcs(cp + c * ldc, fmaf(-alpha, (c & 1) ? cf.y : cf.x, out));
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
    tmem_dealloc(tmem, TCOLS);
  }
}

// C = alpha * sum_z (hi_z + lo_z) + beta C, the sum in FP64 in a fixed order;
// splits = 0 gives C = beta C.
__global__ void tcx_reduce(const float* __restrict__ part, int splits, int64_t M, int64_t N,
                           float alpha, float beta, float* __restrict__ C, int64_t ldc) {
  const int64_t MN = M * N;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < MN;
       e += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int z = 0; z < splits; ++z)
      s += (double)part[(int64_t)(2 * z) * MN + e] + (double)part[(int64_t)(2 * z + 1) * MN + e];
    const int64_t i = e % M, j = e / M;
    float* cp = C + i + j * ldc;
    const float v = alpha * (float)s;
    *cp = beta != 0.0f ? fmaf(beta, *cp, v) : v;
  }
}

// ---------------------------------------------------------------- host side
int64_t rpad(int64_t R, int tile) { return (R + tile - 1) / tile * tile; }

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
int64_t kpad(int64_t K) { return (K + XBK - 1) / XBK * XBK; }

// 3-D map over S slices of Rp rows x Kp k: box = 64 k x `rows` rows x S slices.
cudaError_t make_map(CUtensorMap* map, const __nv_bfloat16* base, int64_t Rp, int64_t Kp, int S,
                     int rows) {
  return make_map_bf16_3d(map, base, (uint64_t)Kp, (uint64_t)Rp, (uint64_t)S, rows, S);
}

template <int S>
cudaError_t split_operand(const float* X, int64_t ld, bool kc, int64_t R, int64_t K, int64_t Rp,
                          int64_t Kp, const int64_t* rmap, __nv_bfloat16* out, int num_sms,
                          cudaStream_t st) {
  if (kc) {
    const bool vec = (ld % 4 == 0) && ((reinterpret_cast<uintptr_t>(X) & 15) == 0);
    const int64_t items = Rp * (Kp / 8);
    int64_t blocks = (items + 255) / 256;
    if (blocks > (int64_t)num_sms * 16) blocks = (int64_t)num_sms * 16;
    tcx_split_kc<S><<<(unsigned)blocks, 256, 0, st>>>(X, ld, R, K, Rp, Kp, rmap, vec, out);
  } else {
    dim3 grid((unsigned)(Rp / 32), (unsigned)(Kp / 64));
    tcx_split_rc<S><<<grid, 256, 0, st>>>(X, ld, R, K, Rp, Kp, out);
  }
  return cudaGetLastError();
}

template <int S>
size_t gemm_smem() {
  return (size_t)xnst(S) * S * (XTILE_A + XTILE_B) + 1024;
}

template <int S>
cudaError_t run(TcGemmArgs g, cudaStream_t st) {
  const int64_t Rm = rpad(g.M, XBM), Rn = rpad(g.N, XBN), Kp = kpad(g.K);
  const int KT = (int)(Kp / XBK);
  const int nsm = g.num_sms > 0 ? g.num_sms : 1;
  if (KT == 0) {
    // C = beta C
    int64_t blocks = (g.M * g.N + 255) / 256;
    if (blocks > (int64_t)nsm * 16) blocks = (int64_t)nsm * 16;
    tcx_reduce<<<(unsigned)blocks, 256, 0, st>>>(nullptr, 0, g.M, g.N, g.alpha, g.beta, g.C, g.ldc);
    return cudaGetLastError();
  }
  if ((size_t)S * Rm * Kp > g.slcapA || (size_t)S * Rn * Kp > g.slcapB || g.slA == nullptr ||
      g.slB == nullptr)
    return cudaErrorInvalidValue;
  // rows of op(A): stored columns when transposed (k-contiguous); columns of
  // op(B): stored columns when not transposed (k-contiguous)
  cudaError_t e = split_operand<S>(g.A, g.lda, g.transA == 'T', g.M, g.K, Rm, Kp, nullptr, g.slA,
                                   nsm, st);
  if (e != cudaSuccess) return e;
  e = split_operand<S>(g.B, g.ldb, g.transB == 'N', g.N, g.K, Rn, Kp,
                       g.transB == 'N' ? g.bcols : nullptr, g.slB, nsm, st);
  if (e != cudaSuccess) return e;
  CUtensorMap ma, mb;
  if ((e = make_map(&ma, g.slA, Rm, Kp, S, XBM)) != cudaSuccess) return e;
  if ((e = make_map(&mb, g.slB, Rn, Kp, S, XBN)) != cudaSuccess) return e;

  TcxArgs x{};
  x.M = g.M;
  x.N = g.N;
  x.KT = KT;
  x.tiles_m = (int)(Rm / XBM);
  x.tiles_n = (int)(Rn / XBN);
  const int64_t tiles = (int64_t)x.tiles_m * x.tiles_n;
  int splits = 1;
  if (g.partial != nullptr && tiles < nsm && KT > 1)
    splits = pick_splits(tiles, KT, nsm,
                         (int)std::min<size_t>(64, g.partial_cap / (2 * (size_t)g.M * g.N)));
  x.kt_per_split = (KT + splits - 1) / splits;
  splits = (KT + x.kt_per_split - 1) / x.kt_per_split;
  x.units = (int)(tiles * splits);
  x.alpha = g.alpha;
  x.beta = g.beta;
  x.C = g.C;
  x.ldc = g.ldc;
  x.part = splits > 1 ? g.partial : nullptr;
  x.status = g.status;

  auto kern = tcx_gemm_kernel<S>;
  const size_t smem = gemm_smem<S>();
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = (int)std::min<int64_t>(x.units, nsm);
  kern<<<grid, XNT, smem, st>>>(ma, mb, x);
  e = cudaGetLastError();
  if (e != cudaSuccess || splits == 1) return e;
  int64_t blocks = (g.M * g.N + 255) / 256;
  if (blocks > (int64_t)nsm * 16) blocks = (int64_t)nsm * 16;
  tcx_reduce<<<(unsigned)blocks, 256, 0, st>>>(g.partial, splits, g.M, g.N, g.alpha, g.beta, g.C,
                                               g.ldc);
  return cudaGetLastError();
}

}  // namespace

size_t tc_slice_elems(int64_t rows, int64_t K, int slices) {
  return (size_t)slices * rpad(rows, XBM) * kpad(K);
}

int tc_launches(int64_t M, int64_t N, int64_t K, int num_sms, size_t partial_cap) {
  if (M <= 0 || N <= 0) return 0;
  if (K <= 0) return 1;
  const int64_t tiles = (rpad(M, XBM) / XBM) * (rpad(N, XBN) / XBN);
  const int KT = (int)(kpad(K) / XBK);
  int splits = 1;
  if (partial_cap > 0 && tiles < num_sms && KT > 1)
    splits = pick_splits(tiles, KT, num_sms,
                         (int)std::min<size_t>(64, partial_cap / (2 * (size_t)M * N)));
  const int per = (KT + splits - 1) / splits;
  splits = (KT + per - 1) / per;
  return splits > 1 ? 4 : 3;
}

cudaError_t launch_tc_gemm(TcGemmArgs g, int slices, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0) return cudaSuccess;
  if (slices == 1) return run<1>(g, st);
  if (slices == 3) return run<3>(g, st);
  return cudaErrorInvalidValue;
}

}  // namespace rq
