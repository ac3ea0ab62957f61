// Split-BF16 GEMM on the 5th-generation tensor cores (tcgen05, sm_103a):
//   C = alpha op(A) op(B) + beta C, FP32 operands and result, column-major.
//
// Each FP32 operand element x is split into S bfloat16 slices
//   x1 = bf16(x), x2 = bf16(x - x1), x3 = bf16(x - x1 - x2)
// (every subtraction is exact in FP32), and the product is the sum of the
// slice products x_s y_t with s + t <= S + 1 -- for S = 3 the six products
// 11, 12, 21, 13, 31, 22 -- accumulated in FP32 in tensor memory.  S = 3
// gives FP32-level accuracy (the mixed-precision form of the trailing-matrix
// update of Alg. 4); S = 1 is a plain BF16 product with FP32
// accumulation (the mixed-precision sketch B = Omega A).
//
// Kernel structure (one 128 x BN output tile per CTA, 128 threads):
//   * all four warps load a 128 x 64 (A) and BN x 64 (B) k-slice of the FP32
//     operands from global memory, split it and store the bf16 slices in the
//     128-byte-swizzled K-major layout the MMA reads (row r at r*128 bytes,
//     16-byte chunk c at position c ^ (r mod 8));
//   * thread 0 issues the tcgen05.mma instructions (M = 128, N = BN, K = 16)
//     for every slice product and k-step, then tcgen05.commit arrives on the
//     stage's mbarrier; two stages let the loads of k-slice t+1 overlap the
//     MMAs of k-slice t;
//   * the accumulator lives in tensor memory (BN columns x 128 lanes); warp w
//     reads lanes 32w..32w+31 with tcgen05.ld and writes C.
// Every mbarrier wait is bounded; on timeout the status word gets
// RQRCP_INFO_TIMEOUT and the kernel frees its tensor memory and returns.
#include <cuda_bf16.h>

#include "kernels.cuh"

namespace rq {
namespace {

constexpr int TBM = 128;   // UMMA M
constexpr int TBK = 64;    // k per stage: one 128-byte swizzle row of bf16
constexpr int TNT = 128;   // threads
constexpr unsigned kWaitPolls = 1u << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait; false when it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (unsigned i = 0; i < kWaitPolls; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if (i > 32) __nanosleep(32);
  }
  return false;
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);       // start address
  d |= (uint64_t)1 << 16;                          // leading byte offset (unused)
  d |= (uint64_t)(1024 >> 4) << 32;                // stride byte offset
  d |= (uint64_t)1 << 46;                          // version
  d |= (uint64_t)2 << 61;                          // 128-byte swizzle
  return d;
}

// Instruction descriptor, kind::f16: FP32 accumulate, BF16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&h);
}

// Split 8 consecutive-k values into S slices and store each as one 16-byte
// chunk of row r of the slice tiles (swizzled position).
template <int S>
__device__ __forceinline__ void split_store(const float* x, unsigned char* tile0, size_t slice_bytes,
                                            int r, int c) {
  float rem[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) rem[e] = x[e];
  const uint32_t off = (uint32_t)r * 128u + ((uint32_t)(c ^ (r & 7)) << 4);
#pragma unroll
  for (int s = 0; s < S; ++s) {
    float hi[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      hi[e] = __bfloat162float(__float2bfloat16_rn(rem[e]));
      rem[e] = rem[e] - hi[e];
    }
    uint4 q = make_uint4(pack_bf16(hi[0], hi[1]), pack_bf16(hi[2], hi[3]), pack_bf16(hi[4], hi[5]),
                         pack_bf16(hi[6], hi[7]));
    *reinterpret_cast<uint4*>(tile0 + (size_t)s * slice_bytes + off) = q;
  }
}

// Load the rows x 64 k-slice of an operand into S swizzled slice tiles.
// KC: element (row, k) at base[row * ld + k] (contiguous along k);
// otherwise at base[row + k * ld] (contiguous along rows).
// rmap (KC only, may be null): tile row r reads stored row rmap[row0 + r].
template <int S, bool KC>
__device__ __forceinline__ void load_tile(const float* __restrict__ base, int64_t ld, int64_t row0,
                                          int64_t nrows_total, int64_t k0, int64_t K, int rows,
                                          bool vec, unsigned char* tile0, size_t slice_bytes,
                                          const int64_t* __restrict__ rmap) {
  const int tid = threadIdx.x;
  if (KC) {
    for (int item = tid; item < rows * 8; item += TNT) {
      const int r = item >> 3, c = item & 7;
      const int64_t gr = row0 + r, gk = k0 + 8 * c;
      float x[8];
      const int64_t sr = (gr < nrows_total && rmap != nullptr) ? rmap[gr] : gr;
      if (gr < nrows_total && vec && gk + 8 <= K) {
        const float4* p = reinterpret_cast<const float4*>(base + sr * ld + gk);
        float4 a = __ldg(p), b = __ldg(p + 1);
        x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
        x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
      } else {
#pragma unroll
        for (int e = 0; e < 8; ++e)
          x[e] = (gr < nrows_total && gk + e < K) ? __ldg(base + sr * ld + gk + e) : 0.0f;
      }
      split_store<S>(x, tile0, slice_bytes, r, c);
    }
  } else {
    for (int item = tid; item < rows * 8; item += TNT) {
      const int r = item % rows, c = item / rows;
      const int64_t gr = row0 + r, gk = k0 + 8 * c;
      float x[8];
#pragma unroll
      for (int e = 0; e < 8; ++e)
        x[e] = (gr < nrows_total && gk + e < K) ? __ldg(base + gr + (gk + e) * ld) : 0.0f;
      split_store<S>(x, tile0, slice_bytes, r, c);
    }
  }
}

template <int S, int BN, char TA, char TB>
__global__ void __launch_bounds__(TNT, 1) tc_gemm_kernel(TcGemmArgs g) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte aligned stage buffers
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  constexpr size_t A_SLICE = (size_t)TBM * 128;
  constexpr size_t B_SLICE = (size_t)BN * 128;
  constexpr size_t STAGE = S * (A_SLICE + B_SLICE);
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t i0 = (int64_t)blockIdx.x * TBM;
  const int64_t j0 = (int64_t)blockIdx.y * BN;
  // split-K: this CTA covers k-slices [kt_beg, kt_end)
  const int KT_all = (int)((g.K + TBK - 1) / TBK);
  const int kt_beg = (int)blockIdx.z * g.kt_per_split;
  const int kt_end = min(KT_all, kt_beg + g.kt_per_split);
  const int KT = max(0, kt_end - kt_beg);

  if (tid == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_fail = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&s_tmem)),
                 "r"((uint32_t)BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  constexpr uint32_t IDESC = idesc_bf16(TBM, BN);

  int issued = 0;  // k-slices whose MMAs were committed (same count in every thread)
  for (int kt = 0; kt < KT; ++kt) {
    const int st = kt & 1;
    unsigned char* a_tile = smem + (size_t)st * STAGE;
    unsigned char* b_tile = a_tile + S * A_SLICE;
    if (kt >= 2) {
      // the MMAs of k-slice kt-2 (commit number (kt-2)/2 on this stage) read this buffer
      if (tid == 0 && !mbar_wait(&mbar[st], (uint32_t)(((kt - 2) >> 1) & 1))) s_fail = 1;
      __syncthreads();
      if (s_fail) break;
    }
    const int64_t k0 = (int64_t)(kt_beg + kt) * TBK;
    // op(A)(i, k): 'N' -> A[i + k lda] (contiguous along rows), 'T' -> A[k + i lda]
    load_tile<S, TA == 'T'>(g.A, g.lda, i0, g.M, k0, g.K, TBM, g.vecA, a_tile, A_SLICE, nullptr);
    // op(B)(k, j): 'N' -> B[k + j ldb] (contiguous along k), 'T' -> B[j + k ldb]
    load_tile<S, TB == 'N'>(g.B, g.ldb, j0, g.N, k0, g.K, BN, g.vecB, b_tile, B_SLICE,
                            TB == 'N' ? g.bcols : nullptr);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t a0 = smem_u32(a_tile), b0 = smem_u32(b_tile);
      // slice products with s + t <= S + 1, smallest terms first
      uint32_t acc = kt > 0 ? 1u : 0u;
#pragma unroll
      for (int d = S + 1; d >= 2; --d) {
#pragma unroll
        for (int s = 1; s <= S; ++s) {
          const int t = d - s;
          if (t < 1 || t > S) continue;
#pragma unroll
          for (int kk = 0; kk < TBK / 16; ++kk) {
            const uint64_t ad = sw128_desc(a0 + (uint32_t)((s - 1) * A_SLICE) + kk * 32);
            const uint64_t bd = sw128_desc(b0 + (uint32_t)((t - 1) * B_SLICE) + kk * 32);
            mma_bf16(tmem, ad, bd, IDESC, acc);
            acc = 1u;
          }
        }
      }
      mma_commit(&mbar[st]);
    }
    ++issued;
  }
  // wait for the last commit (it tracks every earlier MMA of this thread);
  // after a failed wait this is the bounded wait for the MMAs still in flight
  if (issued > 0 && tid == 0) {
    const int last = issued - 1;
    if (!mbar_wait(&mbar[last & 1], (uint32_t)((last >> 1) & 1))) s_fail = 1;
  }
  __syncthreads();
  tc_fence_after();
  if (s_fail) {
    if (tid == 0) atomicOr(g.status, RQRCP_INFO_TIMEOUT);
  } else {
    // epilogue: warp w owns accumulator lanes (rows) 32w..32w+31
    const int64_t i = i0 + 32 * warp + lane;
    for (int c0 = 0; c0 < BN; c0 += 32) {
      float v[32];
      if (issued > 0) {
        tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
      } else {
#pragma unroll
        for (int e = 0; e < 32; ++e) v[e] = 0.0f;
      }
      if (i < g.M) {
        if (g.partial != nullptr) {
          float* pp = g.partial + (int64_t)blockIdx.z * g.M * g.N;
#pragma unroll
          for (int e = 0; e < 32; ++e) {
            const int64_t j = j0 + c0 + e;
            if (j < g.N) pp[i + j * g.M] = v[e];
          }
        } else {
#pragma unroll
          for (int e = 0; e < 32; ++e) {
            const int64_t j = j0 + c0 + e;
            if (j < g.N) {
              float* cp = g.C + i + j * g.ldc;
              float out = g.alpha * v[e];
              if (g.beta != 0.0f) out = fmaf(g.beta, *cp, out);
              *cp = out;
            }
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)BN)
                 : "memory");
}

// C = alpha * sum_z partial[z] + beta C, in a fixed order
__global__ void tc_splitk_reduce(TcGemmArgs g, int splits) {
  const int64_t total = g.M * g.N;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int z = 0; z < splits; ++z) s += g.partial[(int64_t)z * total + e];
    const int64_t i = e % g.M, j = e / g.M;
    float* cp = g.C + i + j * g.ldc;
    float out = g.alpha * s;
    if (g.beta != 0.0f) out = fmaf(g.beta, *cp, out);
    *cp = out;
  }
}

template <int S, int BN>
size_t tc_smem() {
  return 2 * (size_t)S * ((size_t)TBM * 128 + (size_t)BN * 128) + 1024;
}

template <int S, int BN, char TA, char TB>
cudaError_t launch_variant(const TcGemmArgs& g, cudaStream_t st) {
  auto kern = tc_gemm_kernel<S, BN, TA, TB>;
  const size_t smem = tc_smem<S, BN>();
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int KT_all = (int)((g.K + TBK - 1) / TBK);
  const int splits = KT_all > 0 ? (KT_all + g.kt_per_split - 1) / g.kt_per_split : 1;
  dim3 grid((unsigned)((g.M + TBM - 1) / TBM), (unsigned)((g.N + BN - 1) / BN), (unsigned)splits);
  kern<<<grid, TNT, smem, st>>>(g);
  e = cudaGetLastError();
  if (e != cudaSuccess || g.partial == nullptr) return e;
  const int64_t total = g.M * g.N;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  tc_splitk_reduce<<<(unsigned)blocks, 256, 0, st>>>(g, splits);
  return cudaGetLastError();
}

template <int S, int BN>
cudaError_t dispatch_trans(const TcGemmArgs& g, cudaStream_t st) {
  if (g.transA == 'N' && g.transB == 'N') return launch_variant<S, BN, 'N', 'N'>(g, st);
  if (g.transA == 'N') return launch_variant<S, BN, 'N', 'T'>(g, st);
  if (g.transB == 'N') return launch_variant<S, BN, 'T', 'N'>(g, st);
  return launch_variant<S, BN, 'T', 'T'>(g, st);
}

}  // namespace

int tc_pick_splits(int64_t M, int64_t N, int64_t K, int num_sms, size_t cap_floats) {
  const int64_t tiles = ((M + TBM - 1) / TBM) * ((N + 127) / 128);
  const int64_t kts = (K + TBK - 1) / TBK;
  int64_t s = 1;
  while (tiles * s < num_sms && s * 2 <= kts / 2 && (size_t)(s * 2) * M * N <= cap_floats) s *= 2;
  return (int)s;
}

cudaError_t launch_tc_gemm(TcGemmArgs g, int slices, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0) return cudaSuccess;
  // splits > 1 needs the partial buffer; kt_per_split is derived here
  const int KT_all = (int)((g.K + TBK - 1) / TBK);
  if (g.splits <= 1 || g.partial == nullptr || KT_all <= 1) {
    g.splits = 1;
    g.partial = nullptr;
    g.kt_per_split = KT_all > 0 ? KT_all : 1;
  } else {
    g.kt_per_split = (KT_all + g.splits - 1) / g.splits;
  }
  g.vecA = (g.transA == 'T') && (g.lda % 4 == 0) && ((reinterpret_cast<uintptr_t>(g.A) & 15) == 0);
  g.vecB = (g.transB == 'N') && (g.ldb % 4 == 0) && ((reinterpret_cast<uintptr_t>(g.B) & 15) == 0);
  if (slices == 1) return dispatch_trans<1, 128>(g, st);
  if (slices == 3) return dispatch_trans<3, 128>(g, st);
  return cudaErrorInvalidValue;
}

}  // namespace rq
