// Philox4x32-10 (Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as
// easy as 1, 2, 3", SC'11) and the open-interval uniform of the Gaussian
// generator, shared by the Omega kernels and the persistent batched kernel.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace rq {
namespace px {

// Philox4x32 round multipliers and Weyl key increments (Salmon et al. SC'11).
constexpr uint32_t kM0 = 0xD2511F53u;
constexpr uint32_t kM1 = 0xCD9E8D57u;
constexpr uint32_t kW0 = 0x9E3779B9u;
constexpr uint32_t kW1 = 0xBB67AE85u;

__device__ __forceinline__ uint4 philox10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k.x += kW0;
      k.y += kW1;
    }
    uint32_t hi0 = __umulhi(kM0, c.x), lo0 = kM0 * c.x;
    uint32_t hi1 = __umulhi(kM1, c.z), lo1 = kM1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// (top 52 bits of hi:lo + 1/2) * 2^-52, strictly inside (0, 1).
__device__ __forceinline__ double unit_open(uint32_t lo, uint32_t hi) {
  uint64_t t = ((uint64_t)hi << 20) | (uint64_t)(lo >> 12);
  return ((double)t + 0.5) * 0x1.0p-52;
}

}  // namespace px
}  // namespace rq
