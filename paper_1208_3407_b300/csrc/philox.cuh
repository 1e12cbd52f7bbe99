// Philox4x32-10 counter-based generator (Salmon, Moraes, Dror and Shaw,
// "Parallel random numbers: as easy as 1, 2, 3", SC'11), device side.
//
// One round maps the counter (c0, c1, c2, c3) with key (k0, k1) to
//     (hi(M1*c2) ^ c1 ^ k0,  lo(M1*c2),  hi(M0*c0) ^ c3 ^ k1,  lo(M0*c0))
// with M0 = 0xD2511F53, M1 = 0xCD9E8D57; the key advances by the Weyl
// constants (0x9E3779B9, 0xBB67AE85) between rounds; ten rounds.
#pragma once

#include <stdint.h>

namespace bits {

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
  #pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// Uniform offset in [0, range) from the first two output words:
// floor(u * range / 2^64) with u = x1 * 2^32 + x0 (integer-exact).
__device__ __forceinline__ uint32_t philox_offset(uint4 x, uint32_t range) {
  const unsigned long long u = ((unsigned long long)x.y << 32) | x.x;
  return (uint32_t)__umul64hi(u, (unsigned long long)range);
}

}  // namespace bits
