// Philox4x32-10 on the device (Salmon, Moraes, Dror, Shaw, SC'11: ten rounds of
// two 32x32->64 multiplies by 0xD2511F53 / 0xCD9E8D57 with a Weyl key bump of
// 0x9E3779B9 / 0xBB67AE85 between rounds).  The round keys come precomputed in
// kernel-parameter space so each round is two wide multiplies and two
// three-input XORs.
#pragma once

#include <stdint.h>

#include "internal.h"

namespace xzzx {

__device__ __forceinline__ uint4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                               const PhiloxKeys& K) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)c0 * 0xD2511F53u;
    const uint64_t p1 = (uint64_t)c2 * 0xCD9E8D57u;
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ K.k0[r];
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ K.k1[r];
    c1 = (uint32_t)p1;
    c3 = (uint32_t)p0;
    c0 = n0;
    c2 = n2;
  }
  return make_uint4(c0, c1, c2, c3);
}

__device__ __forceinline__ uint32_t lane_of(const uint4& v, int lane) {
  return lane == 0 ? v.x : lane == 1 ? v.y : lane == 2 ? v.z : v.w;
}

}  // namespace xzzx
