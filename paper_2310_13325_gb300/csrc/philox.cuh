// Philox-4x32-10 counter-based generator (Salmon, Moraes, Dror & Shaw,
// "Parallel random numbers: as easy as 1, 2, 3", SC 2011) and the Box-Muller
// mapping used for the sSVGD noise Xi (Eq. 25) and the ADVI draws eta.
//
// Element (row i, column c) of an [n][d] normal array at iteration t under
// seed s uses counter (c/4, i, t mod 2^32, t >> 32) and key (s mod 2^32,
// s >> 32); the output words (u0, u1, u2, u3) give z0, z1 from (u0, u1) and
// z2, z3 from (u2, u3) with U = ((u >> 8) + 1/2) 2^-24,
// r = sqrt(-2 ln U_a), angle = 2 pi U_b, (r cos, r sin); column c takes z_{c%4}.
#pragma once
#include <stdint.h>

namespace vip {

__device__ __forceinline__ uint4 philox4x32_10(uint4 x, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    const uint32_t lo0 = 0xD2511F53u * x.x, hi0 = __umulhi(0xD2511F53u, x.x);
    const uint32_t lo1 = 0xCD9E8D57u * x.z, hi1 = __umulhi(0xCD9E8D57u, x.z);
    x = make_uint4(hi1 ^ x.y ^ k0, lo1, hi0 ^ x.w ^ k1, lo0);
  }
  return x;
}

// Two standard normals from two 32-bit words. With k = ua >> 8, U_a = (k +
// 1/2) 2^-24 and 1 - U_a = (2^24 - k - 1/2) 2^-24 both have at most 24
// significant bits, so each is exact in FP32: ln U_a is taken as logf(U_a)
// below one half and as log1pf(-(1 - U_a)) above, where the argument of logf
// would lose the small difference from 1. FP32 throughout (FP64 is slow on
// this GPU); the radius is within a few FP32 ulps of the FP64 value.
__device__ __forceinline__ float2 box_muller(uint32_t ua, uint32_t ub) {
  const uint32_t k = ua >> 8;
  const float lg = k >= (1u << 23)
                       ? log1pf(-((float)((1u << 24) - k) - 0.5f) * (1.0f / 16777216.0f))
                       : logf(((float)k + 0.5f) * (1.0f / 16777216.0f));
  const float r = sqrtf(-2.0f * lg);
  const float t = fmaf((float)(ub >> 8), 1.0f / 8388608.0f, 1.0f / 16777216.0f);  // 2 U_b
  float s, c;
  sincospif(t, &s, &c);
  return make_float2(r * c, r * s);
}

// Four normals of row i, columns 4q .. 4q+3.
__device__ __forceinline__ float4 philox_normal4(uint64_t seed, uint64_t it, uint32_t i,
                                                 uint32_t q) {
  const uint4 u = philox4x32_10(make_uint4(q, i, (uint32_t)it, (uint32_t)(it >> 32)),
                                (uint32_t)seed, (uint32_t)(seed >> 32));
  const float2 a = box_muller(u.x, u.y), b = box_muller(u.z, u.w);
  return make_float4(a.x, a.y, b.x, b.y);
}

}  // namespace vip
