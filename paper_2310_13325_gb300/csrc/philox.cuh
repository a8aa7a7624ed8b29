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

// Two standard normals from two 32-bit words. The radius is formed from a
// double-precision logarithm so that uniforms near 1 keep their accuracy.
__device__ __forceinline__ float2 box_muller(uint32_t ua, uint32_t ub) {
  const double Ua = ((double)(ua >> 8) + 0.5) * (1.0 / 16777216.0);
  const float r = (float)sqrt(-2.0 * log(Ua));
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
