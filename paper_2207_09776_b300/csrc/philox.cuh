// Philox4x32-10 counter-based generator and Box-Muller normals (device side).
//
// Written from the published definition (Salmon, Moraes, Dror, Shaw, "Parallel
// random numbers: as easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64-bit
// multiplications by 0xD2511F53 and 0xCD9E8D57 mixing a four-word counter with
// a two-word key, the key bumped by the Weyl constants 0x9E3779B9, 0xBB67AE85
// between rounds.
//
// Stream layout: key = (seed lo, seed hi); counter = (pair j, path lo, path hi,
// tag).  Words (x0,x1) and (x2,x3) give two uniforms ((hi:lo >> 12) + 1/2) 2^-52
// in (0, 1) (exact in double), and Box-Muller gives the standard normals of
// fine indices 2j (cosine branch) and 2j+1 (sine branch).
#pragma once

#include <stdint.h>

__host__ __device__ __forceinline__ uint32_t mulhi32(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
  return __umulhi(a, b);
#else
  return (uint32_t)(((uint64_t)a * (uint64_t)b) >> 32);
#endif
}

__host__ __device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = mulhi32(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = mulhi32(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

__device__ __forceinline__ double uniform52(uint32_t lo, uint32_t hi) {
  const uint64_t u = ((uint64_t)hi << 32) | (uint64_t)lo;
  return ((double)(u >> 12) + 0.5) * 0x1p-52;
}

// Standard normals of fine indices 2j and 2j+1 of global path `path`.
__device__ __forceinline__ void brownian_pair(uint64_t seed, uint64_t path, uint32_t tag, uint64_t j,
                                              double& z0, double& z1) {
  const uint4 w = philox4x32_10(
      make_uint4((uint32_t)j, (uint32_t)path, (uint32_t)(path >> 32), tag),
      make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
  const double u1 = uniform52(w.x, w.y);
  const double u2 = uniform52(w.z, w.w);
  const double r = sqrt(-2.0 * log(u1));
  double s, c;
  sincospi(2.0 * u2, &s, &c);
  z0 = r * c;
  z1 = r * s;
}

// The same pair with the normals formed in single precision: uniforms
// (hi + 1/2) 2^-32 from the high word of each half of the counter block
// (within 2^-32 of the double-precision uniforms), Box-Muller in float
// (returned as float, or widened to double).  Used by the float solves, where
// the double-precision Box-Muller would dominate the cost of the Brownian kernel.
__device__ __forceinline__ void brownian_pair_f32f(uint64_t seed, uint64_t path, uint32_t tag, uint64_t j,
                                                   float& z0, float& z1) {
  const uint4 w = philox4x32_10(
      make_uint4((uint32_t)j, (uint32_t)path, (uint32_t)(path >> 32), tag),
      make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
  const float u1 = fmaf((float)w.y, 0x1p-32f, 0x1p-33f);
  const float u2 = fmaf((float)w.w, 0x1p-32f, 0x1p-33f);
  const float r = sqrtf(-2.0f * logf(u1));
  float s, c;
  sincospif(2.0f * u2, &s, &c);
  z0 = r * c;
  z1 = r * s;
}
__device__ __forceinline__ void brownian_pair_f32(uint64_t seed, uint64_t path, uint32_t tag, uint64_t j,
                                                  double& z0, double& z1) {
  float a, b;
  brownian_pair_f32f(seed, path, tag, j, a, b);
  z0 = (double)a;
  z1 = (double)b;
}
