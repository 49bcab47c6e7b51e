// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC 2011) and the Box-Muller
// pair of normals used for every Gaussian sketch of the library (§3.1,
// construction of V-hat, step 1).  Device code only, shared by the kernels.
#pragma once

#include <stdint.h>

namespace rutv {

struct PhiloxKey {
  uint32_t k0, k1;
};

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, PhiloxKey k) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k.k0 += W0;
      k.k1 += W1;
    }
    const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
    const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.k0, lo1, hi0 ^ c.w ^ k.k1, lo0);
  }
  return c;
}

// Two normals from one counter: 53-bit uniforms u1 in (0,1], u2 in [0,1).
__device__ __forceinline__ void box_muller(uint4 w, double* z0, double* z1) {
  const uint64_t j1 = (uint64_t)(w.x >> 5) * 67108864ull + (uint64_t)(w.y >> 6);
  const uint64_t j2 = (uint64_t)(w.z >> 5) * 67108864ull + (uint64_t)(w.w >> 6);
  const double u1 = (double)(j1 + 1ull) * 0x1.0p-53;
  const double u2 = (double)j2 * 0x1.0p-53;
  const double rho = sqrt(-2.0 * log(u1));
  double s, c;
  sincospi(2.0 * u2, &s, &c);
  *z0 = rho * c;
  *z1 = rho * s;
}

// The batched form's FP32 pair: 24-bit uniforms u1 = ((x0 >> 8) + 1) 2^-24
// in (0, 1] and u2 = (x2 >> 8) 2^-24 in [0, 1) (both exact in FP32),
// rho = sqrt(-2 ln u1), (rho cos 2 pi u2, rho sin 2 pi u2) in FP32 arithmetic.
__device__ __forceinline__ void box_muller_f32(uint4 w, float* z0, float* z1) {
  const float u1 = (float)((w.x >> 8) + 1u) * 0x1.0p-24f;
  const float u2 = (float)(w.z >> 8) * 0x1.0p-24f;
  const float rho = sqrtf(-2.f * logf(u1));
  float s, c;
  sincospif(2.f * u2, &s, &c);
  *z0 = rho * c;
  *z1 = rho * s;
}

}  // namespace rutv
