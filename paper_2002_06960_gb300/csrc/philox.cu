// Gaussian sketch generator: Philox4x32-10 + Box-Muller, FP64 output.
//
// The sketch G of each block step is i.i.d. standard normal (§3.1,
// construction of V-hat, step 1).  The generator is counter based
// (Salmon, Moraes, Dror & Shaw, SC 2011), so every element is a pure function
// of (seed, step, matrix id, stream id, element index): no state is carried
// between steps, a resumed factorization draws the same sketch, and the CPU
// checker draws the same words.
#include "common.cuh"

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

__global__ void philox_normal_kernel(PhiloxKey key, uint32_t step, uint32_t mid, uint32_t sid,
                                     int64_t rows, int64_t count, double* __restrict__ G,
                                     int64_t ldg) {
  const int64_t npairs = (count + 1) >> 1;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npairs;
       p += (int64_t)gridDim.x * blockDim.x) {
    const uint4 w = philox4x32_10(make_uint4((uint32_t)p, step, mid, sid), key);
    double z0, z1;
    box_muller(w, &z0, &z1);
    const int64_t l0 = 2 * p;
    G[(l0 % rows) + (l0 / rows) * ldg] = z0;
    if (l0 + 1 < count) G[((l0 + 1) % rows) + ((l0 + 1) / rows) * ldg] = z1;
  }
}

__global__ void philox_words_kernel(PhiloxKey key, uint4 c, int64_t count, uint32_t* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint4 w = philox4x32_10(make_uint4(c.x + (uint32_t)i, c.y, c.z, c.w), key);
    out[4 * i + 0] = w.x;
    out[4 * i + 1] = w.y;
    out[4 * i + 2] = w.z;
    out[4 * i + 3] = w.w;
  }
}

int launch_philox_normal(uint64_t seed, uint32_t step, uint32_t mid, uint32_t sid, int64_t rows,
                         int64_t cols, double* G, int64_t ldg, cudaStream_t st) {
  const int64_t count = rows * cols;
  if (count == 0) return 0;
  const int64_t npairs = (count + 1) >> 1;
  const int threads = 256;
  int64_t blocks = (npairs + threads - 1) / threads;
  const int64_t cap = (int64_t)dev_info().sms * 16;
  if (blocks > cap) blocks = cap;
  PhiloxKey key{(uint32_t)seed, (uint32_t)(seed >> 32)};
  ProfScope prof(K_PHILOX, 0.0, 8.0 * (double)count, st);
  philox_normal_kernel<<<(unsigned)blocks, threads, 0, st>>>(key, step, mid, sid, rows, count, G,
                                                            ldg);
  note_launch();
  RUTV_CK(cudaGetLastError());
  return 0;
}

int launch_philox_words(uint64_t seed, uint4 c, int64_t count, uint32_t* out, cudaStream_t st) {
  if (count == 0) return 0;
  const int threads = 256;
  int64_t blocks = (count + threads - 1) / threads;
  if (blocks > 4096) blocks = 4096;
  PhiloxKey key{(uint32_t)seed, (uint32_t)(seed >> 32)};
  philox_words_kernel<<<(unsigned)blocks, threads, 0, st>>>(key, c, count, out);
  note_launch();
  RUTV_CK(cudaGetLastError());
  return 0;
}

}  // namespace rutv

// ---- BF16 sketch for the mixed-precision path: RNE(bf16) of the same FP64 normals.
#include <cuda_bf16.h>

namespace rutv {

__global__ void philox_normal_bf16_kernel(PhiloxKey key, uint32_t step, uint32_t mid, uint32_t sid,
                                          int64_t rows, int64_t count, __nv_bfloat16* G,
                                          int64_t ldg) {
  const int64_t npairs = (count + 1) >> 1;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npairs;
       p += (int64_t)gridDim.x * blockDim.x) {
    const uint4 w = philox4x32_10(make_uint4((uint32_t)p, step, mid, sid), key);
    double z0, z1;
    box_muller(w, &z0, &z1);
    const int64_t l0 = 2 * p;
    G[(l0 % rows) + (l0 / rows) * ldg] = __double2bfloat16(z0);
    if (l0 + 1 < count) G[((l0 + 1) % rows) + ((l0 + 1) / rows) * ldg] = __double2bfloat16(z1);
  }
}

int philox_normal_bf16(uint64_t seed, uint32_t step, uint32_t mid, uint32_t sid, int64_t rows,
                       int64_t cols, __nv_bfloat16* G, int64_t ldg, cudaStream_t st) {
  const int64_t count = rows * cols;
  if (count == 0) return 0;
  const int64_t npairs = (count + 1) >> 1;
  int64_t blocks = (npairs + 255) / 256;
  const int64_t cap = (int64_t)dev_info().sms * 16;
  if (blocks > cap) blocks = cap;
  PhiloxKey key{(uint32_t)seed, (uint32_t)(seed >> 32)};
  ProfScope prof(K_PHILOX, 0.0, 2.0 * (double)count, st);
  philox_normal_bf16_kernel<<<(unsigned)blocks, 256, 0, st>>>(key, step, mid, sid, rows, count, G,
                                                              ldg);
  note_launch();
  RUTV_CK(cudaGetLastError());
  return 0;
}

}  // namespace rutv
