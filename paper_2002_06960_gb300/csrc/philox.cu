// Gaussian sketch generator: Philox4x32-10 + Box-Muller, FP64 output.
//
// The sketch G of each block step is i.i.d. standard normal (§3.1,
// construction of V-hat, step 1).  The generator is counter based
// (Salmon, Moraes, Dror & Shaw, SC 2011), so every element is a pure function
// of (seed, step, matrix id, stream id, element index): no state is carried
// between steps, a resumed factorization draws the same sketch, and the CPU
// checker draws the same words.
#include "common.cuh"
#include "philox.cuh"

namespace rutv {

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

// Rows row0 .. row0 + nrows - 1 of the rows_total x cols sketch (element
// l = r + c rows_total of the whole), into G (nrows x cols, ld ldg): a tile of
// the sketch that equals the same rows of the whole one.
__global__ void philox_normal_rows_kernel(PhiloxKey key, uint32_t step, uint32_t mid, uint32_t sid,
                                          int64_t rows_total, int64_t row0, int64_t nrows,
                                          int64_t cols, double* __restrict__ G, int64_t ldg) {
  const int64_t total = nrows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e % nrows, c = e / nrows;
    const int64_t l = (row0 + r) + c * rows_total;
    const uint4 w = philox4x32_10(make_uint4((uint32_t)(l >> 1), step, mid, sid), key);
    double z0, z1;
    box_muller(w, &z0, &z1);
    G[r + c * ldg] = (l & 1) ? z1 : z0;
  }
}

int launch_philox_normal_rows(uint64_t seed, uint32_t step, uint32_t mid, uint32_t sid,
                              int64_t rows_total, int64_t row0, int64_t nrows, int64_t cols,
                              double* G, int64_t ldg, cudaStream_t st) {
  const int64_t total = nrows * cols;
  if (total <= 0) return 0;
  int64_t blocks = (total + 255) / 256;
  const int64_t cap = (int64_t)dev_info().sms * 16;
  if (blocks > cap) blocks = cap;
  PhiloxKey key{(uint32_t)seed, (uint32_t)(seed >> 32)};
  ProfScope prof(K_PHILOX, 0.0, 8.0 * (double)total, st);
  philox_normal_rows_kernel<<<(unsigned)blocks, 256, 0, st>>>(key, step, mid, sid, rows_total,
                                                              row0, nrows, cols, G, ldg);
  note_launch();
  RUTV_CK(cudaGetLastError());
  return 0;
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

__global__ void philox_normal_f32_kernel(PhiloxKey key, uint32_t step, uint32_t mid, uint32_t sid,
                                         int64_t rows, int64_t count, float* __restrict__ G,
                                         int64_t ldg) {
  const int64_t npairs = (count + 1) >> 1;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npairs;
       p += (int64_t)gridDim.x * blockDim.x) {
    const uint4 w = philox4x32_10(make_uint4((uint32_t)p, step, mid, sid), key);
    float z0, z1;
    box_muller_f32(w, &z0, &z1);
    const int64_t l0 = 2 * p;
    G[(l0 % rows) + (l0 / rows) * ldg] = z0;
    if (l0 + 1 < count) G[((l0 + 1) % rows) + ((l0 + 1) / rows) * ldg] = z1;
  }
}

int launch_philox_normal_f32(uint64_t seed, uint32_t step, uint32_t mid, uint32_t sid,
                             int64_t rows, int64_t cols, float* G, int64_t ldg, cudaStream_t st) {
  const int64_t count = rows * cols;
  if (count == 0) return 0;
  const int64_t npairs = (count + 1) >> 1;
  int64_t blocks = (npairs + 255) / 256;
  const int64_t cap = (int64_t)dev_info().sms * 16;
  if (blocks > cap) blocks = cap;
  PhiloxKey key{(uint32_t)seed, (uint32_t)(seed >> 32)};
  ProfScope prof(K_PHILOX, 0.0, 4.0 * (double)count, st);
  philox_normal_f32_kernel<<<(unsigned)blocks, 256, 0, st>>>(key, step, mid, sid, rows, count, G,
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
