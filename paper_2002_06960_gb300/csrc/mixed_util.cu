// Conversions between FP32 / FP64 matrices and BF16 planes for the
// mixed-precision path, and the small element-wise kernels around it.
//
// A plane triple holds X = X0 + X1 + X2 with X0 = bf16(X), X1 = bf16(X - X0),
// X2 = bf16(X - X0 - X1), round-to-nearest-even at each step: 24 significant
// bits in all, the precision of FP32 storage.
#include <cuda_bf16.h>

#include "common.cuh"
#include "mixed.h"

namespace rutv {

namespace {

__device__ __forceinline__ void split3(double x, __nv_bfloat16* h0, __nv_bfloat16* h1,
                                       __nv_bfloat16* h2) {
  const __nv_bfloat16 a = __double2bfloat16(x);
  const double r1 = x - (double)__bfloat162float(a);
  const __nv_bfloat16 b = __double2bfloat16(r1);
  const double r2 = r1 - (double)__bfloat162float(b);
  *h0 = a;
  *h1 = b;
  *h2 = __double2bfloat16(r2);
}

__device__ __forceinline__ double join3(const __nv_bfloat16* P0, const __nv_bfloat16* P1,
                                        const __nv_bfloat16* P2, int64_t o) {
  return (double)__bfloat162float(P0[o]) + (double)__bfloat162float(P1[o]) +
         (double)__bfloat162float(P2[o]);
}

template <typename T>
__global__ void split_kernel(const T* __restrict__ src, int64_t lds, int64_t rows, int64_t cols,
                             int trans, __nv_bfloat16* P0, __nv_bfloat16* P1, __nv_bfloat16* P2,
                             int64_t ldp) {
  const int64_t total = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % rows, j = e / rows;
    const double x = trans ? (double)src[j + i * lds] : (double)src[i + j * lds];
    const int64_t o = i + j * ldp;
    split3(x, P0 + o, P1 + o, P2 + o);
  }
}

template <typename T>
__global__ void merge_kernel(const __nv_bfloat16* P0, const __nv_bfloat16* P1,
                             const __nv_bfloat16* P2, int64_t ldp, int64_t rows, int64_t cols,
                             int trans, T* __restrict__ dst, int64_t ldd) {
  const int64_t total = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % rows, j = e / rows;  // element of dst
    const int64_t o = trans ? (j + i * ldp) : (i + j * ldp);
    dst[i + j * ldd] = (T)join3(P0, P1, P2, o);
  }
}

__global__ void absmax_kernel(const float* __restrict__ src, int64_t lds, int64_t rows,
                              int64_t cols, unsigned* out) {
  const int64_t total = rows * cols;
  float m = 0.f;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % rows, j = e / rows;
    m = fmaxf(m, fabsf(src[i + j * lds]));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));  // m >= 0: bits order as values
}

__global__ void scale_bf16_kernel(const float* __restrict__ src, int64_t lds, int64_t rows,
                                  int64_t cols, const unsigned* amax, __nv_bfloat16* dst,
                                  int64_t ldd) {
  int e = 0;
  const float mx = __uint_as_float(*amax);
  if (mx > 0.f && isfinite(mx)) frexpf(mx, &e);
  const float s = ldexpf(1.f, -e);  // exact power of two
  const int64_t total = rows * cols;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t % rows, j = t / rows;
    dst[i + j * ldd] = __float2bfloat16_rn(src[i + j * lds] * s);
  }
}

__global__ void identity_planes_kernel(int64_t rows, int64_t cols, __nv_bfloat16* P0,
                                       __nv_bfloat16* P1, __nv_bfloat16* P2, int64_t ld) {
  const int64_t total = rows * cols;
  const __nv_bfloat16 one = __float2bfloat16(1.f), zero = __float2bfloat16(0.f);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % rows, j = e / rows, o = i + j * ld;
    P0[o] = (i == j) ? one : zero;
    P1[o] = zero;
    P2[o] = zero;
  }
}

__global__ void diag_planes_kernel(__nv_bfloat16* P0, __nv_bfloat16* P1, __nv_bfloat16* P2,
                                   int64_t ld, int64_t k, int64_t bi, const double* D) {
  const int64_t total = bi * bi;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % bi, j = e / bi, o = (k + i) + (k + j) * ld;
    split3(i == j ? D[i] : 0.0, P0 + o, P1 + o, P2 + o);
  }
}

int grid_of(int64_t total) {
  int64_t blocks = (total + 255) / 256;
  const int64_t cap = (int64_t)dev_info().sms * 16;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  return (int)blocks;
}

}  // namespace

int split_f32(const float* src, int64_t lds, int64_t rows, int64_t cols, int trans,
              const Planes& dst, int64_t r0, int64_t c0, cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return 0;
  ProfScope prof(K_CONVERT, 0.0, 10.0 * rows * (double)cols, st);
  split_kernel<float><<<grid_of(rows * cols), 256, 0, st>>>(
      src, lds, rows, cols, trans, dst.at(0, r0, c0), dst.at(1, r0, c0), dst.at(2, r0, c0), dst.ld);
  note_launch();
  RUTV_CK(cudaGetLastError());
  return 0;
}

int split_f64(const double* src, int64_t lds, int64_t rows, int64_t cols, int trans,
              const Planes& dst, int64_t r0, int64_t c0, cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return 0;
  ProfScope prof(K_CONVERT, 0.0, 14.0 * rows * (double)cols, st);
  split_kernel<double><<<grid_of(rows * cols), 256, 0, st>>>(
      src, lds, rows, cols, trans, dst.at(0, r0, c0), dst.at(1, r0, c0), dst.at(2, r0, c0), dst.ld);
  note_launch();
  RUTV_CK(cudaGetLastError());
  return 0;
}

int merge_f32(const Planes& src, int64_t r0, int64_t c0, int64_t rows, int64_t cols, int trans,
              float* dst, int64_t ldd, cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return 0;
  ProfScope prof(K_CONVERT, 0.0, 10.0 * rows * (double)cols, st);
  merge_kernel<float><<<grid_of(rows * cols), 256, 0, st>>>(
      src.at(0, r0, c0), src.at(1, r0, c0), src.at(2, r0, c0), src.ld, rows, cols, trans, dst, ldd);
  note_launch();
  RUTV_CK(cudaGetLastError());
  return 0;
}

int merge_f64(const Planes& src, int64_t r0, int64_t c0, int64_t rows, int64_t cols, int trans,
              double* dst, int64_t ldd, cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return 0;
  ProfScope prof(K_CONVERT, 0.0, 14.0 * rows * (double)cols, st);
  merge_kernel<double><<<grid_of(rows * cols), 256, 0, st>>>(
      src.at(0, r0, c0), src.at(1, r0, c0), src.at(2, r0, c0), src.ld, rows, cols, trans, dst, ldd);
  note_launch();
  RUTV_CK(cudaGetLastError());
  return 0;
}

int scaled_bf16(const float* src, int64_t lds, int64_t rows, int64_t cols, __nv_bfloat16* dst,
                int64_t ldd, float* scratch, cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return 0;
  ProfScope prof(K_CONVERT, 0.0, 10.0 * rows * (double)cols, st);
  unsigned* amax = (unsigned*)scratch;
  RUTV_CK(cudaMemsetAsync(amax, 0, sizeof(unsigned), st));
  absmax_kernel<<<grid_of(rows * cols), 256, 0, st>>>(src, lds, rows, cols, amax);
  scale_bf16_kernel<<<grid_of(rows * cols), 256, 0, st>>>(src, lds, rows, cols, amax, dst, ldd);
  note_launch(2);
  RUTV_CK(cudaGetLastError());
  return 0;
}

int set_identity_planes(const Planes& X, cudaStream_t st) {
  if (X.rows <= 0 || X.cols <= 0) return 0;
  identity_planes_kernel<<<grid_of(X.rows * X.cols), 256, 0, st>>>(X.rows, X.cols, X.p[0], X.p[1],
                                                                   X.p[2], X.ld);
  note_launch();
  RUTV_CK(cudaGetLastError());
  return 0;
}

namespace {
__global__ void check_finite_f32_kernel(int64_t rows, int64_t cols, const float* X, int64_t ld,
                                        unsigned* err) {
  const int64_t total = rows * cols;
  int bad = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    bad |= !isfinite(X[(e % rows) + (e / rows) * ld]);
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) {
    if (atomicCAS(err, 0u, (unsigned)RANDUTV_ENONFINITE) == 0u) atomicExch(err + 1, 100u);
  }
}
}  // namespace

int launch_check_finite_f32(int64_t rows, int64_t cols, const float* X, int64_t ld, unsigned* err,
                            cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return 0;
  check_finite_f32_kernel<<<grid_of(rows * cols), 256, 0, st>>>(rows, cols, X, ld, err);
  note_launch();
  RUTV_CK(cudaGetLastError());
  return 0;
}

int set_diag_planes(const Planes& T, int64_t k, int64_t bi, const double* D, cudaStream_t st) {
  if (bi <= 0) return 0;
  diag_planes_kernel<<<grid_of(bi * bi), 256, 0, st>>>(T.p[0], T.p[1], T.p[2], T.ld, k, bi, D);
  note_launch();
  RUTV_CK(cudaGetLastError());
  return 0;
}

}  // namespace rutv
