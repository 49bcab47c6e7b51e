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

// FP32 split and join in FP32 arithmetic: x - bf16(x) and the next residual
// are exact in FP32, and P0 + P1 spans at most 16 bits, so both give the same
// bits as the FP64 forms (one rounding of an exact sum in the join).
__device__ __forceinline__ void split3f(float x, __nv_bfloat16& h0, __nv_bfloat16& h1,
                                        __nv_bfloat16& h2) {
  h0 = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(h0);
  h1 = __float2bfloat16_rn(r1);
  h2 = __float2bfloat16_rn(r1 - __bfloat162float(h1));
}
__device__ __forceinline__ void split3(double x, __nv_bfloat16& h0, __nv_bfloat16& h1,
                                       __nv_bfloat16& h2) {
  h0 = __double2bfloat16(x);
  const double r1 = x - (double)__bfloat162float(h0);
  h1 = __double2bfloat16(r1);
  h2 = __double2bfloat16(r1 - (double)__bfloat162float(h1));
}
__device__ __forceinline__ void split3t(float x, __nv_bfloat16& a, __nv_bfloat16& b, __nv_bfloat16& c) {
  split3f(x, a, b, c);
}
__device__ __forceinline__ void split3t(double x, __nv_bfloat16& a, __nv_bfloat16& b, __nv_bfloat16& c) {
  split3(x, a, b, c);
}
__device__ __forceinline__ float join3f(__nv_bfloat16 a, __nv_bfloat16 b, __nv_bfloat16 c) {
  return (__bfloat162float(a) + __bfloat162float(b)) + __bfloat162float(c);
}
__device__ __forceinline__ double join3d(__nv_bfloat16 a, __nv_bfloat16 b, __nv_bfloat16 c) {
  return (double)__bfloat162float(a) + (double)__bfloat162float(b) + (double)__bfloat162float(c);
}
template <typename T> __device__ __forceinline__ T join3t(__nv_bfloat16 a, __nv_bfloat16 b, __nv_bfloat16 c);
template <> __device__ __forceinline__ float join3t<float>(__nv_bfloat16 a, __nv_bfloat16 b, __nv_bfloat16 c) {
  return join3f(a, b, c);
}
template <> __device__ __forceinline__ double join3t<double>(__nv_bfloat16 a, __nv_bfloat16 b, __nv_bfloat16 c) {
  return join3d(a, b, c);
}

// Tiles of 32 x 32 elements, 32 x 8 threads.  Without trans both sides are
// read and written along columns; with trans the source tile goes through
// shared memory so that both the read (along the source's columns) and the
// write (along the planes' columns) are coalesced.
constexpr int CT = 32, CR = 8;

template <typename T>
__global__ void __launch_bounds__(CT * CR) split_kernel(const T* __restrict__ src, int64_t lds,
                                                         int64_t rows, int64_t cols, int trans,
                                                         __nv_bfloat16* P0, __nv_bfloat16* P1,
                                                         __nv_bfloat16* P2, int64_t ldp) {
  __shared__ T tile[CT][CT + 1];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int64_t i0 = (int64_t)blockIdx.x * CT, j0 = (int64_t)blockIdx.y * CT;  // dst tile
  if (trans) {
    // dst(i, j) = src(j, i) = src[j + i lds]: read src rows j0.. (contiguous) for columns i0..
#pragma unroll
    for (int k = 0; k < CT; k += CR) {
      const int64_t sj = j0 + tx, si = i0 + ty + k;
      if (sj < cols && si < rows) tile[ty + k][tx] = src[sj + si * lds];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < CT; k += CR) {
      const int64_t i = i0 + tx, j = j0 + ty + k;
      if (i < rows && j < cols) {
        __nv_bfloat16 a, b, c;
        split3t(tile[tx][ty + k], a, b, c);
        const int64_t o = i + j * ldp;
        P0[o] = a;
        P1[o] = b;
        P2[o] = c;
      }
    }
  } else {
#pragma unroll
    for (int k = 0; k < CT; k += CR) {
      const int64_t i = i0 + tx, j = j0 + ty + k;
      if (i < rows && j < cols) {
        __nv_bfloat16 a, b, c;
        split3t(src[i + j * lds], a, b, c);
        const int64_t o = i + j * ldp;
        P0[o] = a;
        P1[o] = b;
        P2[o] = c;
      }
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(CT * CR) merge_kernel(const __nv_bfloat16* P0,
                                                         const __nv_bfloat16* P1,
                                                         const __nv_bfloat16* P2, int64_t ldp,
                                                         int64_t rows, int64_t cols, int trans,
                                                         T* __restrict__ dst, int64_t ldd) {
  __shared__ T tile[CT][CT + 1];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int64_t i0 = (int64_t)blockIdx.x * CT, j0 = (int64_t)blockIdx.y * CT;  // dst tile
  if (trans) {
    // dst(i, j) = planes(j, i): read the planes' rows j0.. for their columns i0..
#pragma unroll
    for (int k = 0; k < CT; k += CR) {
      const int64_t pj = j0 + tx, pi = i0 + ty + k;
      if (pj < cols && pi < rows) {
        const int64_t o = pj + pi * ldp;
        tile[ty + k][tx] = join3t<T>(P0[o], P1[o], P2[o]);
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < CT; k += CR) {
      const int64_t i = i0 + tx, j = j0 + ty + k;
      if (i < rows && j < cols) dst[i + j * ldd] = tile[tx][ty + k];
    }
  } else {
#pragma unroll
    for (int k = 0; k < CT; k += CR) {
      const int64_t i = i0 + tx, j = j0 + ty + k;
      if (i < rows && j < cols) {
        const int64_t o = i + j * ldp;
        dst[i + j * ldd] = join3t<T>(P0[o], P1[o], P2[o]);
      }
    }
  }
}

dim3 tile_grid(int64_t rows, int64_t cols) {
  return dim3((unsigned)((rows + CT - 1) / CT), (unsigned)((cols + CT - 1) / CT));
}

// Columns by grid.y (striding), rows by grid.x x threads: no per-element division.
__global__ void absmax_kernel(const float* __restrict__ src, int64_t lds, int64_t rows,
                              int64_t cols, unsigned* out) {
  float m = 0.f;
  for (int64_t j = blockIdx.y; j < cols; j += gridDim.y)
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows;
         i += (int64_t)gridDim.x * blockDim.x)
      m = fmaxf(m, fabsf(src[i + j * lds]));
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
  for (int64_t j = blockIdx.y; j < cols; j += gridDim.y)
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows;
         i += (int64_t)gridDim.x * blockDim.x)
      dst[i + j * ldd] = __float2bfloat16_rn(src[i + j * lds] * s);
}

// grid of the two kernels above: enough CTAs of 256 threads for the rows of a
// column, times up to the columns (at most 16 CTAs per SM in all)
dim3 col_grid(int64_t rows, int64_t cols) {
  int64_t bx = (rows + 255) / 256;
  const int64_t cap = (int64_t)dev_info().sms * 16;
  if (bx > cap) bx = cap;
  int64_t by = cap / (bx > 0 ? bx : 1);
  if (by > cols) by = cols;
  if (by < 1) by = 1;
  if (by > 65535) by = 65535;
  return dim3((unsigned)(bx > 0 ? bx : 1), (unsigned)by);
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
    split3(i == j ? D[i] : 0.0, P0[o], P1[o], P2[o]);
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
  split_kernel<float><<<tile_grid(rows, cols), dim3(CT, CR), 0, st>>>(
      src, lds, rows, cols, trans, dst.at(0, r0, c0), dst.at(1, r0, c0), dst.at(2, r0, c0), dst.ld);
  note_launch();
  RUTV_CK(cudaGetLastError());
  return 0;
}

int split_f64(const double* src, int64_t lds, int64_t rows, int64_t cols, int trans,
              const Planes& dst, int64_t r0, int64_t c0, cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return 0;
  ProfScope prof(K_CONVERT, 0.0, 14.0 * rows * (double)cols, st);
  split_kernel<double><<<tile_grid(rows, cols), dim3(CT, CR), 0, st>>>(
      src, lds, rows, cols, trans, dst.at(0, r0, c0), dst.at(1, r0, c0), dst.at(2, r0, c0), dst.ld);
  note_launch();
  RUTV_CK(cudaGetLastError());
  return 0;
}

int merge_f32(const Planes& src, int64_t r0, int64_t c0, int64_t rows, int64_t cols, int trans,
              float* dst, int64_t ldd, cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return 0;
  ProfScope prof(K_CONVERT, 0.0, 10.0 * rows * (double)cols, st);
  merge_kernel<float><<<tile_grid(rows, cols), dim3(CT, CR), 0, st>>>(
      src.at(0, r0, c0), src.at(1, r0, c0), src.at(2, r0, c0), src.ld, rows, cols, trans, dst, ldd);
  note_launch();
  RUTV_CK(cudaGetLastError());
  return 0;
}

int merge_f64(const Planes& src, int64_t r0, int64_t c0, int64_t rows, int64_t cols, int trans,
              double* dst, int64_t ldd, cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return 0;
  ProfScope prof(K_CONVERT, 0.0, 14.0 * rows * (double)cols, st);
  merge_kernel<double><<<tile_grid(rows, cols), dim3(CT, CR), 0, st>>>(
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
  absmax_kernel<<<col_grid(rows, cols), 256, 0, st>>>(src, lds, rows, cols, amax);
  scale_bf16_kernel<<<col_grid(rows, cols), 256, 0, st>>>(src, lds, rows, cols, amax, dst, ldd);
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

// ------------------------------------------- final re-orthogonalisation
//
// For X with X^T X = I + E, E small and symmetric, the Cholesky factor of
// I + E is I + Phi(E) + O(E^2), with Phi(E) the strictly upper triangle of E
// plus half its diagonal, so X (I - Phi(E)) is orthogonal to O(E^2).  The
// diagonal of E is taken here in FP64 from the FP32 entries of X (the
// products are exact in FP64); the tensor-core Gram supplies the rest.

namespace {

// d[i] = sum_r X(r, i)^2 - 1 in FP64, one warp per column.
__global__ void colnorm_minus_one_kernel(const float* __restrict__ X, int64_t ldx, int64_t rows,
                                         int64_t cols, double* __restrict__ d) {
  const int warp = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  const int nwarps = (int)((gridDim.x * (int64_t)blockDim.x) >> 5);
  for (int64_t j = warp; j < cols; j += nwarps) {
    double s = 0.0;
    for (int64_t r = lane; r < rows; r += 32) {
      const double x = (double)X[r + j * ldx];
      s = fma(x, x, s);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) d[j] = s - 1.0;
  }
}

// Phi (n x n, BF16, ld ldp) from E (FP32, ld lde; only entries on or above
// the diagonal are read) and d; PhiT = Phi^T when non-null.  32 x 32 tiles,
// transposed through shared memory so that both writes are coalesced.
__global__ void phi_kernel(const float* __restrict__ E, int64_t lde, const double* __restrict__ d,
                           int64_t n, __nv_bfloat16* __restrict__ Phi, int64_t ldp,
                           __nv_bfloat16* __restrict__ PhiT, int64_t ldpt) {
  __shared__ float tile[32][33];
  const int64_t i0 = (int64_t)blockIdx.x * 32, j0 = (int64_t)blockIdx.y * 32;
  for (int jj = threadIdx.y; jj < 32; jj += blockDim.y) {
    const int64_t i = i0 + threadIdx.x, j = j0 + jj;
    float v = 0.f;
    if (i < n && j < n) {
      if (i < j) v = E[i + j * lde];
      else if (i == j) v = (float)(0.5 * d[i]);
      Phi[i + j * ldp] = __float2bfloat16_rn(v);
    }
    tile[jj][threadIdx.x] = v;
  }
  if (!PhiT) return;  // uniform over the block
  __syncthreads();
  for (int ii = threadIdx.y; ii < 32; ii += blockDim.y) {
    const int64_t j = j0 + threadIdx.x, i = i0 + ii;  // PhiT(j, i) = Phi(i, j)
    if (i < n && j < n) PhiT[j + i * ldpt] = __float2bfloat16_rn(tile[threadIdx.x][ii]);
  }
}

// Zeroes the off-diagonal entries of every diagonal block of T (blocks of b
// along the first p = min(m, n) columns, the last one narrower).
__global__ void zero_block_offdiag_kernel(float* T, int64_t ld, int64_t p, int64_t b) {
  const int64_t total = p * b;  // (row offset inside the block, column) pairs
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / b, io = e % b;  // column j, row k + io of its block
    const int64_t k = (j / b) * b;
    const int64_t i = k + io;
    if (i < p && i != j) T[i + j * ld] = 0.f;
  }
}

}  // namespace

int reorth_phi(const float* X, int64_t ldx, int64_t n, const float* E, int64_t lde, double* d,
               __nv_bfloat16* Phi, int64_t ldp, __nv_bfloat16* PhiT, int64_t ldpt,
               cudaStream_t st) {
  if (n <= 0) return 0;
  ProfScope prof(K_OTHER, 2.0 * (double)n * n, 4.0 * (double)n * n + 6.0 * (double)n * n, st);
  int64_t blocks = (n * 32 + 255) / 256;
  const int64_t cap = (int64_t)dev_info().sms * 16;
  if (blocks > cap) blocks = cap;
  colnorm_minus_one_kernel<<<(unsigned)blocks, 256, 0, st>>>(X, ldx, n, n, d);
  const dim3 grid((unsigned)((n + 31) / 32), (unsigned)((n + 31) / 32));
  phi_kernel<<<grid, dim3(32, 8), 0, st>>>(E, lde, d, n, Phi, ldp, PhiT, ldpt);
  note_launch(2);
  RUTV_CK(cudaGetLastError());
  return 0;
}

int zero_block_offdiag(float* T, int64_t ld, int64_t p, int64_t b, cudaStream_t st) {
  if (p <= 0 || b <= 1) return 0;
  zero_block_offdiag_kernel<<<grid_of(p * b), 256, 0, st>>>(T, ld, p, b);
  note_launch();
  RUTV_CK(cudaGetLastError());
  return 0;
}

}  // namespace rutv
