// HQRRP: blocked column-pivoted QR, A P = Q R, with the pivots of each block
// chosen on a Gaussian sketch (§2.1-2.2).  Block step i (offset k, width
// bi = min(b, n - k), rm = m - k, rn = n - k), all FP64 on the device:
//   Omega = sketch(seed, i, stream 6)            rm x bi       philox_normal
//   Y = Omega^T R(k:, k:)                        bi x rn       dgemm
//   bi steps of column-pivoted QR of Y -> swaps  (j <-> p_j)   cpqr_* kernels
//   R(:, k:) and P(k:) permuted by the swaps, in order         swap kernel
//   [W, tau] = QR(R(k:, k:k+bi)) in place; S = wy(W, tau)      householder, wy
//   R(k:, k+bi:) -= (W S^T) (R(k:, k+bi:)^T W)^T  (applies Q^T) dgemm
//   Q(:, k:) -= (Q(:, k:) W) (W S^T)^T                         dgemm
// The sketch is drawn anew at each step, as in the paper's implementation.
//
// The column-pivoted QR of Y runs as two launches per pivot step, so that
// the launch boundary is the only synchronization (no grid-wide waits):
//   * cpqr_pivot_kernel (one CTA): the column of largest remaining norm
//     (largest value, then lowest position: a lexicographic maximum, so the
//     choice does not depend on the order of the partial results), its swap
//     to position j, and its Householder reflector (LAPACK's convention);
//   * cpqr_update_kernel (one warp per column): the reflector applied to the
//     columns right of j, and their norms over the rows below j for the next
//     pivot, reduced to one (value, position) per CTA.
#include <algorithm>
#include <cstdint>

#include "common.cuh"
#include "kernels.h"

namespace rutv {
namespace {

constexpr int CP_WARPS = 8;
constexpr uint32_t kHqrrpStream = 6;

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// (v1, c1) beats (v2, c2): larger value, then lower position
__device__ __forceinline__ bool better(double v1, int64_t c1, double v2, int64_t c2) {
  return v1 > v2 || (v1 == v2 && c1 < c2);
}

// apply != 0: the reflector of step j (v_j = 1, v_i = Y(i, j) below, tau in
// hh[0]) to columns j+1 .. rn-1, then their norms^2 over rows j+1 ..
// apply == 0: the norms^2 of columns j .. rn-1 over rows j .. (first step).
__global__ void __launch_bounds__(CP_WARPS * 32)
cpqr_update_kernel(int bi, int64_t rn, double* __restrict__ Y, int j, int apply,
                   const double* __restrict__ hh, double* best_val, int64_t* best_col) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t c0 = apply ? j + 1 : j;
  const int rn0 = apply ? j + 1 : j;
  const double tau = apply ? hh[0] : 0.0;
  const double* v = Y + (int64_t)j * bi;
  double bv = -1.0;
  int64_t bc = INT64_MAX;
  for (int64_t c = c0 + (int64_t)blockIdx.x * CP_WARPS + warp; c < rn;
       c += (int64_t)gridDim.x * CP_WARPS) {
    double* y = Y + c * bi;
    if (tau != 0.0) {
      double w = 0.0;
      for (int i = j + lane; i < bi; i += 32) w = fma(i == j ? 1.0 : v[i], y[i], w);
      w = warp_sum(w) * tau;
      for (int i = j + lane; i < bi; i += 32) y[i] = fma(-(i == j ? 1.0 : v[i]), w, y[i]);
    }
    double s = 0.0;
    for (int i = rn0 + lane; i < bi; i += 32) s = fma(y[i], y[i], s);
    s = warp_sum(s);
    if (better(s, c, bv, bc)) {
      bv = s;
      bc = c;
    }
  }
  __shared__ double sv[CP_WARPS];
  __shared__ int64_t sc[CP_WARPS];
  if (lane == 0) {
    sv[warp] = bv;
    sc[warp] = bc;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double v0 = sv[0];
    int64_t k0 = sc[0];
    for (int w = 1; w < CP_WARPS; ++w)
      if (better(sv[w], sc[w], v0, k0)) {
        v0 = sv[w];
        k0 = sc[w];
      }
    best_val[blockIdx.x] = v0;
    best_col[blockIdx.x] = k0;
  }
}

// Pivot of step j from the nparts partial results; swap to position j;
// Householder reflector of Y(j:bi, j): Y(j, j) = beta, Y(i, j) = v_i below,
// hh[0] = tau.
__global__ void __launch_bounds__(256)
cpqr_pivot_kernel(int bi, double* __restrict__ Y, int j, int nparts,
                  const double* __restrict__ best_val, const int64_t* __restrict__ best_col,
                  int* swaps, double* hh) {
  __shared__ double rv[256];
  __shared__ int64_t rc[256];
  __shared__ double rs[256];
  __shared__ double s_scale;
  const int t = threadIdx.x;
  double bv = -1.0;
  int64_t bc = INT64_MAX;
  for (int i = t; i < nparts; i += blockDim.x)
    if (better(best_val[i], best_col[i], bv, bc)) {
      bv = best_val[i];
      bc = best_col[i];
    }
  rv[t] = bv;
  rc[t] = bc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (t < o && better(rv[t + o], rc[t + o], rv[t], rc[t])) {
      rv[t] = rv[t + o];
      rc[t] = rc[t + o];
    }
    __syncthreads();
  }
  const int64_t p = (rc[0] == INT64_MAX) ? j : rc[0];
  if (t == 0) swaps[j] = (int)p;
  if (p != j)
    for (int i = t; i < bi; i += blockDim.x) {
      const double a = Y[i + (int64_t)j * bi];
      Y[i + (int64_t)j * bi] = Y[i + p * bi];
      Y[i + p * bi] = a;
    }
  __syncthreads();
  double* x = Y + (int64_t)j * bi;
  double s = 0.0;
  for (int i = j + 1 + t; i < bi; i += blockDim.x) s = fma(x[i], x[i], s);
  rs[t] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (t < o) rs[t] += rs[t + o];
    __syncthreads();
  }
  if (t == 0) {
    const double ss = rs[0], alpha = x[j];
    double tau = 0.0, beta = alpha, scale = 0.0;
    if (ss != 0.0) {
      const double nrm = sqrt(fma(alpha, alpha, ss));
      beta = (alpha >= 0.0) ? -nrm : nrm;
      tau = (beta - alpha) / beta;
      scale = 1.0 / (alpha - beta);
    }
    hh[0] = tau;
    s_scale = scale;
    x[j] = beta;
  }
  __syncthreads();
  const double scale = s_scale;
  for (int i = j + 1 + t; i < bi; i += blockDim.x) x[i] *= scale;
}

// R(r, k + j) <-> R(r, k + swaps[j]) for j = 0 .. bi-1 in order, every row r;
// the first thread applies the same swaps to perm(k:).
__global__ void swap_columns_kernel(int64_t m, int bi, double* R, int64_t ldr,
                                    const int* __restrict__ swaps, int64_t* perm) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r < m) {
    for (int j = 0; j < bi; ++j) {
      const int p = swaps[j];
      if (p != j) {
        const double a = R[r + (int64_t)j * ldr];
        R[r + (int64_t)j * ldr] = R[r + (int64_t)p * ldr];
        R[r + (int64_t)p * ldr] = a;
      }
    }
  }
  if (r == 0 && perm)
    for (int j = 0; j < bi; ++j) {
      const int p = swaps[j];
      if (p != j) {
        const int64_t a = perm[j];
        perm[j] = perm[p];
        perm[p] = a;
      }
    }
}

__global__ void iota_kernel(int64_t n, int64_t* perm) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    perm[i] = i;
}

__global__ void eye_kernel(int64_t m, double* Q) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m * m;
       e += (int64_t)gridDim.x * blockDim.x)
    Q[e] = (e % m == e / m) ? 1.0 : 0.0;
}

__global__ void hq_check_finite_kernel(int64_t rows, int64_t cols, const double* X, int64_t ld,
                                       unsigned* err) {
  int bad = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < rows * cols;
       e += (int64_t)gridDim.x * blockDim.x)
    bad |= !isfinite(X[(e % rows) + (e / rows) * ld]);
  if (__syncthreads_or(bad) && threadIdx.x == 0) {
    if (atomicCAS(err, 0u, (unsigned)RANDUTV_ENONFINITE) == 0u) atomicExch(err + 1, 102u);
  }
}

int grid_cap(int64_t work, int per) {
  const int64_t cap = (int64_t)dev_info().sms * 8;
  return (int)std::max<int64_t>(1, std::min<int64_t>((work + per - 1) / per, cap));
}

struct Hq {
  double *Om, *Y, *W, *WS, *X, *Gm, *S, *tau, *hh, *best_val, *gemm;
  int64_t* best_col;
  int* swaps;
  char* qr;
  size_t gemm_bytes;
  int nparts_cap;
};

size_t hq_bytes(int64_t m, int64_t n, int64_t b, int nparts) {
  const size_t big = (size_t)std::max(m, n) * (size_t)b * 8, small = (size_t)b * (size_t)b * 8;
  size_t s = 0;
  auto add = [&](size_t x) { s += (x + 255) & ~size_t(255); };
  add(big);                  // Omega
  add((size_t)b * n * 8);    // Y
  add(big);                  // W
  add(big);                  // WS
  add(big);                  // X
  add(small);                // Gm
  add(small);                // S
  add((size_t)b * 8);        // tau
  add(64);                   // hh
  add((size_t)nparts * 8);   // best_val
  add((size_t)nparts * 8);   // best_col
  add((size_t)b * 4);        // swaps
  add(householder_scratch_bytes(b));
  add(dgemm_scratch_bytes(std::max(m, n), b));
  return s + 4096;
}

}  // namespace
}  // namespace rutv

using namespace rutv;

extern "C" {

int randutv_hqrrp(int64_t m, int64_t n, const double* A, int64_t lda, int b, uint64_t seed,
                  double* Q, double* R, int64_t* perm, void* stream) {
  if (m < 1) return -1;
  if (n < 1 || n > m) return -2;
  if (!A) return -3;
  if (lda < m) return -4;
  if (b < 1 || b > 256) return -5;
  if (!R) return -8;
  if (R == A && lda != m) return -8;
  if (!perm) return -9;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t bb = std::min<int64_t>(b, n);
  const int nparts = grid_cap(n, CP_WARPS);
  Arena ar;
  RUTV_TRY(scratch_reserve(hq_bytes(m, n, bb, nparts), &ar));
  unsigned* status = nullptr;
  RUTV_TRY(status_words(&status));
  RUTV_CK(cudaMemsetAsync(status, 0, 64 * sizeof(unsigned), st));
  Hq h;
  const size_t big = (size_t)std::max(m, n) * (size_t)bb * 8, small = (size_t)bb * (size_t)bb * 8;
  h.Om = (double*)ar.take(big);
  h.Y = (double*)ar.take((size_t)bb * n * 8);
  h.W = (double*)ar.take(big);
  h.WS = (double*)ar.take(big);
  h.X = (double*)ar.take(big);
  h.Gm = (double*)ar.take(small);
  h.S = (double*)ar.take(small);
  h.tau = (double*)ar.take((size_t)bb * 8);
  h.hh = (double*)ar.take(64);
  h.best_val = (double*)ar.take((size_t)nparts * 8);
  h.best_col = (int64_t*)ar.take((size_t)nparts * 8);
  h.swaps = (int*)ar.take((size_t)bb * 4);
  h.qr = (char*)ar.take(householder_scratch_bytes(bb));
  h.gemm_bytes = dgemm_scratch_bytes(std::max(m, n), bb);
  h.gemm = (double*)ar.take(h.gemm_bytes);
  auto gemm = [&](bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha, const double* Am,
                  int64_t la, const double* Bm, int64_t lb, double beta, double* C, int64_t lc) {
    return launch_dgemm(ta, tb, M, N, K, alpha, Am, la, Bm, lb, beta, C, lc, h.gemm, h.gemm_bytes, st);
  };

  hq_check_finite_kernel<<<grid_cap(m * n, 256), 256, 0, st>>>(m, n, A, lda, status);
  note_launch();
  RUTV_CK(cudaGetLastError());
  if (R != A)
    RUTV_CK(cudaMemcpy2DAsync(R, (size_t)m * 8, A, (size_t)lda * 8, (size_t)m * 8, (size_t)n,
                              cudaMemcpyDeviceToDevice, st));
  iota_kernel<<<grid_cap(n, 256), 256, 0, st>>>(n, perm);
  note_launch();
  if (Q) {
    eye_kernel<<<grid_cap(m * m, 256), 256, 0, st>>>(m, Q);
    note_launch();
  }
  RUTV_CK(cudaGetLastError());

  int step = 0;
  for (int64_t k = 0; k < n; k += bb, ++step) {
    const int64_t bi = std::min<int64_t>(bb, n - k), rm = m - k, rn = n - k;
    double* R22 = R + k + k * m;
    // sketch and its column-pivoted QR
    RUTV_TRY(launch_philox_normal(seed, (uint32_t)step, 0u, kHqrrpStream, rm, bi, h.Om, rm, st));
    RUTV_TRY(gemm(true, false, bi, rn, rm, 1.0, h.Om, rm, R22, m, 0.0, h.Y, bi));
    const int parts = grid_cap(rn, CP_WARPS);
    {
      ProfScope prof(K_OTHER, 4.0 * (double)bi * bi * rn, 8.0 * (double)bi * rn * 2 * bi, st);
      cpqr_update_kernel<<<parts, CP_WARPS * 32, 0, st>>>((int)bi, rn, h.Y, 0, 0, h.hh, h.best_val,
                                                          h.best_col);
      note_launch();
      for (int j = 0; j < (int)bi; ++j) {
        cpqr_pivot_kernel<<<1, 256, 0, st>>>((int)bi, h.Y, j, parts, h.best_val, h.best_col,
                                             h.swaps, h.hh);
        cpqr_update_kernel<<<parts, CP_WARPS * 32, 0, st>>>((int)bi, rn, h.Y, j, 1, h.hh,
                                                            h.best_val, h.best_col);
        note_launch(2);
      }
      RUTV_CK(cudaGetLastError());
    }
    swap_columns_kernel<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(m, (int)bi, R + k * m, m,
                                                                      h.swaps, perm + k);
    note_launch();
    RUTV_CK(cudaGetLastError());
    // unpivoted QR of the chosen columns, and the products with its Q
    RUTV_TRY(launch_householder_qr(rm, bi, R22, m, h.W, h.tau, h.qr, status + 2, status, st));
    RUTV_TRY(gemm(true, false, bi, bi, rm, 1.0, h.W, rm, h.W, rm, 0.0, h.Gm, bi));
    RUTV_TRY(launch_wy_factor(bi, h.Gm, h.tau, h.S, st));
    RUTV_TRY(gemm(false, true, rm, bi, bi, 1.0, h.W, rm, h.S, bi, 0.0, h.WS, rm));
    if (rn > bi) {
      double* R2 = R22 + bi * m;
      const int64_t nc = rn - bi;
      RUTV_TRY(gemm(true, false, nc, bi, rm, 1.0, R2, m, h.W, rm, 0.0, h.X, nc));
      RUTV_TRY(gemm(false, true, rm, nc, bi, -1.0, h.WS, rm, h.X, nc, 1.0, R2, m));
    }
    if (Q) {
      double* Qk = Q + k * m;
      RUTV_TRY(gemm(false, false, m, bi, rm, 1.0, Qk, m, h.W, rm, 0.0, h.X, m));
      RUTV_TRY(gemm(false, true, m, rm, bi, -1.0, h.X, m, h.WS, rm, 1.0, Qk, m));
    }
  }
  return 0;
}

}  // extern "C"
