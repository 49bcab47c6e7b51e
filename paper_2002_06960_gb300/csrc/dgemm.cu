// FP64 matrix products of the randUTV step: C = alpha op(A) op(B) + beta C.
//
// On GB300 the FP64 rate is about 1.2 TFLOP/s for both DFMA and the FP64
// mma.sync path (DFMA measured slightly faster), i.e. two DFMA per clock per
// SM, so every FP64 product of the method -- the sketch and power products
// (§3.1, V-hat step 2), the compact-WY applications of Fig. 2 and the
// fold-back of the small SVD -- is bound by DFMA issue, not by memory.  The
// kernel therefore aims at keeping every SM's DFMA pipe busy: 64 x 64 output
// tiles, 4 x 4 accumulators per thread (16 independent chains), operands
// staged through shared memory, and a deterministic split-K (partials summed
// in a fixed order) when the output has too few tiles to cover the SMs.
#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace rutv {

namespace {
constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

template <bool TA, bool TB>
__global__ void __launch_bounds__(NT)
dgemm_kernel(int64_t M, int64_t N, int64_t K, int64_t kchunk, double alpha,
             const double* __restrict__ A, int64_t lda, const double* __restrict__ B, int64_t ldb,
             double beta, double* __restrict__ C, int64_t ldc, double* __restrict__ P, bool lower) {
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int64_t m0 = (int64_t)blockIdx.x * BM, n0 = (int64_t)blockIdx.y * BN;
  if (lower && n0 >= m0 + BM) return;  // tile wholly above the diagonal: not wanted
  const int64_t kb = (int64_t)blockIdx.z * kchunk;
  const int64_t ke = (kb + kchunk < K) ? kb + kchunk : K;

  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  double ra[4], rb[4];
  auto load = [&](int64_t k0) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      int64_t m, k;
      if (!TA) { m = m0 + (tid & 63); k = k0 + (tid >> 6) + 4 * i; }
      else     { k = k0 + (tid & 15); m = m0 + (tid >> 4) + 16 * i; }
      ra[i] = (m < M && k < ke) ? (TA ? A[k + m * lda] : A[m + k * lda]) : 0.0;
      int64_t n, kk;
      if (!TB) { kk = k0 + (tid & 15); n = n0 + (tid >> 4) + 16 * i; }
      else     { n = n0 + (tid & 63); kk = k0 + (tid >> 6) + 4 * i; }
      rb[i] = (n < N && kk < ke) ? (TB ? B[n + kk * ldb] : B[kk + n * ldb]) : 0.0;
    }
  };
  auto store = [&]() {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (!TA) As[(tid >> 6) + 4 * i][tid & 63] = ra[i];
      else     As[tid & 15][(tid >> 4) + 16 * i] = ra[i];
      if (!TB) Bs[tid & 15][(tid >> 4) + 16 * i] = rb[i];
      else     Bs[(tid >> 6) + 4 * i][tid & 63] = rb[i];
    }
  };

  if (kb < ke) {
    load(kb);
    store();
    __syncthreads();
    for (int64_t k0 = kb; k0 < ke; k0 += BK) {
      const bool more = k0 + BK < ke;
      if (more) load(k0 + BK);
#pragma unroll
      for (int k = 0; k < BK; ++k) {
        double a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = As[k][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) b[j] = Bs[k][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
      }
      __syncthreads();
      if (more) {
        store();
        __syncthreads();
      }
    }
  }

#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t m = m0 + ty + 16 * i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t n = n0 + tx + 16 * j;
      if (n >= N) continue;
      if (P) {
        P[(int64_t)blockIdx.z * M * N + m + n * M] = acc[i][j];
      } else {
        double v = alpha * acc[i][j];
        if (beta != 0.0) v = fma(beta, C[m + n * ldc], v);
        C[m + n * ldc] = v;
      }
    }
  }
}

// C = alpha * sum_z P[z] + beta * C, summed in the order z = 0, 1, ...
// (lower: only the elements of the tiles the product computed).
__global__ void splitk_reduce_kernel(int64_t M, int64_t N, int splits, double alpha,
                                     const double* __restrict__ P, double beta,
                                     double* __restrict__ C, int64_t ldc, bool lower) {
  const int64_t MN = M * N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < MN;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t m = e % M, n = e / M;
    if (lower && (n / BN) * BN >= (m / BM) * BM + BM) continue;
    double s = 0.0;
    for (int z = 0; z < splits; ++z) s += P[z * MN + e];
    double v = alpha * s;
    if (beta != 0.0) v = fma(beta, C[m + n * ldc], v);
    C[m + n * ldc] = v;
  }
}
}  // namespace

// Scratch the split-K path may use for an M x N product: room for up to 16
// partial products of the largest skinny output (M x N with N <= 256), at
// least 64 MiB.
size_t dgemm_scratch_bytes(int64_t M, int64_t N) {
  size_t want = (size_t)16 * (size_t)M * (size_t)N * sizeof(double);
  const size_t lo = (size_t)64 << 20, hi = (size_t)1 << 30;
  return want < lo ? lo : (want > hi ? hi : want);
}

// Number of K splits for an M x N x K product.  Tiles are handed to SMs as
// they free up and every SM's DFMA pipe is shared by its resident CTAs, so
// the time of a launch follows the largest per-SM tile count: the balance of
// u work units over S SMs is (u/S) / ceil(u/S).  Pick the split count with
// the best balance (fewest splits among equals) that keeps >= 128 of K per
// split and fits the scratch.
static int choose_splits(int64_t tiles, int64_t M, int64_t N, int64_t K, int sms,
                         size_t scratch_bytes) {
  if (K < 256 || tiles >= 64 * (int64_t)sms) return 1;
  const int64_t cap = (int64_t)(scratch_bytes / (sizeof(double) * (size_t)(M * N)));
  int64_t smax = K / 128;
  if (smax > cap) smax = cap;
  if (smax > 64) smax = 64;
  int best = 1;
  double best_bal = 0.0;
  for (int64_t s = 1; s <= smax; ++s) {
    const double u = (double)(tiles * s) / sms;
    const double bal = u / std::ceil(u);
    if (bal > best_bal + 0.02) {
      best_bal = bal;
      best = (int)s;
    }
    if (best_bal > 0.97) break;
  }
  return best;
}

int launch_dgemm(bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha,
                 const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
                 double* C, int64_t ldc, double* scratch, size_t scratch_bytes, cudaStream_t st,
                 bool lower) {
  if (M <= 0 || N <= 0) return 0;
  const int64_t tm = (M + BM - 1) / BM, tn = (N + BN - 1) / BN;
  // tiles computed (lower: those that meet or lie below the diagonal) and their elements
  int64_t tiles = tm * tn;
  double elems = (double)M * (double)N;
  if (lower) {
    tiles = 0;
    elems = 0.0;
    for (int64_t i = 0; i < tm; ++i) {
      const int64_t rows = std::min<int64_t>(BM, M - i * BM);
      for (int64_t j = 0; j < tn && j * BN < i * BM + BM; ++j) {
        ++tiles;
        elems += (double)rows * (double)std::min<int64_t>(BN, N - j * BN);
      }
    }
  }
  const int sms = dev_info().sms;
  int splits = scratch ? choose_splits(tiles, M, N, K, sms, scratch_bytes) : 1;
  int64_t kchunk = K;
  if (splits > 1) {
    kchunk = (K + splits - 1) / splits;
    kchunk = (kchunk + BK - 1) / BK * BK;
    splits = (int)((K + kchunk - 1) / kchunk);
  }
  if (K <= 0) kchunk = 0;
  ProfScope prof(K_DGEMM, 2.0 * elems * (double)K,
                 8.0 * ((double)M * K + (double)K * N + elems * (beta != 0.0 ? 2 : 1)), st);
  dim3 grid((unsigned)tm, (unsigned)tn, (unsigned)splits);
  double* P = splits > 1 ? scratch : nullptr;
#define RUTV_DG(TA_, TB_) \
  dgemm_kernel<TA_, TB_><<<grid, NT, 0, st>>>(M, N, K, kchunk, alpha, A, lda, B, ldb, beta, C, ldc, P, lower)
  if (!ta && !tb) RUTV_DG(false, false);
  else if (!ta && tb) RUTV_DG(false, true);
  else if (ta && !tb) RUTV_DG(true, false);
  else RUTV_DG(true, true);
#undef RUTV_DG
  note_launch();
  RUTV_CK(cudaGetLastError());
  if (splits > 1) {
    int64_t n = M * N;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 8 * sms) blocks = 8 * sms;
    splitk_reduce_kernel<<<(unsigned)blocks, 256, 0, st>>>(M, N, splits, alpha, P, beta, C, ldc,
                                                            lower);
    note_launch();
    RUTV_CK(cudaGetLastError());
  }
  return 0;
}

}  // namespace rutv
