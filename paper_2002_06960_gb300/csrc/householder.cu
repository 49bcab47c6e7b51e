// Householder QR of a tall panel and its compact-WY factor (FP64).
//
// Fig. 2 takes an unpivoted QR twice per block step: of the sketch Y (its
// reflectors W_V form V-hat, §3.1 V-hat step 2) and of the new column panel
// [A11; A21] (reflectors W_U, §3.1 step 2), and applies each as
// I - W S W^T (S is the triangular factor the paper calls T_V / T_U).
//
// The panel has r rows (up to the matrix height) and c <= 256 columns, so
// the reflector of each column needs a reduction over all r rows.  One
// cooperative grid (one CTA per SM at most) walks the columns; each CTA owns
// a contiguous slice of rows, held in shared memory when it fits (it does for
// 16384 x 256 on 152 SMs), else read and written in place through L2.  Two
// bounded grid barriers per column separate
//   (1) the partials over own rows below the diagonal of |x|^2 and of
//       x . A(:, l) for the trailing columns l (x the column below the
//       diagonal), and row j, published by the CTA that owns it; the
//       reflector's products follow from these without knowing beta first:
//       v . A(j:, l) = A(j, l) + (x . A(j+1:, l)) / (alpha - beta);
//   (2) the reflector, identical in every CTA, and the sums of the partials:
//       the CTA k owns the trailing columns l = j + 1 + k (mod CTAs) and
//       publishes tau (v . A(j:, l));
//   (3) the rank-1 update of every CTA's rows with the published sums.
// Summing each column's partials once (2') instead of in every CTA keeps the
// traffic per column at O(CTAs * c) rather than O(CTAs^2 * c).  Every
// cross-CTA sum is taken in a fixed order, so the result is bitwise
// reproducible.  Values written by another CTA are read with L2-only loads:
// L1 is not coherent across SMs.
#include "common.cuh"

namespace rutv {

namespace {
constexpr int QR_THREADS = 256;
constexpr int QR_WARPS = QR_THREADS / 32;
constexpr size_t kQrSmemMax = 216 * 1024;  // own rows kept in shared memory up to this size
constexpr int kOwnMax = 37;  // owned columns per warp: ceil(255 / 7) with one CTA, c <= 256
constexpr int kQrMaxCols = 256;   // panel columns
constexpr int kLoadsPerLane = 8;  // partials per lane: CTAs <= 256

// Real: element type of the panel and of its per-element arithmetic (the
// library instantiates double); the cross-CTA partials, tau and the
// reflector scalars are FP64.
template <typename Real>
struct QrArgsT {
  int64_t r, c;
  Real* A;
  int64_t lda;
  Real* W;         // r x c, ld r
  double* tau;     // c
  double* part1;   // nblocks: partial squared norms below the diagonal
  double* part2;   // nblocks x c: partial dot products
  double* tot;     // c: tau * (v . A(:, l)) of the trailing columns (one writer per column)
  double* rowj;    // c: row j of the panel, published by the CTA that owns it
  unsigned* bar;   // {count, generation}
  unsigned* err;
};
using QrArgs = QrArgsT<double>;

template <typename Real, bool kSmem>
__global__ void __launch_bounds__(QR_THREADS) householder_panel_kernel(QrArgsT<Real> a) {
  extern __shared__ __align__(16) unsigned char qr_smem[];
  // kSmem: own rows, column-major with an odd leading dimension ldr (so that
  // a warp's threads, one per column, hit distinct banks), then one column
  // more for the reflector v over own rows
  Real* smA = reinterpret_cast<Real*>(qr_smem);
  __shared__ double red[QR_WARPS];
  __shared__ double s_coef[4];  // tau, scale, beta
  // owned columns' (sum of partials, A(j, l)) per warp 1..: at most
  // ceil((c - 1) / ((QR_WARPS - 1) nb)) each (checked on the host)
  __shared__ double s_own[QR_WARPS - 1][kOwnMax][2];
  __shared__ double s_tot[kQrMaxCols];  // tau (v . A(:, l)) of column j's trailing columns
  const unsigned nb = gridDim.x;
  const int64_t rows_per = (a.r + nb - 1) / nb;
  const int64_t i0 = (int64_t)blockIdx.x * rows_per;
  const int64_t i1 = (i0 + rows_per < a.r) ? i0 + rows_per : a.r;
  const int64_t nr = (i1 > i0) ? i1 - i0 : 0;
  const int64_t ldr = rows_per | 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned epoch = 0;  // grid barriers passed (thread 0)
  // element (i, l) of the panel, i in [i0, i1)
  auto at = [&](int64_t i, int64_t l) -> Real& {
    if (kSmem) return smA[(i - i0) + l * ldr];
    return a.A[i + l * a.lda];
  };
  if (kSmem) {
    for (int64_t l = 0; l < a.c; ++l)
      for (int64_t i = i0 + threadIdx.x; i < i1; i += QR_THREADS) at(i, l) = a.A[i + l * a.lda];
    __syncthreads();
  }

  // W starts as zero above the diagonal; column j is written in step 3 of j.
  for (int64_t j = 0; j < a.c; ++j) {
    // ---- (1) over own rows below the diagonal, x = A(j+1:r, j): the partial
    // |x|^2 and the partial products x . A(j+1:r, l) for the trailing columns
    // l > j.  With v = (1, x / (alpha - beta)) the reflector's products are
    // v . A(j:r, l) = A(j, l) + (x . A(j+1:r, l)) / (alpha - beta), so these
    // partials and the row A(j, j:c) are all the exchange the column needs.
    const int64_t lo = (i0 > j + 1) ? i0 : j + 1;
    if constexpr (kSmem) {
      // thread t < c takes column t: x . A(own rows, t), and |x|^2 for t = j,
      // each a fixed-order sum of its own (no cross-lane reduction)
      const int t = threadIdx.x;
      if (t >= j && t < a.c) {
        const Real* __restrict__ xj = smA + j * ldr;
        const Real* __restrict__ xt = smA + (int64_t)t * ldr;
        Real d0 = 0, d1 = 0;
        int64_t lr = lo - i0;
        for (; lr + 1 < nr; lr += 2) {
          d0 = fma(xj[lr], xt[lr], d0);
          d1 = fma(xj[lr + 1], xt[lr + 1], d1);
        }
        if (lr < nr) d0 = fma(xj[lr], xt[lr], d0);
        const double d = (double)(d0 + d1);
        if (t == j) a.part1[blockIdx.x] = d;
        else a.part2[(int64_t)blockIdx.x * a.c + t] = d;
      }
      if (j >= i0 && j < i1)
        for (int64_t l = j + t; l < a.c; l += QR_THREADS) a.rowj[l] = (double)at(j, l);
    } else {
      Real ss = 0;
      for (int64_t i = lo + threadIdx.x; i < i1; i += QR_THREADS) {
        const Real x = at(i, j);
        ss = fma(x, x, ss);
      }
      // Each warp takes its columns l = j+1+warp+QR_WARPS*t in groups of 8 and
      // walks its rows once per group, so the loads of a row are independent
      // and in flight together.
      for (int64_t l0 = j + 1 + warp; l0 < a.c; l0 += 8 * (int64_t)QR_WARPS) {
        Real d[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) d[t] = 0;
        for (int64_t i = lo + lane; i < i1; i += 32) {
          const Real x = at(i, j);
#pragma unroll
          for (int t = 0; t < 8; ++t) {
            const int64_t l = l0 + (int64_t)t * QR_WARPS;
            if (l < a.c) d[t] = fma(x, at(i, l), d[t]);
          }
        }
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          double y = (double)d[t];
          for (int o = 16; o > 0; o >>= 1) y += __shfl_xor_sync(0xffffffffu, y, o);
          const int64_t l = l0 + (int64_t)t * QR_WARPS;
          if (lane == 0 && l < a.c) a.part2[(int64_t)blockIdx.x * a.c + l] = y;
        }
      }
      // the CTA that owns row j publishes it
      if (j >= i0 && j < i1)
        for (int64_t l = j + threadIdx.x; l < a.c; l += QR_THREADS) a.rowj[l] = (double)at(j, l);
      const double ssum = block_sum((double)ss, red);
      if (threadIdx.x == 0) a.part1[blockIdx.x] = ssum;
    }
    if (!grid_barrier(a.bar, nb, a.err, 1, epoch)) return;

    // ---- (2) reflector scalars (every CTA, same order), and the sums of the
    // partials of the columns this CTA owns: l = j + 1 + k (mod CTAs).  Warp 0
    // reduces |x|^2 while warps 1.. load and sum the owned columns' partials
    // (they do not depend on the reflector), so the two L2 round trips overlap.
    if (warp == 0) {
      // lanes load the partials in parallel, all in flight at once, and add
      // them in a fixed order; the fixed shuffle tree makes the sum identical
      // in every CTA
      double v[kLoadsPerLane];
#pragma unroll
      for (int q = 0; q < kLoadsPerLane; ++q) {
        const unsigned t = lane + 32u * q;
        v[q] = (t < nb) ? __ldcg(a.part1 + t) : 0.0;
      }
      const double alpha = __ldcg(a.rowj + j);
      double sig2 = 0.0;
#pragma unroll
      for (int q = 0; q < kLoadsPerLane; ++q) sig2 += v[q];
      for (int o = 16; o > 0; o >>= 1) sig2 += __shfl_xor_sync(0xffffffffu, sig2, o);
      if (lane == 0) {
        double tau, scale, beta;
        if (sig2 == 0.0) {
          tau = 0.0; beta = alpha; scale = 0.0;
        } else {
          const double nrm = sqrt(fma(alpha, alpha, sig2));
          beta = (alpha >= 0.0) ? -nrm : nrm;
          tau = (beta - alpha) / beta;
          scale = 1.0 / (alpha - beta);
        }
        s_coef[0] = tau; s_coef[1] = scale; s_coef[2] = beta;
      }
    }
    else {
      int t = 0;
      for (int64_t l = j + 1 + blockIdx.x + (int64_t)nb * (warp - 1); l < a.c;
           l += (int64_t)nb * (QR_WARPS - 1), ++t) {
        double v[kLoadsPerLane];
#pragma unroll
        for (int q = 0; q < kLoadsPerLane; ++q) {
          const unsigned u = lane + 32u * q;
          v[q] = (u < nb) ? __ldcg(a.part2 + (int64_t)u * a.c + l) : 0.0;
        }
        double sp = 0.0;
#pragma unroll
        for (int q = 0; q < kLoadsPerLane; ++q) sp += v[q];
        for (int o = 16; o > 0; o >>= 1) sp += __shfl_xor_sync(0xffffffffu, sp, o);
        if (lane == 0) {
          s_own[warp - 1][t][0] = sp;
          s_own[warp - 1][t][1] = __ldcg(a.rowj + l);
        }
      }
    }
    __syncthreads();
    const double tau = s_coef[0], scale = s_coef[1];
    const Real scale_r = (Real)scale;
    if (warp > 0 && lane == 0) {
      int t = 0;
      for (int64_t l = j + 1 + blockIdx.x + (int64_t)nb * (warp - 1); l < a.c;
           l += (int64_t)nb * (QR_WARPS - 1), ++t)
        a.tot[l] = tau * fma(s_own[warp - 1][t][0], scale, s_own[warp - 1][t][1]);
    }
    if (!grid_barrier(a.bar, nb, a.err, 2, epoch)) return;

    // ---- (3) rank-1 update of own rows, write W(:, j), R(j, j), zeros; the
    // published tau (v . A(:, l)) come into shared memory in one round trip
    const int64_t lo3 = (i0 > j) ? i0 : j;
    if constexpr (kSmem) {
      // v over own rows into shared memory, then thread t > j updates column t
      if (tau != 0.0) {
        const int t = threadIdx.x;
        Real w = 0;
        if (t > j && t < a.c) w = (Real)__ldcg(a.tot + t);
        Real* __restrict__ sv = smA + a.c * ldr;
        for (int64_t lr = lo3 - i0 + t; lr < nr; lr += QR_THREADS)
          sv[lr] = (i0 + lr == j) ? (Real)1 : smA[lr + j * ldr] * scale_r;
        __syncthreads();
        if (t > j && t < a.c) {
          Real* __restrict__ xt = smA + (int64_t)t * ldr;
          const Real* __restrict__ svc = sv;
#pragma unroll 4
          for (int64_t lr = lo3 - i0; lr < nr; ++lr) xt[lr] = fma(-svc[lr], w, xt[lr]);
        }
      }
    } else {
      if (tau != 0.0) {
        for (int64_t l = j + 1 + threadIdx.x; l < a.c; l += QR_THREADS) s_tot[l] = __ldcg(a.tot + l);
        __syncthreads();
        for (int64_t l0 = j + 1 + warp; l0 < a.c; l0 += 8 * (int64_t)QR_WARPS) {
          Real w[8];
#pragma unroll
          for (int t = 0; t < 8; ++t) {
            const int64_t l = l0 + (int64_t)t * QR_WARPS;
            w[t] = (l < a.c) ? (Real)s_tot[l] : (Real)0;
          }
          for (int64_t i = lo3 + lane; i < i1; i += 32) {
            const Real v = (i == j) ? (Real)1 : at(i, j) * scale_r;
#pragma unroll
            for (int t = 0; t < 8; ++t) {
              const int64_t l = l0 + (int64_t)t * QR_WARPS;
              if (l < a.c) at(i, l) = fma(-v, w[t], at(i, l));
            }
          }
        }
      }
    }
    __syncthreads();  // the updates above read A(:, j); rewrite it only now
    for (int64_t i = i0 + threadIdx.x; i < i1; i += QR_THREADS) {
      Real wv;
      if (i < j) wv = 0;
      else if (i == j) wv = 1;
      else wv = (tau != 0.0) ? at(i, j) * scale_r : (Real)0;
      a.W[i + j * a.r] = wv;
      if (i > j) at(i, j) = 0;
      if (i == j) at(i, j) = (Real)s_coef[2];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) a.tau[j] = tau;
    __syncthreads();
  }
  if (kSmem) {
    for (int64_t l = 0; l < a.c; ++l)
      for (int64_t i = i0 + threadIdx.x; i < i1; i += QR_THREADS) a.A[i + l * a.lda] = at(i, l);
  }
}

// Number of CTAs of the panel kernel: at least 16 rows each, at most one per SM
// not reserved.  Every column's FP64 work divides over the CTAs (an SM issues
// only two DFMA per clock), so short panels, such as the tiles of the
// by-blocks form, gain from many CTAs of a few rows.
int qr_blocks(int64_t r, int reserve_sms = 0) {
  int sms = dev_info().sms - reserve_sms;
  if (sms < 1) sms = 1;
  int nb = (int)((r + 15) / 16);
  if (nb > sms) nb = sms;
  if (nb < 1) nb = 1;
  return nb;
}

// Scratch layout: part1 (SMs + 1), part2 (SMs x c), tot (c), rowj (c), in doubles.
template <typename Real>
void qr_carve(QrArgsT<Real>& a, double* base, int sms) {
  a.part1 = base;
  a.part2 = a.part1 + sms + 1;
  a.tot = a.part2 + (size_t)sms * a.c;
  a.rowj = a.tot + a.c;
}

template <typename Real>
int qr_launch(QrArgsT<Real>& a, int nb, cudaStream_t st) {
  if (a.c > kQrMaxCols || nb > 32 * kLoadsPerLane ||
      a.c - 1 > (int64_t)(QR_WARPS - 1) * nb * kOwnMax)
    return RANDUTV_EUNSUPPORTED;
  const int64_t rows_per = (a.r + nb - 1) / nb;
  // own rows (leading dimension rows_per | 1) and the reflector column
  const size_t smem = (size_t)(rows_per | 1) * (size_t)(a.c + 1) * sizeof(Real);
  void* args[] = {&a};
  if (smem <= kQrSmemMax) {
    const void* fn = (const void*)householder_panel_kernel<Real, true>;
    RUTV_TRY(ensure_smem(fn, kQrSmemMax));
    RUTV_CK(cudaLaunchCooperativeKernel(fn, dim3(nb), dim3(QR_THREADS), args, smem, st));
  } else {
    RUTV_CK(cudaLaunchCooperativeKernel((const void*)householder_panel_kernel<Real, false>,
                                        dim3(nb), dim3(QR_THREADS), args, 0, st));
  }
  note_launch();
  return 0;
}

// S (c x c, ld c) from the Gram matrix Gm = W^T W (c x c, ld ldg) and tau, the
// compact-WY factor of H_1 ... H_c = I - W S W^T (forward, column-wise):
// S_jj = tau_j, S(0:j, j) = -tau_j S(0:j, 0:j) Gm(0:j, j).
// That recurrence is the inverse of the upper triangle striu(Gm) + diag(1/tau)
// (for tau_j != 0), so every column of S is a back substitution of its own:
//   S(i, k) = tau_i (delta_ik - sum_{l=i+1..k} Gm(i, l) S(l, k)),  i = k..0,
// which also gives the zero rows and columns of reflectors with tau = 0.
// One warp per column k, S(:, k) in shared memory; Gm(i, l) is read as
// Gm(l, i) (Gm is symmetric) so that the lanes read contiguous memory, and
// the next row's operands are loaded while the current row is reduced.  Only
// the strictly lower part of Gm is read (the diagonal enters through tau).
constexpr int WY_WARPS = 1;   // one column per CTA: the FP64 work spreads over the SMs
constexpr int WY_MAXC = 256;

// kInverse: M = (I + D_tau striu(Gm))^-1 instead, M(i, k) = delta_ik - tau_i sum_l Gm(i, l)
// M(l, k) (S = M D_tau; M is needed apart from S where some tau is zero).
template <bool kInverse>
__global__ void __launch_bounds__(WY_WARPS * 32) wy_factor_kernel(int c, const double* __restrict__ Gm,
                                                                   int64_t ldg,
                                                                   const double* __restrict__ tau,
                                                                   double* __restrict__ S) {
  __shared__ double col[WY_WARPS][WY_MAXC];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // the longest columns (largest k) are launched first
  const int k = c - 1 - (int)(blockIdx.x * WY_WARPS + warp);
  if (k < 0) return;  // whole warps leave; no block barrier below
  double* sk = col[warp];
  constexpr int NL = WY_MAXC / 32;  // operands per lane per row
  double gcur[NL], gnext[NL];
  // operands of row i: Gm(l, i) for l = i+1+lane+32t <= k
  auto load_row = [&](int i, double* g) {
#pragma unroll
    for (int t = 0; t < NL; ++t) {
      const int l = i + 1 + lane + 32 * t;
      g[t] = (i >= 0 && l <= k) ? Gm[l + (int64_t)i * ldg] : 0.0;
    }
  };
  load_row(k, gcur);
  double tcur = tau[k];
  for (int i = k; i >= 0; --i) {
    load_row(i - 1, gnext);
    const double tnext = (i > 0) ? tau[i - 1] : 0.0;
    // groups t with a live operand (l = i+1+32t <= k): warp-uniform, so the
    // FMA slots past the column's end are skipped rather than predicated
    const int nt = (k - i + 31) >> 5;
    double acc = 0.0;
#pragma unroll
    for (int t = 0; t < NL; ++t) {
      if (t < nt) {
        const int l = i + 1 + lane + 32 * t;
        if (l <= k) acc = fma(gcur[t], sk[l], acc);
      }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
      if (kInverse) sk[i] = ((i == k) ? 1.0 : 0.0) - tcur * acc;
      else sk[i] = tcur * (((i == k) ? 1.0 : 0.0) - acc);
    }
    __syncwarp();
#pragma unroll
    for (int t = 0; t < NL; ++t) gcur[t] = gnext[t];
    tcur = tnext;
  }
  for (int i = lane; i < c; i += 32) S[i + (int64_t)k * c] = (i <= k) ? sk[i] : 0.0;
}
}  // namespace

size_t householder_scratch_bytes(int64_t c) {
  const int nb = dev_info().sms;
  return ((size_t)nb + 1 + (size_t)nb * (size_t)c + 2 * (size_t)c) * sizeof(double) + 512;
}

int launch_householder_qr(int64_t r, int64_t c, double* A, int64_t lda, double* W, double* tau,
                          char* scratch, unsigned* bar, unsigned* err, cudaStream_t st,
                          int reserve_sms) {
  if (c <= 0) return 0;
  const int nb = qr_blocks(r, reserve_sms);
  QrArgs a;
  a.r = r; a.c = c; a.A = A; a.lda = lda; a.W = W; a.tau = tau;
  qr_carve(a, (double*)scratch, dev_info().sms);
  a.bar = bar; a.err = err;
  ProfScope prof(K_QR, 2.0 * (double)c * c * ((double)r - c / 3.0), 24.0 * (double)r * c, st);
  RUTV_CK(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), st));
  return qr_launch(a, nb, st);
}

int launch_wy_factor(int64_t c, const double* Gm, const double* tau, double* S, cudaStream_t st,
                     int64_t ldg) {
  if (c <= 0) return 0;
  if (c > WY_MAXC) return RANDUTV_EUNSUPPORTED;
  if (ldg == 0) ldg = c;
  if (ldg < c) return RANDUTV_EUNSUPPORTED;
  ProfScope prof(K_WY, (double)c * c * c / 3.0, 16.0 * (double)c * c, st);
  wy_factor_kernel<false><<<(unsigned)((c + WY_WARPS - 1) / WY_WARPS), WY_WARPS * 32, 0, st>>>(
      (int)c, Gm, ldg, tau, S);
  note_launch();
  RUTV_CK(cudaGetLastError());
  return 0;
}

int launch_wy_inverse(int64_t c, const double* Gm, const double* tau, double* M, cudaStream_t st) {
  if (c <= 0) return 0;
  if (c > WY_MAXC) return RANDUTV_EUNSUPPORTED;
  ProfScope prof(K_ADJOINT, (double)c * c * c / 3.0, 16.0 * (double)c * c, st);
  wy_factor_kernel<true><<<(unsigned)((c + WY_WARPS - 1) / WY_WARPS), WY_WARPS * 32, 0, st>>>(
      (int)c, Gm, c, tau, M);
  note_launch();
  RUTV_CK(cudaGetLastError());
  return 0;
}

}  // namespace rutv

// ---------------------------------------------------------------------------
// Householder QR without any allocation.
//
// The panel QR above needs scratch in global memory: the per-CTA partial sums
// (SMs x (c + 1) doubles) and the words of its grid barrier and status.  The
// library normally takes these from its own growing scratch, which it
// allocates with cudaMalloc on first use.  This variant keeps them in one
// fixed array in the library's device image instead, sized for at most
// kNoAllocMaxSms SMs and kNoAllocMaxCols columns (about 390 KiB).  Every GPU
// that loads the library holds that array until the process exits.
#include <mutex>

namespace rutv {
namespace {

constexpr int kNoAllocMaxSms = 192;
constexpr int kNoAllocMaxCols = 256;
constexpr size_t kNoAllocPartials =
    (size_t)kNoAllocMaxSms * (1 + kNoAllocMaxCols) + 1 + 2 * kNoAllocMaxCols;
constexpr size_t kNoAllocBytes = kNoAllocPartials * sizeof(double) + 256;

// Partials first, then 64 status words: [0] error, [1] site, [2..3] barrier.
static __device__ __align__(256) unsigned char g_qr_noalloc_scratch[kNoAllocBytes];

std::mutex g_noalloc_mu;
char* g_noalloc_ptr[64] = {nullptr};

// Device address of the array on the current device; the host-side symbol
// is only a stand-in and must never reach a kernel.  Looked up once per
// device, with that device current.
int noalloc_scratch(char** out) {
  int dev = 0;
  RUTV_CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return RANDUTV_EUNSUPPORTED;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    RUTV_CK(cudaGetSymbolAddress(&p, g_qr_noalloc_scratch));
    g_noalloc_ptr[dev] = (char*)p;
  }
  *out = g_noalloc_ptr[dev];
  return 0;
}

}  // namespace
}  // namespace rutv

extern "C" int randutv_householder_qr_noalloc(int64_t r, int64_t c, double* panel, int64_t ld,
                                              double* W, double* tau, void* stream) {
  using namespace rutv;
  if (r < 1) return -1;
  if (c < 1 || c > r) return -2;
  if (!panel) return -3;
  if (ld < r) return -4;
  if (!W) return -5;
  if (!tau) return -6;
  if (c > kNoAllocMaxCols) {
    set_last_error("randutv_householder_qr_noalloc: more than 256 columns");
    return RANDUTV_EUNSUPPORTED;
  }
  const int sms = dev_info().sms;
  if (sms > kNoAllocMaxSms) {
    set_last_error("randutv_householder_qr_noalloc: device has more than 192 SMs");
    return RANDUTV_EUNSUPPORTED;
  }
  char* base = nullptr;
  RUTV_TRY(noalloc_scratch(&base));
  unsigned* words = (unsigned*)(base + kNoAllocPartials * sizeof(double));
  cudaStream_t st = (cudaStream_t)stream;
  // error, site and barrier words start at zero; the partials are always
  // written before they are read
  RUTV_CK(cudaMemsetAsync(words, 0, 4 * sizeof(unsigned), st));
  const int nb = qr_blocks(r);
  QrArgs a;
  a.r = r; a.c = c; a.A = panel; a.lda = ld; a.W = W; a.tau = tau;
  qr_carve(a, (double*)base, sms);
  a.bar = words + 2;
  a.err = words;
  RUTV_TRY(qr_launch(a, nb, st));
  unsigned h[2] = {0, 0};
  RUTV_CK(cudaMemcpyAsync(h, words, sizeof h, cudaMemcpyDeviceToHost, st));
  RUTV_CK(cudaStreamSynchronize(st));
  return (int)h[0];
}
