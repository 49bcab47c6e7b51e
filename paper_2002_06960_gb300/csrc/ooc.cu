// Out-of-HBM randUTV (§3.2: the factorization of matrices too large for the
// memory that computes on them).  T (in place of A), U and V stay in host
// memory; every pass of a block step over a trailing region streams that
// region through HBM in panels.  One pass reads each panel once, computes on
// it with the FP64 kernels of the in-HBM path, and (for an update) writes it
// back.  Three device buffers rotate between a host-to-device copy stream,
// the compute stream (the caller's) and a device-to-host copy stream, so the
// copy of panel i+1 and the write-back of panel i-1 overlap the arithmetic
// on panel i.
//
// The steps and their order are those of the in-HBM driver (§3.1 steps 1-6,
// Fig. 2): sketch and power products by column panels of T22; the products
// from the right (T Q_V, V Q_V, U Q_U) in two passes over column panels
// (Xw = sum of P W, then P -= Xw (W S^T)^T: whole columns are what the host
// link copies fastest); the panel QR on the column block; the left update of
// T by column panels (column-local); the small SVD; its folds by panels of
// the strips they touch.  Sums over panels (Z = T22 Y) run in
// panel order, so results are deterministic for a given budget; they differ
// from the in-HBM path (and between budgets) only in rounding, since the
// panel cut changes the summation order of some products.
#include <algorithm>
#include <cstring>

#include "common.cuh"
#include "kernels.h"

namespace rutv {
namespace {

constexpr int kBufs = 3;

__global__ void ooc_check_finite_kernel(int64_t rows, int64_t cols, const double* X, int64_t ld,
                                        unsigned* err) {
  const int64_t total = rows * cols;
  int bad = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x)
    bad |= !isfinite(X[(e % rows) + (e / rows) * ld]);
  if (__syncthreads_or(bad) && threadIdx.x == 0) {
    if (atomicCAS(err, 0u, (unsigned)RANDUTV_ENONFINITE) == 0u) atomicExch(err + 1, 101u);
  }
}

// X (bi x bi, ld ld) = diag(D)
__global__ void ooc_diag_kernel(int64_t bi, const double* D, double* X, int64_t ld) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < bi * bi;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % bi, j = e / bi;
    X[i + j * ld] = (i == j) ? D[i] : 0.0;
  }
}

int grid_of(int64_t total) {
  int64_t g = (total + 255) / 256;
  const int64_t cap = (int64_t)dev_info().sms * 8;
  return (int)std::max<int64_t>(1, std::min(g, cap));
}

struct Ooc {
  int64_t m, n, lda;
  int b, q;
  uint64_t seed;
  double *T, *U, *V;  // host
  // device
  double *G, *Y, *Z, *W, *WS, *X, *tau, *D, *Gm, *S, *Us, *Vs, *blk;
  char *qr, *svd;
  double* gemm;
  size_t gemm_bytes;
  double* gemm2;  // dgemm scratch of the SVD on the side stream
  size_t gemm2_bytes;
  SideStream* side = nullptr;
  bool fold_pending = false;  // SVD of block (fold_k, fold_bi) launched, folds not yet applied
  int64_t fold_k = 0, fold_bi = 0;
  double* buf[kBufs];
  int64_t cap;  // elements per buffer
  unsigned* status;
  cudaStream_t cs, h2d, d2h;
  cudaEvent_t loaded[kBufs], computed[kBufs], freed[kBufs], join;
  cudaEvent_t stored[3];  // last write-back into host T, U, V
  int slot = 0;
  double bytes_moved = 0.0;
};

size_t fixed_bytes(int64_t m, int64_t n, int64_t b) {
  const size_t big = (size_t)std::max(m, n) * (size_t)b * sizeof(double);
  const size_t small = (size_t)b * (size_t)b * sizeof(double);
  size_t s = 0;
  auto add = [&](size_t x) { s += (x + 255) & ~size_t(255); };
  for (int i = 0; i < 6; ++i) add(big);                 // G, Y, Z, W, WS, X
  add((size_t)b * 8);                                   // tau
  add((size_t)b * 8);                                   // D
  for (int i = 0; i < 5; ++i) add(small);               // Gm, S, Us, Vs, blk
  add(householder_scratch_bytes(b));
  add(small_svd_scratch_bytes((int)b));
  add(dgemm_scratch_bytes(std::max(m, n), b));
  add(dgemm_scratch_bytes(b, b));
  return s + 4096;
}

int gemm(Ooc& o, bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha, const double* A,
         int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc) {
  return launch_dgemm(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, o.gemm, o.gemm_bytes,
                      o.cs);
}

// Panel length along the cut dimension: as many rows (or columns) of length
// `other` as a buffer holds, at most `limit`, rounded down to a multiple of
// 64 when that leaves at least 64.
int64_t panel_len(const Ooc& o, int64_t other, int64_t limit) {
  int64_t len = o.cap / std::max<int64_t>(1, other);
  if (len >= 128) len = len / 64 * 64;
  return std::max<int64_t>(1, std::min(len, limit));
}

enum HostMat { MAT_T = 0, MAT_U = 1, MAT_V = 2 };

// Streams the rows x cols region of host matrix `mat` (leading dimension
// ldh) through the device buffers, cut into row panels (by_rows) or column
// panels of `len`.  fn(P, ldp, r0, c0, pr, pc) computes on the panel (device,
// ld pr) whose first element is region(r0, c0); with `write` the panel is
// copied back.  The loads of a pass wait for the last write-back into the
// same host matrix; passes over different matrices overlap.
template <class F>
int stream_panels(Ooc& o, int mat, double* host, int64_t ldh, int64_t rows, int64_t cols,
                  bool by_rows, int64_t len, bool write, F&& fn) {
  if (rows <= 0 || cols <= 0) return 0;
  RUTV_CK(cudaStreamWaitEvent(o.h2d, o.stored[mat], 0));
  const int64_t total = by_rows ? rows : cols;
  for (int64_t s0 = 0; s0 < total; s0 += len) {
    const int64_t l = std::min(len, total - s0);
    const int64_t pr = by_rows ? l : rows, pc = by_rows ? cols : l;
    const int64_t r0 = by_rows ? s0 : 0, c0 = by_rows ? 0 : s0;
    const int i = o.slot;
    o.slot = (o.slot + 1) % kBufs;
    double* d = o.buf[i];
    double* h = host + r0 + c0 * ldh;
    RUTV_CK(cudaStreamWaitEvent(o.h2d, o.freed[i], 0));
    RUTV_CK(cudaMemcpy2DAsync(d, (size_t)pr * 8, h, (size_t)ldh * 8, (size_t)pr * 8, (size_t)pc,
                              cudaMemcpyHostToDevice, o.h2d));
    RUTV_CK(cudaEventRecord(o.loaded[i], o.h2d));
    RUTV_CK(cudaStreamWaitEvent(o.cs, o.loaded[i], 0));
    RUTV_TRY(fn(d, pr, r0, c0, pr, pc));
    RUTV_CK(cudaEventRecord(o.computed[i], o.cs));
    o.bytes_moved += 8.0 * (double)pr * (double)pc * (write ? 2.0 : 1.0);
    if (write) {
      RUTV_CK(cudaStreamWaitEvent(o.d2h, o.computed[i], 0));
      RUTV_CK(cudaMemcpy2DAsync(h, (size_t)ldh * 8, d, (size_t)pr * 8, (size_t)pr * 8, (size_t)pc,
                                cudaMemcpyDeviceToHost, o.d2h));
      RUTV_CK(cudaEventRecord(o.freed[i], o.d2h));
    } else {
      RUTV_CK(cudaEventRecord(o.freed[i], o.cs));
    }
  }
  if (write) RUTV_CK(cudaEventRecord(o.stored[mat], o.d2h));
  return 0;
}

// W (r x bi) and tau -> S (bi x bi), then WS = W S^T (r x bi).
int wy_ws(Ooc& o, int64_t r, int64_t bi) {
  RUTV_TRY(gemm(o, true, false, bi, bi, r, 1.0, o.W, r, o.W, r, 0.0, o.Gm, bi));
  RUTV_TRY(launch_wy_factor(bi, o.Gm, o.tau, o.S, o.cs));
  RUTV_TRY(gemm(o, false, true, r, bi, bi, 1.0, o.W, r, o.S, bi, 0.0, o.WS, r));
  return 0;
}

// host region X(rows, 0:r) (ld ldx) <- X - (X W) (W S^T)^T.  The product is
// row-local, but row panels of a column-major host matrix copy as short
// strided pieces, several times slower over the host link than whole
// columns.  So it goes in two passes over column panels: Xw = sum over
// panels of X(:, cols) W(cols, :) (read only), then X(:, cols) -= Xw WS(cols, :)^T.
int right_apply(Ooc& o, int mat, double* X, int64_t ldx, int64_t rows, int64_t r, int64_t bi) {
  const int64_t cw = panel_len(o, rows, r);
  RUTV_TRY(stream_panels(o, mat, X, ldx, rows, r, false, cw, false,
                         [&](double* P, int64_t ldp, int64_t, int64_t c0, int64_t, int64_t pc) {
                           return gemm(o, false, false, rows, bi, pc, 1.0, P, ldp, o.W + c0, r,
                                       c0 == 0 ? 0.0 : 1.0, o.X, rows);
                         }));
  return stream_panels(o, mat, X, ldx, rows, r, false, cw, true,
                       [&](double* P, int64_t ldp, int64_t, int64_t c0, int64_t, int64_t pc) {
                         return gemm(o, false, true, rows, pc, bi, -1.0, o.X, rows, o.WS + c0, r,
                                     1.0, P, ldp);
                       });
}

// Waits for the side stream's SVD of block (fold_k, fold_bi) and applies its
// folds on the compute stream: T(0:k, blk) Vs, Us^T T(blk, k+bi:), V(:, blk)
// Vs, U(:, blk) Us and T(blk, blk) = diag(D).  Of all later passes only the
// products from the right of T read what these write (rows blk of T), so
// the next step calls this before its first such pass; its sketch passes and
// QR run beside the SVD.
int flush_folds(Ooc& o) {
  if (!o.fold_pending) return 0;
  o.fold_pending = false;
  RUTV_CK(cudaStreamWaitEvent(o.cs, o.side->svd, 0));
  const int64_t m = o.m, n = o.n, lda = o.lda, k = o.fold_k, bi = o.fold_bi, rn = n - k;
  double* T22 = o.T + k + k * lda;
  // strips of bi columns (T(0:k, blk), V(:, blk), U(:, blk)): P <- P F, as
  // one panel of whole columns (rows x bi fits a buffer)
  auto fold_cols = [&](int mat, double* X, int64_t ldx, int64_t rows, const double* F) {
    return stream_panels(o, mat, X, ldx, rows, bi, false, bi, true,
                         [&](double* P, int64_t ldp, int64_t, int64_t, int64_t pr, int64_t) {
                           RUTV_TRY(gemm(o, false, false, pr, bi, bi, 1.0, P, ldp, F, bi, 0.0, o.X, pr));
                           RUTV_CK(cudaMemcpy2DAsync(P, (size_t)ldp * 8, o.X, (size_t)pr * 8,
                                                     (size_t)pr * 8, (size_t)bi,
                                                     cudaMemcpyDeviceToDevice, o.cs));
                           return 0;
                         });
  };
  if (k > 0) RUTV_TRY(fold_cols(MAT_T, o.T + k * lda, lda, k, o.Vs));
  if (rn > bi) {  // T(blk, k+bi:) <- Us^T T(blk, k+bi:), by column panels
    const int64_t nc = rn - bi;
    const int64_t big = std::max(m, n);
    RUTV_TRY(stream_panels(o, MAT_T, T22 + bi * lda, lda, bi, nc, false, panel_len(o, bi, std::min(nc, big)),
                           true, [&](double* P, int64_t ldp, int64_t, int64_t, int64_t, int64_t pc) {
                             RUTV_TRY(gemm(o, true, false, bi, pc, bi, 1.0, o.Us, bi, P, ldp, 0.0,
                                           o.X, bi));
                             RUTV_CK(cudaMemcpy2DAsync(P, (size_t)ldp * 8, o.X, (size_t)bi * 8,
                                                       (size_t)bi * 8, (size_t)pc,
                                                       cudaMemcpyDeviceToDevice, o.cs));
                             return 0;
                           }));
  }
  if (o.V) RUTV_TRY(fold_cols(MAT_V, o.V + k * n, n, n, o.Vs));
  if (o.U) RUTV_TRY(fold_cols(MAT_U, o.U + k * m, m, m, o.Us));
  // T(blk, blk) = diag(D)
  RUTV_TRY(stream_panels(o, MAT_T, T22, lda, bi, bi, false, bi, true,
                         [&](double* P, int64_t ldp, int64_t, int64_t, int64_t, int64_t) {
                           ooc_diag_kernel<<<grid_of(bi * bi), 256, 0, o.cs>>>(bi, o.D, P, ldp);
                           note_launch();
                           RUTV_CK(cudaGetLastError());
                           return 0;
                         }));
  return 0;
}

int ooc_step(Ooc& o, int step, int64_t k, int64_t bi) {
  const int64_t m = o.m, n = o.n, lda = o.lda, rm = m - k, rn = n - k;
  double* T22 = o.T + k + k * lda;
  // ---- right transform
  if (rn > bi) {
    RUTV_TRY(launch_philox_normal(o.seed, (uint32_t)step, 0u, 0u, rm, bi, o.G, rm, o.cs));
    const int64_t cw = panel_len(o, rm, rn);
    // Y = T22^T G
    RUTV_TRY(stream_panels(o, MAT_T, T22, lda, rm, rn, false, cw, false,
                           [&](double* P, int64_t ldp, int64_t, int64_t c0, int64_t, int64_t pc) {
                             return gemm(o, true, false, pc, bi, rm, 1.0, P, ldp, o.G, rm, 0.0,
                                         o.Y + c0, rn);
                           }));
    for (int it = 0; it < o.q; ++it) {
      // Z = T22 Y, summed over the column panels in order
      RUTV_TRY(stream_panels(o, MAT_T, T22, lda, rm, rn, false, cw, false,
                             [&](double* P, int64_t ldp, int64_t, int64_t c0, int64_t, int64_t pc) {
                               return gemm(o, false, false, rm, bi, pc, 1.0, P, ldp, o.Y + c0, rn,
                                           c0 == 0 ? 0.0 : 1.0, o.Z, rm);
                             }));
      RUTV_TRY(stream_panels(o, MAT_T, T22, lda, rm, rn, false, cw, false,
                             [&](double* P, int64_t ldp, int64_t, int64_t c0, int64_t, int64_t pc) {
                               return gemm(o, true, false, pc, bi, rm, 1.0, P, ldp, o.Z, rm, 0.0,
                                           o.Y + c0, rn);
                             }));
    }
    // the previous block's SVD may still hold SMs: leave them to it
    RUTV_TRY(launch_householder_qr(rn, bi, o.Y, rn, o.W, o.tau, o.qr, o.status + 2, o.status,
                                   o.cs, o.fold_pending ? kSvdSms : 0));
    RUTV_TRY(wy_ws(o, rn, bi));
    RUTV_TRY(flush_folds(o));
    RUTV_TRY(right_apply(o, MAT_T, o.T + k * lda, lda, m, rn, bi));
    if (o.V) RUTV_TRY(right_apply(o, MAT_V, o.V + k * n, n, n, rn, bi));
  }
  // ---- left transform (the panel QR also leaves the diagonal block in blk)
  RUTV_TRY(flush_folds(o));
  if (rm > bi) {
    RUTV_TRY(stream_panels(o, MAT_T, T22, lda, rm, bi, false, bi, true,
                           [&](double* P, int64_t ldp, int64_t, int64_t, int64_t, int64_t) {
                             RUTV_TRY(launch_householder_qr(rm, bi, P, ldp, o.W, o.tau, o.qr,
                                                            o.status + 2, o.status, o.cs));
                             RUTV_CK(cudaMemcpy2DAsync(o.blk, (size_t)bi * 8, P, (size_t)ldp * 8,
                                                       (size_t)bi * 8, (size_t)bi,
                                                       cudaMemcpyDeviceToDevice, o.cs));
                             return 0;
                           }));
    RUTV_TRY(wy_ws(o, rm, bi));
    if (rn > bi) {
      const int64_t nc = rn - bi;
      RUTV_TRY(stream_panels(o, MAT_T, T22 + bi * lda, lda, rm, nc, false, panel_len(o, rm, nc), true,
                             [&](double* P, int64_t ldp, int64_t, int64_t, int64_t, int64_t pc) {
                               RUTV_TRY(gemm(o, true, false, pc, bi, rm, 1.0, P, ldp, o.W, rm, 0.0,
                                             o.X, pc));
                               return gemm(o, false, true, rm, pc, bi, -1.0, o.WS, rm, o.X, pc, 1.0,
                                           P, ldp);
                             }));
    }
    if (o.U) RUTV_TRY(right_apply(o, MAT_U, o.U + k * m, m, m, rm, bi));
  } else {
    RUTV_TRY(stream_panels(o, MAT_T, T22, lda, bi, bi, false, bi, false,
                           [&](double* P, int64_t ldp, int64_t, int64_t, int64_t, int64_t) {
                             RUTV_CK(cudaMemcpy2DAsync(o.blk, (size_t)bi * 8, P, (size_t)ldp * 8,
                                                       (size_t)bi * 8, (size_t)bi,
                                                       cudaMemcpyDeviceToDevice, o.cs));
                             return 0;
                           }));
  }
  // ---- small SVD of the diagonal block, on the side stream: it runs beside
  // the next step's sketch passes and QR; its folds wait for flush_folds
  RUTV_TRY(flush_folds(o));
  RUTV_CK(cudaEventRecord(o.side->panel, o.cs));
  RUTV_CK(cudaStreamWaitEvent(o.side->st, o.side->panel, 0));
  RUTV_TRY(launch_small_svd((int)bi, o.blk, bi, o.D, o.Us, o.Vs, o.status + 8, o.svd, o.gemm2,
                            o.gemm2_bytes, o.side->st));
  RUTV_CK(cudaEventRecord(o.side->svd, o.side->st));
  o.fold_pending = true;
  o.fold_k = k;
  o.fold_bi = bi;
  return 0;
}

struct OocStreams {
  cudaStream_t h2d = nullptr, d2h = nullptr;
  cudaEvent_t ev[3 * kBufs + 4] = {};
  bool ok = false;
};
OocStreams g_ooc[64];

int ooc_streams(OocStreams** out) {
  int dev = 0;
  RUTV_CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return RANDUTV_EUNSUPPORTED;
  OocStreams& s = g_ooc[dev];
  if (!s.ok) {
    RUTV_CK(cudaStreamCreateWithFlags(&s.h2d, cudaStreamNonBlocking));
    RUTV_CK(cudaStreamCreateWithFlags(&s.d2h, cudaStreamNonBlocking));
    for (auto& e : s.ev) RUTV_CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    s.ok = true;
  }
  *out = &s;
  return 0;
}

}  // namespace
}  // namespace rutv

using namespace rutv;

extern "C" {

size_t randutv_ooc_min_device_bytes(int64_t m, int64_t n, int b) {
  if (m < 1 || n < 1 || b < 1) return 0;
  const int64_t p = m < n ? m : n;
  const int64_t bb = b < p ? b : p;
  return fixed_bytes(m, n, bb) + (size_t)kBufs * (size_t)std::max(m, n) * (size_t)bb * 8 + 4096;
}

int randutv_factor_ooc(int64_t m, int64_t n, double* A, int64_t lda, int b, int q, uint64_t seed,
                       double* U, double* V, size_t device_bytes, double* bytes_moved,
                       void* stream) {
  if (m < 1) return -1;
  if (n < 1) return -2;
  if (!A) return -3;
  if (lda < m) return -4;
  if (b < 1 || b > 256) return -5;
  if (q < 0 || q > 16) return -6;
  const size_t need = randutv_ooc_min_device_bytes(m, n, b);
  if (device_bytes < need) return -10;
  const int64_t p = m < n ? m : n;
  const int64_t bb = b < p ? b : p;
  OocStreams* os = nullptr;
  RUTV_TRY(ooc_streams(&os));
  const size_t fixed = fixed_bytes(m, n, bb);
  const int64_t cap = (int64_t)((device_bytes - fixed - 4096) / kBufs / 8);
  Arena ar;
  RUTV_TRY(scratch_reserve(fixed + (size_t)kBufs * (size_t)cap * 8 + 8192, &ar));
  Ooc o;
  o.m = m;
  o.n = n;
  o.lda = lda;
  o.b = (int)bb;
  o.q = q;
  o.seed = seed;
  o.T = A;
  o.U = U;
  o.V = V;
  const size_t big = (size_t)std::max(m, n) * (size_t)bb * 8, small = (size_t)bb * (size_t)bb * 8;
  o.G = (double*)ar.take(big);
  o.Y = (double*)ar.take(big);
  o.Z = (double*)ar.take(big);
  o.W = (double*)ar.take(big);
  o.WS = (double*)ar.take(big);
  o.X = (double*)ar.take(big);
  o.tau = (double*)ar.take((size_t)bb * 8);
  o.D = (double*)ar.take((size_t)bb * 8);
  o.Gm = (double*)ar.take(small);
  o.S = (double*)ar.take(small);
  o.Us = (double*)ar.take(small);
  o.Vs = (double*)ar.take(small);
  o.blk = (double*)ar.take(small);
  o.qr = (char*)ar.take(householder_scratch_bytes(bb));
  o.svd = (char*)ar.take(small_svd_scratch_bytes((int)bb));
  o.gemm_bytes = dgemm_scratch_bytes(std::max(m, n), bb);
  o.gemm = (double*)ar.take(o.gemm_bytes);
  o.gemm2_bytes = dgemm_scratch_bytes(bb, bb);
  o.gemm2 = (double*)ar.take(o.gemm2_bytes);
  for (int i = 0; i < kBufs; ++i) o.buf[i] = (double*)ar.take((size_t)cap * 8);
  RUTV_TRY(side_stream(&o.side));
  o.cap = cap;
  RUTV_TRY(status_words(&o.status));
  o.cs = (cudaStream_t)stream;
  o.h2d = os->h2d;
  o.d2h = os->d2h;
  for (int i = 0; i < kBufs; ++i) {
    o.loaded[i] = os->ev[i];
    o.computed[i] = os->ev[kBufs + i];
    o.freed[i] = os->ev[2 * kBufs + i];
  }
  o.join = os->ev[3 * kBufs];
  for (int i = 0; i < 3; ++i) o.stored[i] = os->ev[3 * kBufs + 1 + i];
  RUTV_CK(cudaMemsetAsync(o.status, 0, 64 * sizeof(unsigned), o.cs));
  // every copy stream starts after the work already queued on the caller's stream
  RUTV_CK(cudaEventRecord(o.join, o.cs));
  RUTV_CK(cudaStreamWaitEvent(o.h2d, o.join, 0));
  RUTV_CK(cudaStreamWaitEvent(o.d2h, o.join, 0));
  for (int i = 0; i < kBufs; ++i) RUTV_CK(cudaEventRecord(o.freed[i], o.cs));
  for (int i = 0; i < 3; ++i) RUTV_CK(cudaEventRecord(o.stored[i], o.cs));
  // U = I, V = I on the host
  if (U)
    for (int64_t j = 0; j < m; ++j) {
      std::memset(U + j * m, 0, (size_t)m * 8);
      U[j + j * m] = 1.0;
    }
  if (V)
    for (int64_t j = 0; j < n; ++j) {
      std::memset(V + j * n, 0, (size_t)n * 8);
      V[j + j * n] = 1.0;
    }
  RUTV_TRY(stream_panels(o, MAT_T, A, lda, m, n, false, panel_len(o, m, n), false,
                         [&](double* P, int64_t ldp, int64_t, int64_t, int64_t pr, int64_t pc) {
                           ooc_check_finite_kernel<<<grid_of(pr * pc), 256, 0, o.cs>>>(pr, pc, P, ldp,
                                                                                       o.status);
                           note_launch();
                           RUTV_CK(cudaGetLastError());
                           return 0;
                         }));
  unsigned h = 0;
  RUTV_CK(cudaMemcpyAsync(&h, o.status, sizeof h, cudaMemcpyDeviceToHost, o.cs));
  RUTV_CK(cudaStreamSynchronize(o.cs));
  if (h != 0) return (int)h;
  int step = 0;
  for (int64_t k = 0; k < p; k += bb, ++step) {
    const int64_t bi = (bb < p - k) ? bb : p - k;
    RUTV_TRY(ooc_step(o, step, k, bi));
  }
  RUTV_TRY(flush_folds(o));
  // the caller's stream, and this call's return, follow the last write-back
  RUTV_CK(cudaEventRecord(o.join, o.d2h));
  RUTV_CK(cudaStreamWaitEvent(o.cs, o.join, 0));
  RUTV_CK(cudaStreamSynchronize(o.cs));
  if (bytes_moved) *bytes_moved = o.bytes_moved;
  RUTV_CK(cudaMemcpy(&h, o.status, sizeof h, cudaMemcpyDeviceToHost));
  return (int)h;
}

}  // extern "C"
