// Mixed-precision randUTV (the same block step as the FP64 path, §3.1 and
// Fig. 2, with different arithmetic):
//   * T, U^T and V^T are held as three BF16 planes each (FP32-level storage);
//     U and V are kept transposed so that every update of them contracts
//     over their row index, which is the K-major operand layout of the MMA.
//   * Sketch and power products Y = T22^T G, Z = T22 Y: one BF16 product on
//     tcgen05 (plane 0 of T is the BF16 shadow of T22), FP32 accumulation,
//     with Y and Z rescaled by exact powers of two between products.
//   * Every compact-WY update and the fold-back of the small SVD: the six-
//     product BF16 split on tcgen05, FP32 accuracy, FP32 accumulation.
//   * Householder vectors and norms (the panel QRs), the WY factor S and the
//     b x b SVD: FP64, the same kernels as the FP64 path.
//   * After the last step, one re-orthogonalisation pass of U and V (their
//     Gram's diagonal in FP64, a first-order Cholesky correction), with T
//     corrected alongside so that U T V^T and the shape of T are kept.
#include <cuda_bf16.h>

#include <utility>
#include <vector>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"
#include "mixed.h"

namespace rutv {

namespace {

__global__ void f32_to_f64_kernel(const float* __restrict__ src, int64_t lds, int64_t rows,
                                  int64_t cols, double* __restrict__ dst, int64_t ldd) {
  const int64_t total = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % rows, j = e / rows;
    dst[i + j * ldd] = (double)src[i + j * lds];
  }
}

// P(i, j) -= D(i, j) for an FP64 P and an FP32 D (rows x cols), columns by grid.y.
__global__ void sub_f32_from_f64_kernel(double* __restrict__ P, int64_t ldp,
                                        const float* __restrict__ D, int64_t ldd, int64_t rows,
                                        int64_t cols) {
  for (int64_t j = blockIdx.y; j < cols; j += gridDim.y)
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows;
         i += (int64_t)gridDim.x * blockDim.x)
      P[i + j * ldp] -= (double)D[i + j * ldd];
}

// tau_j <- 2 / Gm(j, j) for the reflectors that are not the identity (tau_j = 0).
__global__ void retau_kernel(int c, const double* __restrict__ Gm, int64_t ldg,
                             double* __restrict__ tau) {
  for (int j = threadIdx.x; j < c; j += blockDim.x)
    if (tau[j] != 0.0) tau[j] = 2.0 / Gm[j + (int64_t)j * ldg];
}

int grid_of(int64_t total) {
  int64_t blocks = (total + 255) / 256;
  const int64_t cap = (int64_t)dev_info().sms * 16;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  return (int)blocks;
}

int f32_to_f64(const float* src, int64_t lds, int64_t rows, int64_t cols, double* dst, int64_t ldd,
               cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return 0;
  f32_to_f64_kernel<<<grid_of(rows * cols), 256, 0, st>>>(src, lds, rows, cols, dst, ldd);
  note_launch();
  RUTV_CK(cudaGetLastError());
  return 0;
}

// Operand from planes; rows x cols is the extent of the valid source (a
// smaller leading block of a larger buffer), so that TMA zero-fills past it.
BgemmOperand opnd(const Planes& P, int nplanes, int64_t x0, int64_t y0, int mn_major,
                  int64_t rows = -1, int64_t cols = -1) {
  BgemmOperand o;
  for (int i = 0; i < 3; ++i) o.planes[i] = P.p[i];
  o.nplanes = nplanes;
  o.rows = rows < 0 ? P.rows : rows;
  o.cols = cols < 0 ? P.cols : cols;
  o.ld = P.ld;
  o.x0 = x0;
  o.y0 = y0;
  o.mn_major = mn_major;
  return o;
}

BgemmOperand opnd_bf16(const __nv_bfloat16* X, int64_t rows, int64_t cols, int64_t ld,
                       int mn_major) {
  BgemmOperand o;
  o.planes[0] = X;
  o.nplanes = 1;
  o.rows = rows;
  o.cols = cols;
  o.ld = ld;
  o.mn_major = mn_major;
  return o;
}

BgemmOut out_f32(float* C, int64_t ldc, float alpha = 1.f, float beta = 0.f) {
  BgemmOut o;
  o.mode = 0;
  o.C = C;
  o.ldc = ldc;
  o.alpha = alpha;
  o.beta = beta;
  return o;
}

BgemmOut out_planes(const Planes& P, int64_t r0, int64_t c0, float alpha) {
  BgemmOut o;
  o.mode = 1;
  o.alpha = alpha;
  for (int i = 0; i < 3; ++i) o.planes[i] = P.at(i, r0, c0);
  o.ldp = P.ld;
  return o;
}

struct MixedWork {
  Planes T, Ut, Vt;             // m x n, m x m (U^T), n x n (V^T)
  Planes W, WSt, Xp, Sp, Vs;     // small operands as planes
  Planes Pp;                     // blocked panel QR: the second half of the panel as planes
  Planes UsAll;                 // U_s of every block step, b x (steps b), kept for the row folds
  __nv_bfloat16 *G, *Yb;        // BF16 sketch operands
  float *Y, *Z, *X, *tmp, *scal;
  double *Y64, *W64, *tau, *Gram64, *S64, *D, *Us64, *Vs64, *blk64;
  double* W2;        // blocked panel QR: reflectors of the second half (ld r - h)
  double *qrX, *qrY; // blocked panel QR: W1^T P2 and S1^T W1^T P2
  char* qr;
  char* svd;
  double* dgemm;
  size_t dgemm_bytes;
  float* tmp2;     // side stream: fold-back products
  double* dgemm2;  // side stream: dgemm scratch
  // final re-orthogonalisation of U and V
  float* E;                    // X^T X - I (FP32, max(m,n)^2)
  __nv_bfloat16 *Phi, *PhiT;   // its first-order Cholesky correction and transpose
  double* dcol;                // FP64 diagonal of X^T X - I
};

size_t planes_bytes(int64_t rows, int64_t cols) {
  return 3 * (size_t)pad8(rows) * (size_t)cols * sizeof(__nv_bfloat16) + 3 * 256;
}

Planes carve_planes(Arena& ar, int64_t rows, int64_t cols) {
  Planes P;
  P.rows = rows;
  P.cols = cols;
  P.ld = pad8(rows);
  for (int i = 0; i < 3; ++i)
    P.p[i] = (__nv_bfloat16*)ar.take((size_t)P.ld * (size_t)cols * sizeof(__nv_bfloat16));
  return P;
}

int64_t nsteps(int64_t m, int64_t n, int64_t b) {
  const int64_t p = m < n ? m : n;
  return (p + b - 1) / b;
}

// Columns [c0, c0 + cols) of P as planes of their own (the base moves by
// c0 ld elements, a multiple of 16 bytes since ld is a multiple of 8).
Planes plane_cols(const Planes& P, int64_t c0, int64_t cols) {
  Planes V = P;
  for (int i = 0; i < 3; ++i) V.p[i] = P.p[i] + c0 * P.ld;
  V.cols = cols;
  return V;
}

size_t mixed_bytes(int64_t m, int64_t n, int64_t b) {
  const int64_t big = m > n ? m : n;
  size_t s = 0;
  auto add = [&](size_t x) { s += (x + 255) & ~size_t(255); };
  add(planes_bytes(m, n));
  add(planes_bytes(m, m));
  add(planes_bytes(n, n));
  add(planes_bytes(big, b));      // W
  add(planes_bytes(b, big));      // WSt
  add(planes_bytes(b, big));      // Xp (X^T or Xv/Xl)
  add(planes_bytes(b, b));        // Sp (S^T)
  add(planes_bytes(big, b));      // Pp
  add(planes_bytes(b, nsteps(m, n, b) * b));  // UsAll
  add(planes_bytes(b, b));        // Vs
  add((size_t)pad8(big) * b * 2); // G
  add((size_t)pad8(big) * b * 2); // Yb
  for (int i = 0; i < 4; ++i) add((size_t)big * b * 4);  // Y, Z, X, tmp
  add(256);                       // scal
  for (int i = 0; i < 3; ++i) add((size_t)big * b * 8);  // Y64, W64, W2
  for (int i = 0; i < 2; ++i) add((size_t)b * b * 8);    // qrX, qrY
  add((size_t)b * 8 * 2);         // tau, D
  for (int i = 0; i < 5; ++i) add((size_t)b * b * 8);    // Gram64, S64, Us64, Vs64, blk64
  add(householder_scratch_bytes(b));
  add(small_svd_scratch_bytes(b));
  add(dgemm_scratch_bytes(b, b));
  add((size_t)big * b * 4);          // tmp2
  add(dgemm_scratch_bytes(b, b));    // dgemm2
  add((size_t)big * big * 4);        // E
  add((size_t)pad8(big) * big * 2);  // Phi
  add((size_t)pad8(n) * n * 2);      // PhiT
  add((size_t)big * 8);              // dcol
  return s + 8192;
}

MixedWork carve_mixed(Arena& ar, int64_t m, int64_t n, int64_t b) {
  const int64_t big = m > n ? m : n;
  MixedWork w;
  w.T = carve_planes(ar, m, n);
  w.Ut = carve_planes(ar, m, m);
  w.Vt = carve_planes(ar, n, n);
  w.W = carve_planes(ar, big, b);
  w.WSt = carve_planes(ar, b, big);
  w.Xp = carve_planes(ar, b, big);
  w.Sp = carve_planes(ar, b, b);
  w.Pp = carve_planes(ar, big, b);
  w.UsAll = carve_planes(ar, b, nsteps(m, n, b) * b);
  w.Vs = carve_planes(ar, b, b);
  w.G = (__nv_bfloat16*)ar.take((size_t)pad8(big) * b * 2);
  w.Yb = (__nv_bfloat16*)ar.take((size_t)pad8(big) * b * 2);
  w.Y = (float*)ar.take((size_t)big * b * 4);
  w.Z = (float*)ar.take((size_t)big * b * 4);
  w.X = (float*)ar.take((size_t)big * b * 4);
  w.tmp = (float*)ar.take((size_t)big * b * 4);
  w.scal = (float*)ar.take(256);
  w.Y64 = (double*)ar.take((size_t)big * b * 8);
  w.W64 = (double*)ar.take((size_t)big * b * 8);
  w.W2 = (double*)ar.take((size_t)big * b * 8);
  w.qrX = (double*)ar.take((size_t)b * b * 8);
  w.qrY = (double*)ar.take((size_t)b * b * 8);
  w.tau = (double*)ar.take((size_t)b * 8);
  w.D = (double*)ar.take((size_t)b * 8);
  w.Gram64 = (double*)ar.take((size_t)b * b * 8);
  w.S64 = (double*)ar.take((size_t)b * b * 8);
  w.Us64 = (double*)ar.take((size_t)b * b * 8);
  w.Vs64 = (double*)ar.take((size_t)b * b * 8);
  w.blk64 = (double*)ar.take((size_t)b * b * 8);
  w.qr = (char*)ar.take(householder_scratch_bytes(b));
  w.svd = (char*)ar.take(small_svd_scratch_bytes(b));
  w.dgemm_bytes = dgemm_scratch_bytes(b, b);
  w.dgemm = (double*)ar.take(w.dgemm_bytes);
  w.tmp2 = (float*)ar.take((size_t)big * b * 4);
  w.dgemm2 = (double*)ar.take(w.dgemm_bytes);
  w.E = (float*)ar.take((size_t)big * big * 4);
  w.Phi = (__nv_bfloat16*)ar.take((size_t)pad8(big) * big * 2);
  w.PhiT = (__nv_bfloat16*)ar.take((size_t)pad8(n) * n * 2);
  w.dcol = (double*)ar.take((size_t)big * 8);
  return w;
}

struct MCtx {
  int64_t m, n;
  int b, q;
  uint64_t seed;
  bool want_u, want_v;
  MixedWork w;
  unsigned* status;
  cudaStream_t st;
  // The small SVD of each block and its column folds (T(0:k, blk) V_s,
  // V(:, blk) V_s, U(:, blk) U_s) run on the side stream beside the later
  // block steps.  The row fold T(blk, k+b:) <- U_s^T T(blk, k+b:) is a left
  // product on rows that no later step reads across: every later right
  // update multiplies those rows from the right, which commutes with it, and
  // every later left update, panel and sketch lies below them.  So all row
  // folds wait until after the last step and then run on the main stream,
  // and the main stream never waits for an SVD.  Once an SVD may be running,
  // the main stream's persistent kernels leave it kSvdSms SMs.
  SideStream* side = nullptr;
  bool svd_live = false;
  std::vector<std::pair<int64_t, int64_t>> folds;  // (k, bi) of each pending row fold
  int reserve() const { return svd_live ? kSvdSms : 0; }
  int cap() const { return svd_live ? dev_info().sms - kSvdSms : 0; }
};

// From the rounded reflectors (W64 = W~, r x bi, and their planes), tau and
// the lower triangle of their Gram W~^T W~ (left by mixed_qr): S (FP64), and
// WSt = (W S^T)^T as planes (bi x r).
//
// The reflectors the updates apply are the rounded W~ held in the planes.  S
// is built from W~ itself: its Gram in FP64 (over r terms; an FP32
// accumulation would be off by about sqrt(r) ulp) and tau~_j = 2 / |w~_j|^2,
// so that every H_j = I - tau~_j w~_j w~_j^T, and with them I - W~ S W~^T,
// is orthogonal to FP64 accuracy rather than to the accuracy of the rounding.
int mixed_wy(MCtx& c, int64_t r, int64_t bi) {
  MixedWork& w = c.w;
  retau_kernel<<<1, 256, 0, c.st>>>((int)bi, w.Gram64, bi, w.tau);
  note_launch();
  RUTV_CK(cudaGetLastError());
  RUTV_TRY(launch_wy_factor(bi, w.Gram64, w.tau, w.S64, c.st));
  // WS = W S^T (r x bi): A = W (MN-major), B = S^T held as planes of S^T
  RUTV_TRY(split_f64(w.S64, bi, bi, bi, 1, w.Sp, 0, 0, c.st));
  RUTV_TRY(launch_bgemm(opnd(w.W, 3, 0, 0, 1, r, bi), opnd(w.Sp, 3, 0, 0, 0, bi, bi), (int)r, (int)bi, (int)bi, 3,
                        out_f32(w.tmp, r), c.status, c.st, c.cap()));
  RUTV_TRY(split_f32(w.tmp, r, bi, r, 1, w.WSt, 0, 0, c.st));
  return 0;
}

// X <- X - (X_in W) (W S^T)^T for a transposed factor Xt (rows k: of U^T or V^T):
// Xt(k:, :) <- Xt(k:, :) - WS (W^T Xt(k:, :)).
int mixed_apply_transposed(MCtx& c, const Planes& Xt, int64_t k, int64_t r, int64_t bi) {
  MixedWork& w = c.w;
  const int64_t cols = Xt.cols;
  // Xv = W^T Xt(k:, :)   (bi x cols)
  RUTV_TRY(launch_bgemm(opnd(w.W, 3, 0, 0, 0, r, bi), opnd(Xt, 3, k, 0, 0), (int)bi, (int)cols, (int)r, 3,
                        out_f32(w.X, bi), c.status, c.st, c.cap()));
  RUTV_TRY(split_f32(w.X, bi, bi, cols, 0, w.Xp, 0, 0, c.st));
  // Xt(k:, :) -= WS Xv   (A = WS via its transpose planes, K-major)
  RUTV_TRY(launch_bgemm(opnd(w.WSt, 3, 0, 0, 0, bi, r), opnd(w.Xp, 3, 0, 0, 0, bi, cols), (int)r, (int)cols,
                        (int)bi, 3, out_planes(Xt, k, 0, -1.f), c.status, c.st, c.cap()));
  return 0;
}

// Rounds the reflectors W64(:, c0:c0+nc) to their planes (columns c0: of W)
// and writes the rounded values back, so that W64 holds W~ from here on.
int mixed_round_w(MCtx& c, int64_t r, int64_t c0, int64_t nc) {
  MixedWork& w = c.w;
  RUTV_TRY(split_f64(w.W64 + c0 * r, r, r, nc, 0, w.W, 0, c0, c.st));
  return merge_f64(w.W, 0, c0, r, nc, 0, w.W64 + c0 * r, r, c.st);
}

// Householder QR (FP64) of the panel P (r x bi, ld r) into the rounded
// reflectors W~ (W64, ld r, and the planes W), tau, and the lower triangle of
// the Gram W~^T W~ (Gram64, ld bi) that mixed_wy needs.  Panels of more than
// 128 columns are factored in two halves: the QR of the first h = 128
// columns, whose rounded block reflector I - W~1 S1 W~1^T (S1 from the
// Gram's leading block, tau~ = 2 / |w~|^2) is applied to the rest,
// P2 <- (I - W~1 S1 W~1^T)^T P2 (its long products to FP32 accuracy on the
// tensor cores, as every other update of the panel's source), then the QR of
// P2 below row h in FP64.  The
// reflectors are those of the unblocked factorization up to rounding; each
// half keeps its rows in shared memory where the whole panel would not fit,
// and its columns see at most 127 trailing columns.  The Gram is built by
// blocks: the leading block before the second half, then the blocks of the
// second half's reflectors over rows h: (above them W~2 is zero), and only
// the tiles on or below the diagonal of the symmetric blocks.
int mixed_qr(MCtx& c, int64_t r, int64_t bi, double* P, int reserve) {
  MixedWork& w = c.w;
  constexpr int64_t h = 128;
  if (bi <= h || r - h < bi - h) {
    RUTV_TRY(launch_householder_qr(r, bi, P, r, w.W64, w.tau, w.qr, c.status + 2, c.status, c.st,
                                   reserve));
    RUTV_TRY(mixed_round_w(c, r, 0, bi));
    return launch_dgemm(true, false, bi, bi, r, 1.0, w.W64, r, w.W64, r, 0.0, w.Gram64, bi, w.dgemm,
                        w.dgemm_bytes, c.st, true);
  }
  const int64_t h2 = bi - h;
  RUTV_TRY(launch_householder_qr(r, h, P, r, w.W64, w.tau, w.qr, c.status + 2, c.status, c.st,
                                 reserve));
  RUTV_TRY(mixed_round_w(c, r, 0, h));
  RUTV_TRY(launch_dgemm(true, false, h, h, r, 1.0, w.W64, r, w.W64, r, 0.0, w.Gram64, bi, w.dgemm,
                        w.dgemm_bytes, c.st, true));
  retau_kernel<<<1, 256, 0, c.st>>>((int)h, w.Gram64, bi, w.tau);
  note_launch();
  RUTV_CK(cudaGetLastError());
  RUTV_TRY(launch_wy_factor(h, w.Gram64, w.tau, w.S64, c.st, bi));
  // P2 <- P2 - W~1 (S1^T (W~1^T P2)): the two long products on the tensor
  // cores with the six-pair split (FP32-level, like every update of T), the
  // h x h product by S1 in FP64
  double* P2 = P + h * r;
  RUTV_TRY(split_f64(P2, r, r, h2, 0, w.Pp, 0, 0, c.st));
  {
    // a 128 x 128 output over K = r: split K across the SMs (partials in Z)
    BgemmOut ox = out_f32(w.X, h);
    ox.ksplit = (c.cap() > 0 ? c.cap() : dev_info().sms) / 2;
    ox.splitk_ws = w.Z;
    ox.splitk_floats = (size_t)(c.m > c.n ? c.m : c.n) * (size_t)c.b;  // Z: max(m, n) x b
    RUTV_TRY(launch_bgemm(opnd(w.W, 3, 0, 0, 0, r, h), opnd(w.Pp, 3, 0, 0, 0, r, h2), (int)h,
                          (int)h2, (int)r, 3, ox, c.status, c.st, c.cap()));
  }
  RUTV_TRY(f32_to_f64(w.X, h, h, h2, w.qrX, h, c.st));
  RUTV_TRY(launch_dgemm(true, false, h, h2, h, 1.0, w.S64, h, w.qrX, h, 0.0, w.qrY, h, w.dgemm,
                        w.dgemm_bytes, c.st));
  RUTV_TRY(split_f64(w.qrY, h, h, h2, 0, w.Sp, 0, 0, c.st));
  RUTV_TRY(launch_bgemm(opnd(w.W, 3, 0, 0, 1, r, h), opnd(w.Sp, 3, 0, 0, 0, h, h2), (int)r, (int)h2,
                        (int)h, 3, out_f32(w.tmp, r), c.status, c.st, c.cap()));
  {
    ProfScope prof(K_CONVERT, 0.0, 20.0 * (double)r * h2, c.st);
    const int64_t bx = (r + 255) / 256;
    sub_f32_from_f64_kernel<<<dim3((unsigned)(bx < 64 ? bx : 64), (unsigned)h2), 256, 0, c.st>>>(
        P2, r, w.tmp, r, r, h2);
    note_launch();
    RUTV_CK(cudaGetLastError());
  }
  RUTV_TRY(launch_householder_qr(r - h, h2, P2 + h, r, w.W2, w.tau + h, w.qr, c.status + 2,
                                 c.status, c.st, reserve));
  // W(:, h:) = [0; W2], rounded
  double* Wr = w.W64 + h * r;
  RUTV_CK(cudaMemset2DAsync(Wr, (size_t)r * 8, 0, (size_t)h * 8, (size_t)h2, c.st));
  RUTV_CK(cudaMemcpy2DAsync(Wr + h, (size_t)r * 8, w.W2, (size_t)(r - h) * 8, (size_t)(r - h) * 8,
                            (size_t)h2, cudaMemcpyDeviceToDevice, c.st));
  RUTV_TRY(mixed_round_w(c, r, h, h2));
  // Gram(h:, :h) = W~2^T W~1 and the lower part of Gram(h:, h:) = W~2^T W~2, rows h: only
  RUTV_TRY(launch_dgemm(true, false, h2, h, r - h, 1.0, Wr + h, r, w.W64 + h, r, 0.0, w.Gram64 + h,
                        bi, w.dgemm, w.dgemm_bytes, c.st));
  return launch_dgemm(true, false, h2, h2, r - h, 1.0, Wr + h, r, Wr + h, r, 0.0,
                      w.Gram64 + h + h * bi, bi, w.dgemm, w.dgemm_bytes, c.st, true);
}

// Joins the side stream and applies the pending row folds
// T(blk, k+b:) <- U_s^T T(blk, k+b:) on the main stream, in step order.
int mixed_flush_folds(MCtx& c) {
  if (!c.svd_live) return 0;
  c.svd_live = false;
  RUTV_CK(cudaStreamWaitEvent(c.st, c.side->svd, 0));
  MixedWork& w = c.w;
  for (const auto& f : c.folds) {
    const int64_t k = f.first, bi = f.second, nc = c.n - k - bi;
    const Planes Us = plane_cols(w.UsAll, k, bi);
    RUTV_TRY(launch_bgemm(opnd(Us, 3, 0, 0, 0, bi, bi), opnd(w.T, 3, k, k + bi, 0), (int)bi,
                          (int)nc, (int)bi, 3, out_f32(w.tmp, bi), c.status, c.st));
    RUTV_TRY(split_f32(w.tmp, bi, bi, nc, 0, w.T, k, k + bi, c.st));
  }
  c.folds.clear();
  return 0;
}

// Final re-orthogonalisation of U and V (FP32 outputs Uo, Vo) with T (FP32
// output To) carried along, so that U T V^T stays the same product and T
// stays upper triangular.  For X = U or V, E = X^T X - I holds the loss of
// orthogonality of the FP32-level factorization (about 1e-6).  With Phi =
// striu(E) + diag(E)/2 (the first-order Cholesky factor of I + E, minus I):
//   U' = U (I - Phi_U),  V' = V (I - Phi_V^T),  T' = (I + Phi_U) T (I + Phi_V),
// and U'^T U' = I + O(E^2), V'^T V' = I + O(E^2), U' T' V'^T = U T V^T + O(E^2),
// with T' upper triangular (a product of upper triangular factors).  E's
// diagonal is summed in FP64 from the FP32 entries; its off-diagonal entries
// come from the six-product split (FP32-accurate; they are random-signed
// sums, which the tensor-core accumulation handles without bias).  The three
// corrections are O(E) terms, so one BF16 product each is accurate enough.
// The planes of T (the state before the pass) feed both T products; the
// planes of U^T and V^T, no longer needed, hold the planes of U and V.
// Finally the off-diagonal entries that the pass leaves inside the diagonal
// b x b blocks of T (about |E| times their diagonal) are zeroed, restoring
// exactly diagonal blocks.
int mixed_reorth(MCtx& c, float* To, float* Uo, float* Vo) {
  MixedWork& w = c.w;
  const int64_t m = c.m, n = c.n, p = m < n ? m : n;
  ProfScope prof(K_REORTH, 0.0, 0.0, c.st);
  if (c.want_u) {
    Planes P = w.Ut;  // m x m, now the planes of U (not U^T)
    RUTV_TRY(split_f32(Uo, m, m, m, 0, P, 0, 0, c.st));
    BgemmTri upper_only;  // only E's tiles on and above the diagonal are read
    upper_only.out_upper = 1;
    RUTV_TRY(launch_bgemm(opnd(P, 3, 0, 0, 0), opnd(P, 3, 0, 0, 0), (int)m, (int)m, (int)m, 3,
                          out_f32(w.E, m), c.status, c.st, 0, upper_only));
    RUTV_TRY(reorth_phi(Uo, m, m, w.E, m, w.dcol, w.Phi, pad8(m), nullptr, 0, c.st));
    // U -= U Phi_U
    BgemmTri tri;
    tri.b_upper = 1;  // Phi_U upper triangular
    RUTV_TRY(launch_bgemm(opnd(P, 1, 0, 0, 1), opnd_bf16(w.Phi, m, m, pad8(m), 0), (int)m, (int)m,
                          (int)m, 1, out_f32(Uo, m, -1.f, 1.f), c.status, c.st, 0, tri));
    // T += Phi_U T
    tri.a_upper = 1;  // Phi_U and T both upper triangular
    RUTV_TRY(launch_bgemm(opnd_bf16(w.Phi, m, m, pad8(m), 1), opnd(w.T, 1, 0, 0, 0), (int)m,
                          (int)n, (int)m, 1, out_f32(To, m, 1.f, 1.f), c.status, c.st, 0, tri));
  }
  if (c.want_v) {
    Planes P = w.Vt;  // n x n, now the planes of V
    RUTV_TRY(split_f32(Vo, n, n, n, 0, P, 0, 0, c.st));
    BgemmTri upper_only;
    upper_only.out_upper = 1;
    RUTV_TRY(launch_bgemm(opnd(P, 3, 0, 0, 0), opnd(P, 3, 0, 0, 0), (int)n, (int)n, (int)n, 3,
                          out_f32(w.E, n), c.status, c.st, 0, upper_only));
    RUTV_TRY(reorth_phi(Vo, n, n, w.E, n, w.dcol, w.Phi, pad8(n), w.PhiT, pad8(n), c.st));
    // V -= V Phi_V^T
    BgemmTri lower;
    lower.b_lower = 1;  // Phi_V^T lower triangular
    RUTV_TRY(launch_bgemm(opnd(P, 1, 0, 0, 1), opnd_bf16(w.PhiT, n, n, pad8(n), 0), (int)n, (int)n,
                          (int)n, 1, out_f32(Vo, n, -1.f, 1.f), c.status, c.st, 0, lower));
    // T += T Phi_V
    BgemmTri tri;
    tri.a_upper = 1;  // T and Phi_V both upper triangular
    tri.b_upper = 1;
    RUTV_TRY(launch_bgemm(opnd(w.T, 1, 0, 0, 1), opnd_bf16(w.Phi, n, n, pad8(n), 0), (int)m,
                          (int)n, (int)n, 1, out_f32(To, m, 1.f, 1.f), c.status, c.st, 0, tri));
  }
  if (c.want_u || c.want_v) RUTV_TRY(zero_block_offdiag(To, m, p, c.b, c.st));
  return 0;
}

int mixed_step(MCtx& c, int step, int64_t k, int64_t bi) {
  const int64_t m = c.m, n = c.n, rm = m - k, rn = n - k;
  MixedWork& w = c.w;
  // ---------------- right transform
  if (rn > bi) {
    RUTV_TRY(philox_normal_bf16(c.seed, (uint32_t)step, 0u, 0u, rm, bi, w.G, pad8(rm), c.st));
    // Y = T22^T G   (plane 0 of T is the BF16 copy of T22)
    RUTV_TRY(launch_bgemm(opnd(w.T, 1, k, k, 0), opnd_bf16(w.G, rm, bi, pad8(rm), 0), (int)rn,
                          (int)bi, (int)rm, 1, out_f32(w.Y, rn), c.status, c.st, c.cap()));
    for (int it = 0; it < c.q; ++it) {
      RUTV_TRY(scaled_bf16(w.Y, rn, rn, bi, w.Yb, pad8(rn), w.scal, c.st));
      RUTV_TRY(launch_bgemm(opnd(w.T, 1, k, k, 1), opnd_bf16(w.Yb, rn, bi, pad8(rn), 0), (int)rm,
                            (int)bi, (int)rn, 1, out_f32(w.Z, rm), c.status, c.st, c.cap()));
      RUTV_TRY(scaled_bf16(w.Z, rm, rm, bi, w.Yb, pad8(rm), w.scal, c.st));
      RUTV_TRY(launch_bgemm(opnd(w.T, 1, k, k, 0), opnd_bf16(w.Yb, rm, bi, pad8(rm), 0), (int)rn,
                            (int)bi, (int)rm, 1, out_f32(w.Y, rn), c.status, c.st, c.cap()));
    }
    RUTV_TRY(f32_to_f64(w.Y, rn, rn, bi, w.Y64, rn, c.st));
    RUTV_TRY(mixed_qr(c, rn, bi, w.Y64, c.reserve()));
    RUTV_TRY(mixed_wy(c, rn, bi));
    // X = T(:, k:) W (m x bi), then T(:, k:) -= X WS^T with X^T as planes
    RUTV_TRY(launch_bgemm(opnd(w.T, 3, 0, k, 1), opnd(w.W, 3, 0, 0, 0, rn, bi), (int)m, (int)bi, (int)rn, 3,
                          out_f32(w.X, m), c.status, c.st, c.cap()));
    RUTV_TRY(split_f32(w.X, m, bi, m, 1, w.Xp, 0, 0, c.st));
    RUTV_TRY(launch_bgemm(opnd(w.Xp, 3, 0, 0, 0, bi, m), opnd(w.WSt, 3, 0, 0, 0, bi, rn), (int)m, (int)rn, (int)bi,
                          3, out_planes(w.T, 0, k, -1.f), c.status, c.st, c.cap()));
    if (c.want_v) RUTV_TRY(mixed_apply_transposed(c, w.Vt, k, rn, bi));
  }
  // ---------------- left transform
  if (rm > bi) {
    RUTV_TRY(merge_f64(w.T, k, k, rm, bi, 0, w.Y64, rm, c.st));
    RUTV_TRY(mixed_qr(c, rm, bi, w.Y64, c.reserve()));
    RUTV_TRY(split_f64(w.Y64, rm, rm, bi, 0, w.T, k, k, c.st));  // R and exact zeros
    RUTV_TRY(mixed_wy(c, rm, bi));
    if (rn > bi) {
      const int64_t nc = rn - bi;
      RUTV_TRY(launch_bgemm(opnd(w.W, 3, 0, 0, 0, rm, bi), opnd(w.T, 3, k, k + bi, 0), (int)bi, (int)nc,
                            (int)rm, 3, out_f32(w.X, bi), c.status, c.st, c.cap()));
      RUTV_TRY(split_f32(w.X, bi, bi, nc, 0, w.Xp, 0, 0, c.st));
      RUTV_TRY(launch_bgemm(opnd(w.WSt, 3, 0, 0, 0, bi, rm), opnd(w.Xp, 3, 0, 0, 0, bi, nc), (int)rm, (int)nc,
                            (int)bi, 3, out_planes(w.T, k, k + bi, -1.f), c.status, c.st, c.cap()));
    }
    if (c.want_u) RUTV_TRY(mixed_apply_transposed(c, w.Ut, k, rm, bi));
  }
  // ---------------- small SVD (FP64) and fold-back (six-product BF16), side stream
  cudaStream_t ss = c.side->st;
  const Planes Us = plane_cols(w.UsAll, k, bi);
  RUTV_CK(cudaEventRecord(c.side->panel, c.st));
  RUTV_CK(cudaStreamWaitEvent(ss, c.side->panel, 0));
  RUTV_TRY(merge_f64(w.T, k, k, bi, bi, 0, w.blk64, bi, ss));
  RUTV_TRY(launch_small_svd((int)bi, w.blk64, bi, w.D, w.Us64, w.Vs64, c.status + 8, w.svd,
                            w.dgemm2, w.dgemm_bytes, ss));
  RUTV_TRY(split_f64(w.Us64, bi, bi, bi, 0, Us, 0, 0, ss));
  RUTV_TRY(split_f64(w.Vs64, bi, bi, bi, 0, w.Vs, 0, 0, ss));
  if (k > 0) {  // T(0:k, blk) <- T(0:k, blk) Vs
    RUTV_TRY(launch_bgemm(opnd(w.T, 3, 0, k, 1), opnd(w.Vs, 3, 0, 0, 0, bi, bi), (int)k, (int)bi, (int)bi, 3,
                          out_f32(w.tmp2, k), c.status, ss, kSvdSms));
    RUTV_TRY(split_f32(w.tmp2, k, k, bi, 0, w.T, 0, k, ss));
  }
  if (c.want_v) {  // V(:, blk) <- V(:, blk) Vs, i.e. V^T(blk, :) <- Vs^T V^T(blk, :)
    RUTV_TRY(launch_bgemm(opnd(w.Vs, 3, 0, 0, 0, bi, bi), opnd(w.Vt, 3, k, 0, 0), (int)bi, (int)n, (int)bi,
                          3, out_f32(w.tmp2, bi), c.status, ss, kSvdSms));
    RUTV_TRY(split_f32(w.tmp2, bi, bi, n, 0, w.Vt, k, 0, ss));
  }
  if (c.want_u) {
    RUTV_TRY(launch_bgemm(opnd(Us, 3, 0, 0, 0, bi, bi), opnd(w.Ut, 3, k, 0, 0), (int)bi, (int)m, (int)bi,
                          3, out_f32(w.tmp2, bi), c.status, ss, kSvdSms));
    RUTV_TRY(split_f32(w.tmp2, bi, bi, m, 0, w.Ut, k, 0, ss));
  }
  RUTV_TRY(set_diag_planes(w.T, k, bi, w.D, ss));
  RUTV_CK(cudaEventRecord(c.side->svd, ss));
  c.svd_live = true;
  if (rn > bi) c.folds.emplace_back(k, bi);  // T(blk, k+bi:) <- U_s^T T(blk, k+bi:)
  return 0;
}

}  // namespace

size_t mixed_workspace_bytes(int64_t m, int64_t n, int64_t b) { return mixed_bytes(m, n, b); }

}  // namespace rutv

using namespace rutv;

extern "C" {

int randutv_factor_mixed(int64_t m, int64_t n, const float* A, int64_t lda, int b, int q,
                         uint64_t seed, float* U, float* T, float* V, int max_steps, void* stream) {
  if (m < 1) return -1;
  if (n < 1) return -2;
  if (!A) return -3;
  if (lda < m) return -4;
  if (b < 8 || b > 256 || (b % 8) != 0) return -5;
  if (q < 0 || q > 16) return -6;
  if (!T) return -9;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t p = m < n ? m : n;
  const int64_t bb = b < p ? b : p;
  if ((bb % 8) != 0 && bb != p) return -5;
  Arena ar;
  RUTV_TRY(scratch_reserve(mixed_bytes(m, n, b), &ar));
  unsigned* status = nullptr;
  RUTV_TRY(status_words(&status));
  RUTV_CK(cudaMemsetAsync(status, 0, 64 * sizeof(unsigned), st));
  MCtx c;
  c.m = m;
  c.n = n;
  c.b = b;
  c.q = q;
  c.seed = seed;
  c.want_u = U != nullptr;
  c.want_v = V != nullptr;
  c.w = carve_mixed(ar, m, n, b);
  c.status = status;
  c.st = st;
  RUTV_TRY(launch_check_finite_f32(m, n, A, lda, status, st));
  RUTV_TRY(split_f32(A, lda, m, n, 0, c.w.T, 0, 0, st));
  if (c.want_u) RUTV_TRY(set_identity_planes(c.w.Ut, st));
  if (c.want_v) RUTV_TRY(set_identity_planes(c.w.Vt, st));
  RUTV_TRY(side_stream(&c.side));
  int step = 0;
  for (int64_t k = 0; k < p; k += b, ++step) {
    const int64_t bi = (b < p - k) ? b : p - k;
    if (max_steps >= 0 && step >= max_steps) break;
    RUTV_TRY(mixed_step(c, step, k, bi));
  }
  RUTV_TRY(mixed_flush_folds(c));  // also joins the side stream into the caller's stream
  RUTV_TRY(merge_f32(c.w.T, 0, 0, m, n, 0, T, m, st));
  if (c.want_u) RUTV_TRY(merge_f32(c.w.Ut, 0, 0, m, m, 1, U, m, st));
  if (c.want_v) RUTV_TRY(merge_f32(c.w.Vt, 0, 0, n, n, 1, V, n, st));
  if (step == (int)nsteps(m, n, b)) RUTV_TRY(mixed_reorth(c, T, U, V));  // completed runs only
  return 0;
}

int randutv_gemm_bf16(char transa, int64_t M, int64_t N, int64_t K, float alpha, const float* A,
                      int64_t lda, const float* B, int64_t ldb, float beta, float* C, int64_t ldc,
                      int planes, void* stream) {
  const bool ta = (transa == 'T' || transa == 't');
  if (!ta && !(transa == 'N' || transa == 'n')) return -1;
  if (M < 1) return -2;
  if (N < 1) return -3;
  if (K < 1) return -4;
  if (!A) return -6;
  if (lda < (ta ? K : M)) return -7;
  if (!B) return -8;
  if (ldb < K) return -9;
  if (!C) return -11;
  if (ldc < M) return -12;
  if (planes != 1 && planes != 3) return -13;
  if (M > (1 << 30) || N > (1 << 30) || K > (1 << 30)) return RANDUTV_EUNSUPPORTED;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t ar_rows = ta ? K : M, ar_cols = ta ? M : K;
  // beta = 0 and an output of few 128 x 64 tiles over a long K: split K across the SMs
  // (partial products in the scratch, at most 64 MB of them, summed in a fixed order)
  const int64_t tiles = ((M + 127) / 128) * ((N + 63) / 64);
  const int sms = dev_info().sms;
  int64_t ks = 1;
  size_t ws_floats = 0;
  if (beta == 0.f && 2 * tiles <= sms && K >= 1024) {
    ks = std::min<int64_t>(sms / tiles, (K + 63) / 64);
    ks = std::min<int64_t>(ks, (int64_t)(((size_t)16 << 20) / ((size_t)M * (size_t)N)));
    if (ks > 1) ws_floats = (size_t)ks * (size_t)M * (size_t)N;
  }
  Arena ar;
  RUTV_TRY(scratch_reserve(planes_bytes(ar_rows, ar_cols) + planes_bytes(K, N) + ws_floats * 4 +
                               4096, &ar));
  unsigned* status = nullptr;
  RUTV_TRY(status_words(&status));
  RUTV_CK(cudaMemsetAsync(status, 0, 64 * sizeof(unsigned), st));
  Planes Pa = carve_planes(ar, ar_rows, ar_cols);
  Planes Pb = carve_planes(ar, K, N);
  RUTV_TRY(split_f32(A, lda, ar_rows, ar_cols, 0, Pa, 0, 0, st));
  RUTV_TRY(split_f32(B, ldb, K, N, 0, Pb, 0, 0, st));
  BgemmOut out = out_f32(C, ldc, alpha, beta);
  if (ws_floats > 0) {
    out.ksplit = (int)ks;
    out.splitk_ws = (float*)ar.take(ws_floats * 4);
    out.splitk_floats = ws_floats;
  }
  return launch_bgemm(opnd(Pa, planes, 0, 0, ta ? 0 : 1), opnd(Pb, planes, 0, 0, 0), (int)M,
                      (int)N, (int)K, planes, out, status, st);
}

}  // extern "C"
