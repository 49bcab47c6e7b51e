// Rank-k approximation through randUTV and its adjoint (FP64).
//
// A_k = U(:, 0:k) U(:, 0:k)^T A (§1.1: A_k = U(:,1:k) R(1:k,:) V^*), for k a
// multiple of b.  Only the first k/b block steps of §3.1 / Fig. 2 fix the span
// of U(:, 0:k), and the block SVDs rotate columns inside a block without
// changing that span or any later trailing matrix, so the map A -> A_k runs
// through the sketch, the power iteration and the two Householder transforms
// of each step only.  With the sketch fixed it is smooth in A (for generic
// A), and its adjoint is written out here step by step in reverse:
//
//   * an application X -> X Q or Q^T X with Q = I - W S W^T: the adjoint of
//     X and of the compact-WY pair (W, S) by matrix products;
//   * S = larft(W, tau) (S_jj = tau_j, S(0:j,j) = -tau_j S(0:j,0:j) G(0:j,j),
//     G = W^T W): the recurrence run backwards column by column;
//   * the Householder QR of a panel: columns in reverse order; the panel
//     before column j is rebuilt from the one after it with H_j (a reflector
//     is its own inverse) and the column itself from (v_j, tau_j, beta_j), so
//     no intermediate panel is stored;
//   * the power-iteration products.
// The forward steps are recomputed inside the backward call (the factors are
// not kept between calls).
#include <cmath>
#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace rutv {

namespace {

// ---------------------------------------------------------- panel QR adjoint
// Column j of the reverse sweep.  X: panel state after column j (r x c, ld r),
// Xb: its adjoint, W (r x c, ld r), tau (c), Wb (r x c) adjoint of W, taub.
// K1: for each trailing column l: a_l = v.X(:,l), p_l = v.Xb(:,l), rows j..r-1.
__global__ void hqr_rev_dots(int r, int c, int j, const double* __restrict__ X,
                             const double* __restrict__ Xb, const double* __restrict__ W,
                             double* __restrict__ ap) {
  __shared__ double red[2][8];
  const int l = j + 1 + blockIdx.x;
  if (l >= c) return;
  double a = 0.0, p = 0.0;
  for (int i = j + threadIdx.x; i < r; i += blockDim.x) {
    const double v = W[i + (int64_t)j * r];
    a = fma(v, X[i + (int64_t)l * r], a);
    p = fma(v, Xb[i + (int64_t)l * r], p);
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    p += __shfl_xor_sync(0xffffffffu, p, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = a;
    red[1][threadIdx.x >> 5] = p;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sa = 0.0, sp = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { sa += red[0][w]; sp += red[1][w]; }
    ap[2 * l] = sa;
    ap[2 * l + 1] = sp;
  }
}

// K2: per row i >= j: X_prev = X - tau v a^T (restored in place), s = a (1 - tau v.v),
// Wb(i, j) += -tau (Xb(i,:) s + X_prev(i,:) p), Xb(i,:) <- Xb(i,:) - tau v_i p.
__global__ void hqr_rev_rows(int r, int c, int j, double tau, double vv, double* __restrict__ X,
                             double* __restrict__ Xb, const double* __restrict__ W,
                             double* __restrict__ Wb, const double* __restrict__ ap) {
  const int i = j + blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= r) return;
  const double vi = W[i + (int64_t)j * r];
  const double sfac = 1.0 - tau * vv;
  double acc = 0.0;
  for (int l = j + 1; l < c; ++l) {
    const double a = ap[2 * l], p = ap[2 * l + 1];
    const int64_t o = i + (int64_t)l * r;
    const double xp = fma(-tau * vi, a, X[o]);
    const double yb = Xb[o];
    acc = fma(yb, a * sfac, acc);
    acc = fma(xp, p, acc);
    X[o] = xp;
    Xb[o] = fma(-tau * vi, p, yb);
  }
  if (i > j) Wb[i + (int64_t)j * r] += -tau * acc;
}

// K3: reverse of the generation of reflector j from its column x (rows j..r-1).
// One block.  Restores X(j:, j) = x and writes its adjoint into Xb(j:, j).
// vv = v.v (the host holds W and computes it once per column).
__global__ void hqr_rev_gen(int r, int c, int j, double tau, double vv, double* __restrict__ X,
                            double* __restrict__ Xb, const double* __restrict__ W,
                            const double* __restrict__ Wb, double taub_in,
                            const double* __restrict__ ap) {
  __shared__ double red[32];
  __shared__ double sh[4];
  const double beta = X[j + (int64_t)j * r];
  // tau adjoint from the trailing update: -sum_l p_l s_l, summed by the first
  // warp in a fixed order (lanes stride the columns, then a shuffle tree)
  if (threadIdx.x < 32) {
    const double sfac = 1.0 - tau * vv;
    double tb = 0.0;
    for (int l = j + 1 + (int)threadIdx.x; l < c; l += 32) tb -= ap[2 * l + 1] * ap[2 * l] * sfac;
    for (int o = 16; o > 0; o >>= 1) tb += __shfl_xor_sync(0xffffffffu, tb, o);
    if (threadIdx.x == 0) sh[0] = tb + taub_in;
  }
  __syncthreads();
  const double taub = sh[0];
  // x = beta (e1 - tau v): alpha = x_0, x1 = x_{1:}
  const double alpha = beta * (1.0 - tau);
  double ux = 0.0, n1 = 0.0;
  for (int i = j + 1 + threadIdx.x; i < r; i += blockDim.x) {
    const double x1 = -beta * tau * W[i + (int64_t)j * r];
    ux = fma(Wb[i + (int64_t)j * r], x1, ux);
    n1 = fma(x1, x1, n1);
  }
  for (int o = 16; o > 0; o >>= 1) {
    ux += __shfl_xor_sync(0xffffffffu, ux, o);
    n1 += __shfl_xor_sync(0xffffffffu, n1, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[threadIdx.x >> 5] = ux;
    red[16 + (threadIdx.x >> 5)] = n1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a += red[w]; b += red[16 + w]; }
    sh[1] = a;
    sh[2] = b;
  }
  __syncthreads();
  const double ubx1 = sh[1];
  const double betab = Xb[j + (int64_t)j * r];
  double alphab, x1fac, x1scale;
  if (tau == 0.0) {
    // x2 == 0: v = e1, beta = alpha; only beta depends on alpha
    alphab = betab;
    x1fac = 0.0;
    x1scale = 0.0;
  } else {
    const double nrm = fabs(beta);
    const double sg = (alpha >= 0.0) ? 1.0 : -1.0;
    const double g = alpha - beta;
    const double bt = betab + taub * alpha / (beta * beta) + ubx1 / (g * g);
    alphab = -taub / beta - ubx1 / (g * g) + bt * (-sg) * alpha / nrm;
    x1fac = 1.0 / g;               // multiplies ub_i
    x1scale = bt * (-sg) / nrm;    // multiplies x1_i
  }
  for (int i = j + threadIdx.x; i < r; i += blockDim.x) {
    const int64_t o = i + (int64_t)j * r;
    if (i == j) {
      X[o] = alpha;
      Xb[o] = alphab;
    } else {
      const double x1 = -beta * tau * W[o];
      X[o] = x1;
      Xb[o] = Wb[o] * x1fac + x1 * x1scale;
    }
  }
}

// ------------------------------------------------------------ larft adjoint
// Mb = triu(Sb) diag(tau)  (b x b, ld b)
__global__ void larft_rev_scale_kernel(int c, const double* __restrict__ Sb,
                                       const double* __restrict__ tau, double* __restrict__ Mb) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < c * c; e += gridDim.x * blockDim.x) {
    const int i = e % c, j = e / c;
    Mb[e] = (i <= j) ? Sb[e] * tau[j] : 0.0;
  }
}

// Row i (one warp): Gb(i, l) = tau_i Kb(i, l) for l > i (0 elsewhere in the row), and
// taub_i += sum_j M(j, i) Sb(j, i) [j <= i] + sum_{l > i} Kb(i, l) Gm(i, l), each sum in a
// fixed order (lane strides, then a shuffle tree).
__global__ void larft_rev_finish_kernel(int c, const double* __restrict__ Kb,
                                        const double* __restrict__ M,
                                        const double* __restrict__ Sb,
                                        const double* __restrict__ Gm,
                                        const double* __restrict__ tau, double* __restrict__ Gb,
                                        double* __restrict__ taub) {
  const int i = blockIdx.x, lane = threadIdx.x;
  const double ti = tau[i];
  double acc = 0.0;
  for (int l = lane; l < c; l += 32) {
    const int64_t o = i + (int64_t)l * c;
    const double kb = Kb[o];
    if (l > i) {
      Gb[o] = ti * kb;
      acc = fma(kb, Gm[o], acc);
    } else {
      Gb[o] = 0.0;
    }
    // (M^T triu(Sb))_ii: column i of M and of Sb, rows l <= i
    if (l <= i) acc = fma(M[l + (int64_t)i * c], Sb[l + (int64_t)i * c], acc);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) taub[i] += acc;
}

__global__ void axpy_kernel(int64_t n, double a, const double* x, double* y) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    y[e] = fma(a, x[e], y[e]);
}

// B = A^T (n x n, ld n)
__global__ void transpose_kernel(int n, const double* __restrict__ A, double* __restrict__ B) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * n; e += gridDim.x * blockDim.x) {
    const int i = e % n, j = e / n;
    B[j + (int64_t)i * n] = A[e];
  }
}

__global__ void eye_kernel(int64_t rows, int64_t cols, double* X, int64_t ld) {
  const int64_t total = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % rows, j = e / rows;
    X[i + j * ld] = (i == j) ? 1.0 : 0.0;
  }
}

__global__ void keep_strict_lower(int64_t r, int64_t c, double* Wb) {
  // W's unit diagonal and zeros above are fixed: their adjoint is dropped
  const int64_t total = r * c;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % r, j = e / r;
    if (i <= j) Wb[e] = 0.0;
  }
}

int grid_of(int64_t n) {
  int64_t b = (n + 255) / 256;
  const int64_t cap = (int64_t)dev_info().sms * 8;
  return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

// --------------------------------------------------------------- context
struct LCtx {
  cudaStream_t st;
  double* gs;  // dgemm split-K scratch
  size_t gsb;
  unsigned* status;
  char* qr;
};

int G(LCtx& c, bool ta, bool tb, int64_t M, int64_t N, int64_t K, double al, const double* A,
      int64_t lda, const double* B, int64_t ldb, double be, double* C, int64_t ldc) {
  return launch_dgemm(ta, tb, M, N, K, al, A, lda, B, ldb, be, C, ldc, c.gs, c.gsb, c.st);
}

int copy(LCtx& c, double* dst, int64_t ldd, const double* src, int64_t lds, int64_t rows,
         int64_t cols) {
  if (rows <= 0 || cols <= 0) return 0;
  RUTV_CK(cudaMemcpy2DAsync(dst, ldd * 8, src, lds * 8, rows * 8, cols, cudaMemcpyDeviceToDevice,
                            c.st));
  return 0;
}

int zero(LCtx& c, double* p, size_t count) {
  if (count) RUTV_CK(cudaMemsetAsync(p, 0, count * 8, c.st));
  return 0;
}

// Householder QR of P (r x b, ld r) in place -> W, tau, S (and Gram in Gm).
int hqr_wy(LCtx& c, int64_t r, int64_t b, double* P, double* W, double* tau, double* Gm,
           double* S) {
  RUTV_TRY(launch_householder_qr(r, b, P, r, W, tau, c.qr, c.status + 2, c.status, c.st));
  RUTV_TRY(G(c, true, false, b, b, r, 1.0, W, r, W, r, 0.0, Gm, b));
  RUTV_TRY(launch_wy_factor(b, Gm, tau, S, c.st));
  return 0;
}

// Reverse of the panel QR: X = panel after QR (r x b, consumed), W, tau; Wb, taub
// (adjoints of W and tau from downstream; Wb consumed) -> Pb (r x b) adjoint of
// the input panel (R's adjoint taken as zero: R is not used downstream).
int hqr_reverse(LCtx& c, int64_t r, int64_t b, double* X, const double* W, const double* tau_dev,
                double* Wb, double* taub_dev, double* Pb, double* ap) {
  std::vector<double> tau(b), taub(b);
  RUTV_CK(cudaMemcpyAsync(tau.data(), tau_dev, b * 8, cudaMemcpyDeviceToHost, c.st));
  RUTV_CK(cudaMemcpyAsync(taub.data(), taub_dev, b * 8, cudaMemcpyDeviceToHost, c.st));
  std::vector<double> Wh((size_t)r * b);
  RUTV_CK(cudaMemcpyAsync(Wh.data(), W, (size_t)r * b * 8, cudaMemcpyDeviceToHost, c.st));
  RUTV_CK(cudaStreamSynchronize(c.st));
  RUTV_TRY(zero(c, Pb, (size_t)r * b));
  ProfScope prof(K_ADJOINT, 4.0 * (double)r * b * b, 40.0 * (double)r * b, c.st);
  for (int64_t j = b - 1; j >= 0; --j) {
    double vv = 0.0;
    for (int64_t i = j; i < r; ++i) vv += Wh[i + j * r] * Wh[i + j * r];
    if (j + 1 < b) {
      hqr_rev_dots<<<(unsigned)(b - j - 1), 256, 0, c.st>>>((int)r, (int)b, (int)j, X, Pb, W, ap);
      const int64_t rows = r - j;
      hqr_rev_rows<<<(unsigned)((rows + 255) / 256), 256, 0, c.st>>>((int)r, (int)b, (int)j,
                                                                      tau[j], vv, X, Pb, W, Wb, ap);
      note_launch(2);
    }
    hqr_rev_gen<<<1, 512, 0, c.st>>>((int)r, (int)b, (int)j, tau[j], vv, X, Pb, W, Wb, taub[j],
                                     ap);
    note_launch();
    RUTV_CK(cudaGetLastError());
  }
  return 0;
}

// Adjoints of X -> X Q (right) for Q = I - W S W^T (X rows x cols, W cols x b):
// Xb = Ob Q^T (written into Xb), Sb += -(XW)^T (ObW), Wb += -X^T ObW S^T - Ob^T XW S.
// XW: X W kept from the forward (rows x b, ld rows), or null to recompute it into t1.
int right_apply_rev(LCtx& c, int64_t rows, int64_t cols, int64_t b, const double* X, int64_t ldx,
                    const double* Ob, int64_t ldo, const double* W, const double* S, double* Xb,
                    int64_t ldxb, double* Wb, double* Sb, double* t1, double* t2, double* t3,
                    const double* XW = nullptr) {
  if (XW) t1 = const_cast<double*>(XW);  // read only below
  else RUTV_TRY(G(c, false, false, rows, b, cols, 1.0, X, ldx, W, cols, 0.0, t1, rows));  // XW
  RUTV_TRY(G(c, false, false, rows, b, cols, 1.0, Ob, ldo, W, cols, 0.0, t2, rows));   // ObW
  RUTV_TRY(G(c, true, false, b, b, rows, -1.0, t1, rows, t2, rows, 1.0, Sb, b));       // Sb
  RUTV_TRY(G(c, false, true, rows, b, b, 1.0, t2, rows, S, b, 0.0, t3, rows));         // ObW S^T
  RUTV_TRY(G(c, true, false, cols, b, rows, -1.0, X, ldx, t3, rows, 1.0, Wb, cols));   // -X^T ObW S^T
  RUTV_TRY(G(c, false, false, rows, b, b, 1.0, t1, rows, S, b, 0.0, t2 /*reuse after*/, rows));
  // t2 now XW S; t3 holds ObW S^T
  RUTV_TRY(G(c, true, false, cols, b, rows, -1.0, Ob, ldo, t2, rows, 1.0, Wb, cols));  // -Ob^T XW S
  if (Xb != Ob) RUTV_TRY(copy(c, Xb, ldxb, Ob, ldo, rows, cols));
  RUTV_TRY(G(c, false, true, rows, cols, b, -1.0, t3, rows, W, cols, 1.0, Xb, ldxb));  // Ob Q^T
  return 0;
}

// Adjoints of X -> Q^T X (left) for Q = I - W S W^T (X rows x cols, W rows x b):
// Xb = Q Ob, Sb += -(W^T X)(W^T Ob)^T, Wb += -Ob (W^T X)^T S - X (W^T Ob)^T S^T.
// WX: W^T X kept from the forward (b x cols, ld b), or null to recompute it into t1.
int left_apply_rev(LCtx& c, int64_t rows, int64_t cols, int64_t b, const double* X, int64_t ldx,
                   const double* Ob, int64_t ldo, const double* W, const double* S, double* Xb,
                   int64_t ldxb, double* Wb, double* Sb, double* t1, double* t2, double* t3,
                   const double* WX = nullptr) {
  if (WX) t1 = const_cast<double*>(WX);  // read only below
  else RUTV_TRY(G(c, true, false, b, cols, rows, 1.0, W, rows, X, ldx, 0.0, t1, b));  // WX
  RUTV_TRY(G(c, true, false, b, cols, rows, 1.0, W, rows, Ob, ldo, 0.0, t2, b));    // WOb
  RUTV_TRY(G(c, false, true, b, b, cols, -1.0, t1, b, t2, b, 1.0, Sb, b));          // Sb
  RUTV_TRY(G(c, true, false, cols, b, b, 1.0, t1, b, S, b, 0.0, t3, cols));         // WX^T S (cols x b)
  RUTV_TRY(G(c, false, false, rows, b, cols, -1.0, Ob, ldo, t3, cols, 1.0, Wb, rows));
  RUTV_TRY(G(c, true, true, cols, b, b, 1.0, t2, b, S, b, 0.0, t3, cols));          // WOb^T S^T
  RUTV_TRY(G(c, false, false, rows, b, cols, -1.0, X, ldx, t3, cols, 1.0, Wb, rows));
  // Xb = Ob - W S (W^T Ob)   (S WOb into t3, free again; t1 may be the forward's W^T X)
  RUTV_TRY(G(c, false, false, b, cols, b, 1.0, S, b, t2, b, 0.0, t3, b));           // S WOb
  if (Xb != Ob) RUTV_TRY(copy(c, Xb, ldxb, Ob, ldo, rows, cols));
  RUTV_TRY(G(c, false, false, rows, cols, b, -1.0, W, rows, t3, b, 1.0, Xb, ldxb));
  return 0;
}

// S and tau adjoint (Sb, upper part, consumed) -> taub += ..., Wb += W (Gb + Gb^T).
// S = M D with M = (I + D N)^-1, D = diag(tau), N = striu(Gm): with Mb = triu(Sb) D and
// Kb = -M^T Mb M^T, the Gram adjoint is striu(D Kb) and taub_i gets (M^T triu(Sb))_ii +
// sum_{l > i} Kb_il N_il.  Four b x b products instead of a column-by-column walk in one
// CTA.  ws: 4 b^2 doubles.
int larft_reverse(LCtx& c, int64_t r, int64_t b, const double* W, const double* tau,
                  const double* S, const double* Gm, double* Sb, double* Wb, double* taub,
                  double* Gb, double* ws) {
  (void)S;
  double* M = ws;
  double* Mb = M + b * b;
  double* T1 = Mb + b * b;
  double* Kb = T1 + b * b;
  RUTV_TRY(launch_wy_inverse(b, Gm, tau, M, c.st));
  {
    ProfScope prof(K_ADJOINT, 0.0, 24.0 * (double)b * b, c.st);
    larft_rev_scale_kernel<<<grid_of(b * b), 256, 0, c.st>>>((int)b, Sb, tau, Mb);
    note_launch();
    RUTV_CK(cudaGetLastError());
  }
  RUTV_TRY(G(c, false, true, b, b, b, 1.0, Mb, b, M, b, 0.0, T1, b));     // Mb M^T
  RUTV_TRY(G(c, true, false, b, b, b, -1.0, M, b, T1, b, 0.0, Kb, b));    // -M^T Mb M^T
  {
    ProfScope prof(K_ADJOINT, 0.0, 32.0 * (double)b * b, c.st);
    larft_rev_finish_kernel<<<(unsigned)b, 32, 0, c.st>>>((int)b, Kb, M, Sb, Gm, tau, Gb, taub);
    note_launch();
    RUTV_CK(cudaGetLastError());
  }
  RUTV_TRY(G(c, false, false, r, b, b, 1.0, W, r, Gb, b, 1.0, Wb, r));
  RUTV_TRY(G(c, false, true, r, b, b, 1.0, W, r, Gb, b, 1.0, Wb, r));
  return 0;
}

struct StepState {
  int64_t k, rm, rn;
  bool right, left;
  double *M, *N;                 // input of the step, and after the right transform
  double* Xin;                   // U_k chain: the block U(k:m, k:kk) before Q_U of this step
  double *MW, *WN;               // forward products kept for the reverse: M W_V, W_U^T N(:, b:)
  double *Ych, *Zch;             // power chain: Y_0..Y_q (rn x b each), Z_0..Z_{q-1}
  double *PV, *WV, *tauV, *SV, *GV;  // sketch QR: final panel, reflectors, WY factor, Gram
  double *PU, *WU, *tauU, *SU, *GU;  // panel QR of the new block column
};

}  // namespace

}  // namespace rutv



using namespace rutv;

namespace {

struct Pool {
  std::vector<void*> ptrs;
  ~Pool() {
    for (void* p : ptrs) cudaFree(p);
  }
  double* get(size_t count) {
    void* p = nullptr;
    if (cudaMalloc(&p, (count ? count : 1) * sizeof(double)) != cudaSuccess) return nullptr;
    ptrs.push_back(p);
    return (double*)p;
  }
};

int check_args(int64_t m, int64_t n, const double* A, int64_t lda, int k, int b, int q) {
  if (m < 1) return -1;
  if (n < 1) return -2;
  if (!A) return -3;
  if (lda < m) return -4;
  const int64_t p = m < n ? m : n;
  if (k < 1 || k >= p) return -5;
  if (b < 1 || b > 256 || (k % b) != 0) return -6;
  if (q < 0 || q > 16) return -7;
  return 0;
}

// Forward steps of the low-rank map; fills the step states and U (m x m).
int lowrank_forward(LCtx& c, Pool& pool, int64_t m, int64_t n, const double* A, int64_t lda,
                    int k, int b, int q, uint64_t seed, std::vector<StepState>& st, double* U,
                    double* ap) {
  const int s = k / b;
  st.resize(s);
  double* Min = pool.get((size_t)m * n);
  if (!Min) return RANDUTV_ENOMEM;
  RUTV_TRY(copy(c, Min, m, A, lda, m, n));
  (void)ap;
  for (int i = 0; i < s; ++i) {
    StepState& S = st[i];
    S.k = (int64_t)i * b;
    S.rm = m - S.k;
    S.rn = n - S.k;
    S.right = S.rn > b;
    S.left = S.rm > b;
    S.M = Min;
    const int64_t rm = S.rm, rn = S.rn;
    S.N = pool.get((size_t)rm * rn);
    if (!S.N) return RANDUTV_ENOMEM;
    if (S.right) {
      S.Ych = pool.get((size_t)(q + 1) * rn * b);
      S.Zch = pool.get((size_t)(q > 0 ? q : 1) * rm * b);
      S.PV = pool.get((size_t)rn * b);
      S.WV = pool.get((size_t)rn * b);
      S.tauV = pool.get(b);
      S.SV = pool.get((size_t)b * b);
      S.GV = pool.get((size_t)b * b);
      double* Gs = pool.get((size_t)rm * b);
      if (!S.Ych || !S.Zch || !S.PV || !S.WV || !S.tauV || !S.SV || !S.GV || !Gs)
        return RANDUTV_ENOMEM;
      RUTV_TRY(launch_philox_normal(seed, (uint32_t)i, 0u, 0u, rm, b, Gs, rm, c.st));
      RUTV_TRY(G(c, true, false, rn, b, rm, 1.0, S.M, rm, Gs, rm, 0.0, S.Ych, rn));
      for (int it = 0; it < q; ++it) {
        double* Yt = S.Ych + (size_t)it * rn * b;
        double* Zt = S.Zch + (size_t)it * rm * b;
        RUTV_TRY(G(c, false, false, rm, b, rn, 1.0, S.M, rm, Yt, rn, 0.0, Zt, rm));
        RUTV_TRY(G(c, true, false, rn, b, rm, 1.0, S.M, rm, Zt, rm, 0.0, Yt + (size_t)rn * b, rn));
      }
      RUTV_TRY(copy(c, S.PV, rn, S.Ych + (size_t)q * rn * b, rn, rn, b));
      RUTV_TRY(hqr_wy(c, rn, b, S.PV, S.WV, S.tauV, S.GV, S.SV));
      // N = M Q_V
      RUTV_TRY(copy(c, S.N, rm, S.M, rm, rm, rn));
      S.MW = pool.get((size_t)rm * b);
      double* t2 = pool.get((size_t)rm * b);
      if (!S.MW || !t2) return RANDUTV_ENOMEM;
      RUTV_TRY(G(c, false, false, rm, b, rn, 1.0, S.M, rm, S.WV, rn, 0.0, S.MW, rm));
      RUTV_TRY(G(c, false, false, rm, b, b, 1.0, S.MW, rm, S.SV, b, 0.0, t2, rm));
      RUTV_TRY(G(c, false, true, rm, rn, b, -1.0, t2, rm, S.WV, rn, 1.0, S.N, rm));
    } else {
      RUTV_TRY(copy(c, S.N, rm, S.M, rm, rm, rn));
    }
    // panel QR of N(:, 0:b); M_{i+1} = (Q_U^T N)(b:, b:); U(:, k:) <- U(:, k:) Q_U
    S.PU = pool.get((size_t)rm * b);
    S.WU = pool.get((size_t)rm * b);
    S.tauU = pool.get(b);
    S.SU = pool.get((size_t)b * b);
    S.GU = pool.get((size_t)b * b);
    double* Nr = pool.get((size_t)rm * (rn - b));
    double* wx = pool.get((size_t)b * (rn > m ? rn : m));
    double* wx2 = pool.get((size_t)b * (rn > m ? rn : m));
    if (!S.PU || !S.WU || !S.tauU || !S.SU || !S.GU || !Nr || !wx || !wx2) return RANDUTV_ENOMEM;
    RUTV_TRY(copy(c, S.PU, rm, S.N, rm, rm, b));
    RUTV_TRY(hqr_wy(c, rm, b, S.PU, S.WU, S.tauU, S.GU, S.SU));
    const int64_t nc = rn - b;
    RUTV_TRY(copy(c, Nr, rm, S.N + b * rm, rm, rm, nc));
    RUTV_TRY(G(c, true, false, b, nc, rm, 1.0, S.WU, rm, Nr, rm, 0.0, wx, b));        // W^T X
    S.WN = wx;  // kept for the reverse
    RUTV_TRY(G(c, true, false, b, nc, b, 1.0, S.SU, b, wx, b, 0.0, wx2, b));           // S^T W^T X
    RUTV_TRY(G(c, false, false, rm, nc, b, -1.0, S.WU, rm, wx2, b, 1.0, Nr, rm));      // Q^T X
    double* Mnext = pool.get((size_t)(rm - b) * nc);
    if (!Mnext) return RANDUTV_ENOMEM;
    RUTV_TRY(copy(c, Mnext, rm - b, Nr + b, rm, rm - b, nc));
    Min = Mnext;
  }
  // U_k = Qt_0 (Qt_1 (... (Qt_{s-1} E_k))), Qt_i = diag(I_{k_i}, Q_U of step i), the first
  // k columns of the product the blocked loop accumulates into U.  Step i changes only the
  // block U(k_i:m, k_i:k), so the chain costs O(m k b) per step instead of O(m^2 b); the
  // block's input is kept for the reverse.
  eye_kernel<<<grid_of(m * (int64_t)k), 256, 0, c.st>>>(m, k, U, m);
  note_launch();
  double* wk = pool.get((size_t)b * k);
  double* wk2 = pool.get((size_t)b * k);
  if (!wk || !wk2) return RANDUTV_ENOMEM;
  for (int i = s - 1; i >= 0; --i) {
    StepState& S = st[i];
    const int64_t r = S.rm, cc = k - S.k;
    double* X = U + S.k + S.k * m;
    S.Xin = pool.get((size_t)r * cc);
    if (!S.Xin) return RANDUTV_ENOMEM;
    RUTV_TRY(copy(c, S.Xin, r, X, m, r, cc));
    RUTV_TRY(G(c, true, false, b, cc, r, 1.0, S.WU, r, X, m, 0.0, wk, b));      // W^T X
    RUTV_TRY(G(c, false, false, b, cc, b, 1.0, S.SU, b, wk, b, 0.0, wk2, b));   // S W^T X
    RUTV_TRY(G(c, false, false, r, cc, b, -1.0, S.WU, r, wk2, b, 1.0, X, m));   // Q_U X
  }
  return 0;
}

int lowrank_ctx(LCtx& c, void* stream) {
  c.st = (cudaStream_t)stream;
  Arena ar;
  const size_t gsb = dgemm_scratch_bytes(16384, 256);
  RUTV_TRY(scratch_reserve(gsb + householder_scratch_bytes(256) + 8192, &ar));
  c.gs = (double*)ar.take(gsb);
  c.gsb = gsb;
  c.qr = (char*)ar.take(householder_scratch_bytes(256));
  RUTV_TRY(status_words(&c.status));
  RUTV_CK(cudaMemsetAsync(c.status, 0, 64 * sizeof(unsigned), c.st));
  return 0;
}

}  // namespace

extern "C" {

int randutv_lowrank(int64_t m, int64_t n, const double* A, int64_t lda, int k, int b, int q,
                    uint64_t seed, double* Ak, void* stream) {
  RUTV_TRY(check_args(m, n, A, lda, k, b, q));
  if (!Ak) return -9;
  LCtx c;
  RUTV_TRY(lowrank_ctx(c, stream));
  Pool pool;
  double* U = pool.get((size_t)m * m);
  double* ap = pool.get(512);
  double* UtA = pool.get((size_t)k * n);
  if (!U || !ap || !UtA) return RANDUTV_ENOMEM;
  std::vector<StepState> st;
  RUTV_TRY(lowrank_forward(c, pool, m, n, A, lda, k, b, q, seed, st, U, ap));
  RUTV_TRY(G(c, true, false, k, n, m, 1.0, U, m, A, lda, 0.0, UtA, k));
  RUTV_TRY(G(c, false, false, m, n, k, 1.0, U, m, UtA, k, 0.0, Ak, m));
  RUTV_CK(cudaStreamSynchronize(c.st));  // the pool is freed on return
  unsigned h = 0;
  RUTV_CK(cudaMemcpy(&h, c.status, sizeof h, cudaMemcpyDeviceToHost));
  return (int)h;
}

int randutv_lowrank_backward(int64_t m, int64_t n, const double* A, int64_t lda, int k, int b,
                             int q, uint64_t seed, const double* dAk, double* dA, void* stream) {
  RUTV_TRY(check_args(m, n, A, lda, k, b, q));
  if (!dAk) return -9;
  if (!dA) return -10;
  LCtx c;
  RUTV_TRY(lowrank_ctx(c, stream));
  Pool pool;
  const int64_t big = m > n ? m : n;
  double* U = pool.get((size_t)m * m);
  double* ap = pool.get(1024);
  double* Ub = pool.get((size_t)m * m);
  double* UtA = pool.get((size_t)k * n);
  double* t1 = pool.get((size_t)big * b);
  double* t2 = pool.get((size_t)big * b);
  double* t3 = pool.get((size_t)big * b);
  double* Wb = pool.get((size_t)big * b);
  double* Sb = pool.get((size_t)b * b);
  double* Gb = pool.get((size_t)b * b);
  double* lws = pool.get((size_t)4 * b * b);  // larft_reverse workspace
  double* taub = pool.get(b);
  double* Pb = pool.get((size_t)big * b);
  double* Mb = pool.get((size_t)m * n);
  double* Nb = pool.get((size_t)m * n);
  double* Ob = pool.get((size_t)m * big);  // holds m x n and m x rm adjoints
  if (!U || !ap || !Ub || !UtA || !t1 || !t2 || !t3 || !Wb || !Sb || !Gb || !lws || !taub || !Pb ||
      !Mb || !Nb || !Ob)
    return RANDUTV_ENOMEM;
  std::vector<StepState> st;
  RUTV_TRY(lowrank_forward(c, pool, m, n, A, lda, k, b, q, seed, st, U, ap));
  // A_k = U_k (U_k^T A):  dA = U_k (U_k^T dAk) + (through U_k)
  // Ub_k = dAk (A^T U_k) + A (dAk^T U_k)
  RUTV_TRY(zero(c, Ub, (size_t)m * m));
  double* AtU = pool.get((size_t)n * k);
  double* AkU = pool.get((size_t)n * k);
  if (!AtU || !AkU) return RANDUTV_ENOMEM;
  RUTV_TRY(G(c, true, false, n, k, m, 1.0, A, lda, U, m, 0.0, AtU, n));
  RUTV_TRY(G(c, true, false, n, k, m, 1.0, dAk, m, U, m, 0.0, AkU, n));
  RUTV_TRY(G(c, false, false, m, k, n, 1.0, dAk, m, AtU, n, 0.0, Ub, m));
  RUTV_TRY(G(c, false, false, m, k, n, 1.0, A, lda, AkU, n, 1.0, Ub, m));
  RUTV_TRY(G(c, true, false, k, n, m, 1.0, U, m, dAk, m, 0.0, UtA, k));
  RUTV_TRY(G(c, false, false, m, n, k, 1.0, U, m, UtA, k, 0.0, dA, m));
  // The U_k chain backwards (its forward ran from the last step to the first, so its reverse
  // runs from the first): the block X_i = Q_U X_{i+1} with Q_U = I - W S W^T is the left
  // application X -> Q'^T X with Q' = I - W S^T W^T, whose adjoint left_apply_rev gives
  // (with S^T in place of S, and the S adjoint transposed back).  The W and S adjoints of each
  // step are kept for the step's panel-QR reverse below.
  const int ns = (int)st.size();
  std::vector<double*> WbU(ns), SbU(ns);
  double* SUt = pool.get((size_t)b * b);
  double* SbUt = pool.get((size_t)b * b);
  if (!SUt || !SbUt) return RANDUTV_ENOMEM;
  for (int i = 0; i < ns; ++i) {
    StepState& S = st[i];
    const int64_t r = S.rm, cc = k - S.k;
    WbU[i] = pool.get((size_t)r * b);
    SbU[i] = pool.get((size_t)b * b);
    if (!WbU[i] || !SbU[i]) return RANDUTV_ENOMEM;
    RUTV_TRY(zero(c, WbU[i], (size_t)r * b));
    RUTV_TRY(zero(c, SbUt, (size_t)b * b));
    transpose_kernel<<<grid_of((int64_t)b * b), 256, 0, c.st>>>(b, S.SU, SUt);
    note_launch();
    double* Xb = Ub + S.k + S.k * m;  // adjoint of the block, updated in place
    RUTV_TRY(left_apply_rev(c, r, cc, b, S.Xin, r, Xb, m, S.WU, SUt, Xb, m, WbU[i], SbUt, t1, t2,
                            t3));
    transpose_kernel<<<grid_of((int64_t)b * b), 256, 0, c.st>>>(b, SbUt, SbU[i]);
    note_launch();
  }
  RUTV_CK(cudaGetLastError());
  // adjoint of the input of the step after the last one: zero
  double* Mb_next = nullptr;
  for (int i = ns - 1; i >= 0; --i) {
    StepState& S = st[i];
    const int64_t rm = S.rm, rn = S.rn, nc = rn - b;
    // ---- the step's W_U and S_U adjoints start from the U_k chain's
    RUTV_TRY(copy(c, Wb, rm, WbU[i], rm, rm, b));
    RUTV_TRY(copy(c, Sb, b, SbU[i], b, b, b));
    RUTV_TRY(zero(c, taub, b));
    // ---- M_{i+1} = (Q_U^T N(:, b:))(b:, b:)
    RUTV_TRY(zero(c, Ob, (size_t)rm * nc));
    if (Mb_next) RUTV_TRY(copy(c, Ob + b, rm, Mb_next, rm - b, rm - b, nc));
    RUTV_TRY(zero(c, Nb, (size_t)rm * rn));
    RUTV_TRY(left_apply_rev(c, rm, nc, b, S.N + b * rm, rm, Ob, rm, S.WU, S.SU, Nb + b * rm, rm,
                            Wb, Sb, t1, t2, t3, S.WN));
    // ---- panel QR of N(:, 0:b)
    RUTV_TRY(larft_reverse(c, rm, b, S.WU, S.tauU, S.SU, S.GU, Sb, Wb, taub, Gb, lws));
    keep_strict_lower<<<grid_of(rm * b), 256, 0, c.st>>>(rm, b, Wb);
    note_launch();
    RUTV_TRY(hqr_reverse(c, rm, b, S.PU, S.WU, S.tauU, Wb, taub, Pb, ap));
    RUTV_TRY(copy(c, Nb, rm, Pb, rm, rm, b));
    // ---- N = M Q_V
    if (S.right) {
      RUTV_TRY(zero(c, Wb, (size_t)rn * b));
      RUTV_TRY(zero(c, Sb, (size_t)b * b));
      RUTV_TRY(zero(c, taub, b));
      RUTV_TRY(right_apply_rev(c, rm, rn, b, S.M, rm, Nb, rm, S.WV, S.SV, Mb, rm, Wb, Sb, t1, t2,
                               t3, S.MW));
      RUTV_TRY(larft_reverse(c, rn, b, S.WV, S.tauV, S.SV, S.GV, Sb, Wb, taub, Gb, lws));
      keep_strict_lower<<<grid_of(rn * b), 256, 0, c.st>>>(rn, b, Wb);
      note_launch();
      RUTV_TRY(hqr_reverse(c, rn, b, S.PV, S.WV, S.tauV, Wb, taub, Pb, ap));
      // Pb is the adjoint of Y_q; run the power chain backwards
      double* Yb = Pb;
      for (int it = q - 1; it >= 0; --it) {
        double* Yt = S.Ych + (size_t)it * rn * b;
        double* Zt = S.Zch + (size_t)it * rm * b;
        // Y_{t+1} = M^T Z_t: Mb += Z_t Yb^T, Zb = M Yb
        RUTV_TRY(G(c, false, true, rm, rn, b, 1.0, Zt, rm, Yb, rn, 1.0, Mb, rm));
        RUTV_TRY(G(c, false, false, rm, b, rn, 1.0, S.M, rm, Yb, rn, 0.0, t1, rm));
        // Z_t = M Y_t: Mb += Zb Y_t^T, Yb = M^T Zb
        RUTV_TRY(G(c, false, true, rm, rn, b, 1.0, t1, rm, Yt, rn, 1.0, Mb, rm));
        RUTV_TRY(G(c, true, false, rn, b, rm, 1.0, S.M, rm, t1, rm, 0.0, t2, rn));
        RUTV_TRY(copy(c, Yb, rn, t2, rn, rn, b));
      }
      // Y_0 = M^T G: Mb += G Yb^T (G redrawn)
      RUTV_TRY(launch_philox_normal(seed, (uint32_t)i, 0u, 0u, rm, b, t1, rm, c.st));
      RUTV_TRY(G(c, false, true, rm, rn, b, 1.0, t1, rm, Yb, rn, 1.0, Mb, rm));
    } else {
      RUTV_TRY(copy(c, Mb, rm, Nb, rm, rm, rn));
    }
    // Mb is the adjoint of this step's input; keep it for the step before
    if (i > 0) {
      double* keep = pool.get((size_t)rm * rn);
      if (!keep) return RANDUTV_ENOMEM;
      RUTV_TRY(copy(c, keep, rm, Mb, rm, rm, rn));
      Mb_next = keep;
    } else {
      axpy_kernel<<<grid_of(m * n), 256, 0, c.st>>>(m * n, 1.0, Mb, dA);
      note_launch();
    }
  }
  RUTV_CK(cudaStreamSynchronize(c.st));
  unsigned h = 0;
  RUTV_CK(cudaMemcpy(&h, c.status, sizeof h, cudaMemcpyDeviceToHost));
  return (int)h;
}

}  // extern "C"
