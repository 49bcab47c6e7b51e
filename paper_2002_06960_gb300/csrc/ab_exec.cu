// The executor of randUTV by blocks (§3.2.2-3.2.4): it runs the analyzer's
// task list (ab_tasks.cu) on b x b tiles, each task as a few FP64 kernels
// (the panel QR, WY factor, small SVD and dgemm of the blocked path, on
// tiles), on a set of streams.  Tasks are ordered by data flow only: every
// block keeps the event of its last writer and of its readers since, a task
// waits for the writers of what it reads and writes and for the readers of
// what it writes, and nothing joins the streams between block steps.  This
// is what the paper's runtime gets from algorithms-by-blocks: the tasks of
// step k+1 start as soon as their blocks are final, beside the end of step k.
//
// Tiles of A (T as it is formed), U and V are either views into the caller's
// device matrices (in HBM) or slots of an HBM cache of blocks whose backing
// store is host memory (out of HBM, the cache of §3.2.4 with least-recently-
// used replacement and write-back of modified blocks; copies run on two copy
// streams beside the compute streams).  The sketch, its products and the
// compact-WY and SVD factors stay in HBM.
//
// Operations on tiles (r_x rows of tile row x, c_x columns of tile column x,
// bi the width of block k; W S W^T the compact-WY form of a QR's Q):
//   dense QR of X (bi x bi):      X <- R, W (unit lower), S, WS = W S^T
//   td QR of [R; X_l]:            R <- R', W = [I; V], S, VS = V S^T
//   right, dense:  X <- X - (X W)(WS)^T
//   right, td:     t = X_k + X_l V;  X_k -= t S;  X_l -= t VS^T
//   left, dense:   t = W^T A_kj;  A_kj -= WS t
//   left, td:      t = A_kj + V^T A_ij;  A_kj -= S^T t;  A_ij -= VS t
#include <algorithm>
#include <cstring>
#include <unordered_map>
#include <vector>

#include "ab.h"
#include "common.cuh"
#include "kernels.h"

namespace rutv {
namespace {

constexpr int kMaxStreams = 16;

int grid_of(int64_t total) {
  int64_t g = (total + 255) / 256;
  const int64_t cap = (int64_t)dev_info().sms * 8;
  return (int)std::max<int64_t>(1, std::min(g, cap));
}

__global__ void ab_identity_kernel(int64_t rows, int64_t cols, double* X, int64_t ld) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < rows * cols;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % rows, j = e / rows;
    X[i + j * ld] = (i == j) ? 1.0 : 0.0;
  }
}

__global__ void ab_check_finite_kernel(int64_t rows, int64_t cols, const double* X, int64_t ld,
                                       unsigned* err) {
  int bad = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < rows * cols;
       e += (int64_t)gridDim.x * blockDim.x)
    bad |= !isfinite(X[(e % rows) + (e / rows) * ld]);
  if (__syncthreads_or(bad) && threadIdx.x == 0) {
    if (atomicCAS(err, 0u, (unsigned)RANDUTV_ENONFINITE) == 0u) atomicExch(err + 1, 102u);
  }
}

// X (rows x cols) <- 0 strictly below the diagonal (keep_upper) or
// X <- diag(D) (D non-null; rows == cols).
__global__ void ab_tri_kernel(int64_t rows, int64_t cols, double* X, int64_t ld, const double* D) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < rows * cols;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % rows, j = e / rows;
    if (D) X[i + j * ld] = (i == j) ? D[i] : 0.0;
    else if (i > j) X[i + j * ld] = 0.0;
  }
}

// Scratch of one compute stream: tile temporaries and the scratch of the
// kernels a task launches (QR partials and barrier words, dgemm split-K
// partials, SVD).
struct StreamRes {
  cudaStream_t st = nullptr;
  double *t = nullptr, *stack = nullptr, *W = nullptr, *tau = nullptr, *Gm = nullptr;
  char* qr = nullptr;
  double* gemm = nullptr;
  size_t gemm_bytes = 0;
  char* svd = nullptr;
  double* svd_gemm = nullptr;
  size_t svd_gemm_bytes = 0;
  unsigned* bar = nullptr;  // 2 barrier words of this stream's panel QRs
};

// Events, each shared by the block states that refer to it; an event is
// recorded again only once nothing refers to its last recording.
struct EventPool {
  std::vector<cudaEvent_t> ev;
  std::vector<int> ref;
  std::vector<int> idle;
  int get(int* out) {
    if (!idle.empty()) {
      *out = idle.back();
      idle.pop_back();
      return 0;
    }
    cudaEvent_t e;
    RUTV_CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    ev.push_back(e);
    ref.push_back(0);
    *out = (int)ev.size() - 1;
    return 0;
  }
  void hold(int i) { ++ref[i]; }
  void drop(int i) {
    if (--ref[i] == 0) idle.push_back(i);
  }
  ~EventPool() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
  }
};

struct BlockState {
  int writer = -1;
  std::vector<int> readers;
};

// Per-block ordering: before a task, the waits it needs; after it, its event.
struct Dataflow {
  EventPool pool;
  std::unordered_map<int64_t, BlockState> state;
  int wait_for(cudaStream_t st, const AbTask& a) {
    for (int x = 0; x < a.nin; ++x) {
      auto it = state.find(a.in[x]);
      if (it != state.end() && it->second.writer >= 0)
        RUTV_CK(cudaStreamWaitEvent(st, pool.ev[it->second.writer], 0));
    }
    for (int x = 0; x < a.nout; ++x) {
      auto it = state.find(a.out[x]);
      if (it == state.end()) continue;
      if (it->second.writer >= 0) RUTV_CK(cudaStreamWaitEvent(st, pool.ev[it->second.writer], 0));
      for (int r : it->second.readers) RUTV_CK(cudaStreamWaitEvent(st, pool.ev[r], 0));
    }
    return 0;
  }
  int done(cudaStream_t st, const AbTask& a) {
    int e = -1;
    RUTV_TRY(pool.get(&e));
    RUTV_CK(cudaEventRecord(pool.ev[e], st));
    pool.hold(e);  // held by this call until the states below take it
    for (int x = 0; x < a.nin; ++x) {
      bool written = false;
      for (int y = 0; y < a.nout; ++y) written |= (a.out[y] == a.in[x]);
      if (written) continue;
      BlockState& s = state[a.in[x]];
      s.readers.push_back(e);
      pool.hold(e);
    }
    for (int x = 0; x < a.nout; ++x) {
      BlockState& s = state[a.out[x]];
      if (s.writer >= 0) pool.drop(s.writer);
      for (int r : s.readers) pool.drop(r);
      s.readers.clear();
      s.writer = e;
      pool.hold(e);
    }
    pool.drop(e);
    return 0;
  }
  // the last event of a block (its writer), or -1
  int writer_of(int64_t blk) {
    auto it = state.find(blk);
    return it == state.end() ? -1 : it->second.writer;
  }
};

struct TileCache;  // out-of-HBM block cache (below)

struct AbExec {
  int64_t m = 0, n = 0, b = 0, p = 0;
  int q = 0;
  uint64_t seed = 0;
  std::vector<int64_t> rs, cs;  // tile starts (rows of A and U, columns of A and V)
  int64_t Mt = 0, Nt = 0;
  double *T = nullptr, *U = nullptr, *V = nullptr;  // device matrices (in HBM)
  double *G = nullptr, *Y = nullptr, *Z = nullptr;  // b x b tiles (ld b) by tile index
  double *Bs = nullptr, *Cs = nullptr;              // WY blocks: 3 b^2 each
  double *P = nullptr, *Q = nullptr, *D = nullptr;  // per step: U_s, V_s (ld bi), D
  unsigned* status = nullptr;
  StreamRes res[kMaxStreams];
  int nst = 0;
  Dataflow df;
  TileCache* cache = nullptr;
};

int64_t rows_of(const AbExec& x, int kind, int64_t i) {
  const std::vector<int64_t>& s = (kind == AB_V) ? x.cs : x.rs;
  return s[i + 1] - s[i];
}
int64_t cols_of(const AbExec& x, int kind, int64_t j) {
  const std::vector<int64_t>& s = (kind == AB_A || kind == AB_V) ? x.cs : x.rs;
  return s[j + 1] - s[j];
}

int cache_tile(AbExec& x, int64_t blk, double** ptr, int64_t* ld);  // below

// Device address and leading dimension of a block.
int tile(AbExec& x, int64_t blk, double** ptr, int64_t* ld) {
  const int kind = ab_kind(blk);
  const int64_t i = ab_bi(blk), j = ab_bj(blk), bb = x.b * x.b;
  switch (kind) {
    case AB_A:
      if (x.cache) return cache_tile(x, blk, ptr, ld);
      *ptr = x.T + x.rs[i] + x.cs[j] * x.m; *ld = x.m; return 0;
    case AB_U:
      if (x.cache) return cache_tile(x, blk, ptr, ld);
      *ptr = x.U + x.rs[i] + x.rs[j] * x.m; *ld = x.m; return 0;
    case AB_V:
      if (x.cache) return cache_tile(x, blk, ptr, ld);
      *ptr = x.V + x.cs[i] + x.cs[j] * x.n; *ld = x.n; return 0;
    case AB_G: *ptr = x.G + i * bb; *ld = x.b; return 0;
    case AB_Y: *ptr = x.Y + i * bb; *ld = x.b; return 0;
    case AB_Z: *ptr = x.Z + i * bb; *ld = x.b; return 0;
    case AB_B: *ptr = x.Bs + i * 3 * bb; *ld = x.b; return 0;
    case AB_C: *ptr = x.Cs + i * 3 * bb; *ld = x.b; return 0;
    case AB_P: *ptr = x.P + i * bb; *ld = 0; return 0;
    case AB_Q: *ptr = x.Q + i * bb; *ld = 0; return 0;
    default: return RANDUTV_EUNSUPPORTED;
  }
}

int gemm(StreamRes& r, bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha,
         const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* C,
         int64_t ldc) {
  return launch_dgemm(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, r.gemm, r.gemm_bytes,
                      r.st);
}

int copy2d(StreamRes& r, double* dst, int64_t ldd, const double* src, int64_t lds, int64_t rows,
           int64_t cols) {
  RUTV_CK(cudaMemcpy2DAsync(dst, (size_t)ldd * 8, src, (size_t)lds * 8, (size_t)rows * 8,
                            (size_t)cols, cudaMemcpyDeviceToDevice, r.st));
  return 0;
}

// The WY block of a QR: S (bi x bi, ld bi) at the base, W S^T (or V S^T) at
// b^2, W (or V) at 2 b^2, both with ld b.
struct WyBlock {
  double *S, *WS, *W;
};
WyBlock wy_block(const AbExec& x, double* base) {
  const int64_t bb = x.b * x.b;
  return WyBlock{base, base + bb, base + 2 * bb};
}

// Compact-WY factor of the r x bi reflectors Wsrc (ld r): S, W S^T, and a copy of
// rows w0 .. r-1 of W (all of them for a dense QR, the V rows for a td QR).
int make_wy(AbExec& x, StreamRes& r, int64_t rr, int64_t bi, const double* Wsrc, int64_t w0,
            WyBlock& o) {
  RUTV_TRY(gemm(r, true, false, bi, bi, rr, 1.0, Wsrc, rr, Wsrc, rr, 0.0, r.Gm, bi));
  RUTV_TRY(launch_wy_factor(bi, r.Gm, r.tau, o.S, r.st));
  RUTV_TRY(copy2d(r, o.W, x.b, Wsrc + w0, rr, rr - w0, bi));
  RUTV_TRY(gemm(r, false, true, rr - w0, bi, bi, 1.0, Wsrc + w0, rr, o.S, bi, 0.0, o.WS, x.b));
  return 0;
}

int run_task(AbExec& x, StreamRes& r, const AbTask& a) {
  const int64_t k = a.step, bi = x.cs[k + 1] - x.cs[k];
  double *X0 = nullptr, *X1 = nullptr, *X2 = nullptr, *X3 = nullptr;
  int64_t l0 = 0, l1 = 0, l2 = 0, l3 = 0;
  switch (a.op) {
    case OP_GEN: {
      const int64_t i = ab_bi(a.out[0]);
      RUTV_TRY(tile(x, a.out[0], &X0, &l0));
      return launch_philox_normal_rows(x.seed, (uint32_t)k, 0u, 0u, x.m - x.rs[k], x.rs[i] - x.rs[k],
                                       rows_of(x, AB_A, i), bi, X0, l0, r.st);
    }
    case OP_TN_OZ:
    case OP_TN_OO: {  // Y_j (+)= A_ij^T X_i
      const int64_t i = ab_bi(a.in[0]), j = ab_bj(a.in[0]);
      RUTV_TRY(tile(x, a.in[0], &X0, &l0));
      RUTV_TRY(tile(x, a.in[1], &X1, &l1));
      RUTV_TRY(tile(x, a.out[0], &X2, &l2));
      return gemm(r, true, false, cols_of(x, AB_A, j), bi, rows_of(x, AB_A, i), 1.0, X0, l0, X1, l1,
                  a.op == OP_TN_OO ? 1.0 : 0.0, X2, l2);
    }
    case OP_NN_OZ:
    case OP_NN_OO: {  // Z_i (+)= A_ij Y_j
      const int64_t i = ab_bi(a.in[0]), j = ab_bj(a.in[0]);
      RUTV_TRY(tile(x, a.in[0], &X0, &l0));
      RUTV_TRY(tile(x, a.in[1], &X1, &l1));
      RUTV_TRY(tile(x, a.out[0], &X2, &l2));
      return gemm(r, false, false, rows_of(x, AB_A, i), bi, cols_of(x, AB_A, j), 1.0, X0, l0, X1, l1,
                  a.op == OP_NN_OO ? 1.0 : 0.0, X2, l2);
    }
    case OP_QR_DENSE: {  // X (bi x bi) <- R; WY block of its reflectors
      RUTV_TRY(tile(x, a.in[0], &X0, &l0));
      RUTV_TRY(tile(x, a.out[1], &X1, &l1));
      WyBlock o = wy_block(x, X1);
      RUTV_TRY(launch_householder_qr(bi, bi, X0, l0, r.W, r.tau, r.qr, r.bar, x.status, r.st));
      return make_wy(x, r, bi, bi, r.W, 0, o);
    }
    case OP_QR_TD: {  // [R in X_k; X_l] -> R', W = [I; V]
      const int kind = ab_kind(a.in[1]);
      const int64_t rl = (kind == AB_Y) ? cols_of(x, AB_A, ab_bi(a.in[1]))
                                        : rows_of(x, AB_A, ab_bi(a.in[1]));
      const int64_t sr = bi + rl;
      RUTV_TRY(tile(x, a.in[0], &X0, &l0));
      RUTV_TRY(tile(x, a.in[1], &X1, &l1));
      RUTV_TRY(tile(x, a.out[2], &X2, &l2));
      WyBlock o = wy_block(x, X2);
      RUTV_TRY(copy2d(r, r.stack, sr, X0, l0, bi, bi));
      RUTV_TRY(copy2d(r, r.stack + bi, sr, X1, l1, rl, bi));
      RUTV_TRY(launch_householder_qr(sr, bi, r.stack, sr, r.W, r.tau, r.qr, r.bar, x.status, r.st));
      RUTV_TRY(copy2d(r, X0, l0, r.stack, sr, bi, bi));
      return make_wy(x, r, sr, bi, r.W, bi, o);
    }
    case OP_RIGHT_DENSE: {  // X <- X - (X W)(W S^T)^T
      RUTV_TRY(tile(x, a.in[1], &X1, &l1));
      RUTV_TRY(tile(x, a.out[0], &X2, &l2));
      const WyBlock o = wy_block(x, X1);
      const int64_t rows = rows_of(x, ab_kind(a.out[0]), ab_bi(a.out[0]));
      RUTV_TRY(gemm(r, false, false, rows, bi, bi, 1.0, X2, l2, o.W, x.b, 0.0, r.t, x.b));
      return gemm(r, false, true, rows, bi, bi, -1.0, r.t, x.b, o.WS, x.b, 1.0, X2, l2);
    }
    case OP_RIGHT_TD: {  // t = X_k + X_l V;  X_k -= t S;  X_l -= t (V S^T)^T
      const int kind = ab_kind(a.out[0]);
      RUTV_TRY(tile(x, a.in[1], &X1, &l1));
      RUTV_TRY(tile(x, a.out[0], &X2, &l2));
      RUTV_TRY(tile(x, a.out[1], &X3, &l3));
      const WyBlock o = wy_block(x, X1);
      const int64_t rows = rows_of(x, kind, ab_bi(a.out[0]));
      const int64_t rl = cols_of(x, kind, ab_bj(a.out[1]));
      RUTV_TRY(copy2d(r, r.t, x.b, X2, l2, rows, bi));
      RUTV_TRY(gemm(r, false, false, rows, bi, rl, 1.0, X3, l3, o.W, x.b, 1.0, r.t, x.b));
      RUTV_TRY(gemm(r, false, false, rows, bi, bi, -1.0, r.t, x.b, o.S, bi, 1.0, X2, l2));
      return gemm(r, false, true, rows, rl, bi, -1.0, r.t, x.b, o.WS, x.b, 1.0, X3, l3);
    }
    case OP_LEFT_DENSE: {  // t = W^T A_kj;  A_kj -= (W S^T) t
      RUTV_TRY(tile(x, a.in[1], &X1, &l1));
      RUTV_TRY(tile(x, a.out[0], &X2, &l2));
      const WyBlock o = wy_block(x, X1);
      const int64_t cj = cols_of(x, AB_A, ab_bj(a.out[0]));
      RUTV_TRY(gemm(r, true, false, bi, cj, bi, 1.0, o.W, x.b, X2, l2, 0.0, r.t, x.b));
      return gemm(r, false, false, bi, cj, bi, -1.0, o.WS, x.b, r.t, x.b, 1.0, X2, l2);
    }
    case OP_LEFT_TD: {  // t = A_kj + V^T A_ij;  A_kj -= S^T t;  A_ij -= (V S^T) t
      RUTV_TRY(tile(x, a.in[1], &X1, &l1));
      RUTV_TRY(tile(x, a.out[0], &X2, &l2));
      RUTV_TRY(tile(x, a.out[1], &X3, &l3));
      const WyBlock o = wy_block(x, X1);
      const int64_t cj = cols_of(x, AB_A, ab_bj(a.out[0]));
      const int64_t ri = rows_of(x, AB_A, ab_bi(a.out[1]));
      RUTV_TRY(copy2d(r, r.t, x.b, X2, l2, bi, cj));
      RUTV_TRY(gemm(r, true, false, bi, cj, ri, 1.0, o.W, x.b, X3, l3, 1.0, r.t, x.b));
      RUTV_TRY(gemm(r, true, false, bi, cj, bi, -1.0, o.S, bi, r.t, x.b, 1.0, X2, l2));
      return gemm(r, false, false, ri, cj, bi, -1.0, o.WS, x.b, r.t, x.b, 1.0, X3, l3);
    }
    case OP_KEEP_UPPER: {
      RUTV_TRY(tile(x, a.out[0], &X0, &l0));
      ab_tri_kernel<<<grid_of(bi * bi), 256, 0, r.st>>>(bi, bi, X0, l0, nullptr);
      note_launch();
      RUTV_CK(cudaGetLastError());
      return 0;
    }
    case OP_SET_ZERO: {
      RUTV_TRY(tile(x, a.out[0], &X0, &l0));
      const int64_t rows = rows_of(x, AB_A, ab_bi(a.out[0]));
      RUTV_CK(cudaMemset2DAsync(X0, (size_t)l0 * 8, 0, (size_t)rows * 8, (size_t)bi, r.st));
      return 0;
    }
    case OP_SVD: {  // A_kk = P diag(D) Q^T -> A_kk = diag(D)
      RUTV_TRY(tile(x, a.in[0], &X0, &l0));
      RUTV_TRY(tile(x, a.out[1], &X1, &l1));
      RUTV_TRY(tile(x, a.out[2], &X2, &l2));
      double* D = x.D + k * x.b;
      RUTV_TRY(launch_small_svd((int)bi, X0, l0, D, X1, X2, x.status + 8, r.svd, r.svd_gemm,
                                r.svd_gemm_bytes, r.st));
      ab_tri_kernel<<<grid_of(bi * bi), 256, 0, r.st>>>(bi, bi, X0, l0, D);
      note_launch();
      RUTV_CK(cudaGetLastError());
      return 0;
    }
    case OP_ABTA: {  // A_kj <- P^T A_kj
      RUTV_TRY(tile(x, a.in[0], &X0, &l0));
      RUTV_TRY(tile(x, a.out[0], &X2, &l2));
      const int64_t cj = cols_of(x, AB_A, ab_bj(a.out[0]));
      RUTV_TRY(gemm(r, true, false, bi, cj, bi, 1.0, X0, bi, X2, l2, 0.0, r.t, x.b));
      return copy2d(r, X2, l2, r.t, x.b, bi, cj);
    }
    case OP_AABT:
    case OP_AAB: {  // X <- X V_s (A above the block, V) or X <- X U_s (U)
      RUTV_TRY(tile(x, a.out[0], &X2, &l2));
      RUTV_TRY(tile(x, a.in[1], &X1, &l1));
      const int64_t rows = rows_of(x, ab_kind(a.out[0]), ab_bi(a.out[0]));
      RUTV_TRY(gemm(r, false, false, rows, bi, bi, 1.0, X2, l2, X1, bi, 0.0, r.t, x.b));
      return copy2d(r, X2, l2, r.t, x.b, rows, bi);
    }
    default:
      return RANDUTV_EUNSUPPORTED;
  }
}

}  // namespace
}  // namespace rutv

// ------------------------------------------------------ out-of-HBM cache
namespace rutv {
namespace {

// Slots of b x b doubles (ld b) in HBM, each holding one tile of A, U or V,
// whose home is the caller's host matrix.  Decisions are taken on the host
// in task order (least recently used, ties to the lowest slot); the copies
// run on the copy streams, ordered against the compute streams by the
// blocks' events: a slot is reloaded only after every task that used its
// old block and after the old block's write-back, and a task runs only
// after its blocks' loads.
struct TileCache {
  int64_t nslots = 0;
  double* base = nullptr;
  std::vector<int64_t> blk, last;
  std::vector<char> dirty;
  std::unordered_map<int64_t, int64_t> where;
  std::unordered_map<int64_t, char> checked;  // A tiles whose first load was checked for NaN/Inf
  double *Ah = nullptr, *Uh = nullptr, *Vh = nullptr;
  int64_t lda = 0;
  cudaStream_t h2d = nullptr, d2h = nullptr;
  int64_t reads = 0, writes = 0, tick = 0;
  double bytes = 0.0;
};

// Host address (ld) and extent of a tile of A, U or V.
void host_tile(const AbExec& x, int64_t blk, double** h, int64_t* ldh, int64_t* rows, int64_t* cols) {
  const TileCache& c = *x.cache;
  const int kind = ab_kind(blk);
  const int64_t i = ab_bi(blk), j = ab_bj(blk);
  *rows = rows_of(x, kind, i);
  *cols = cols_of(x, kind, j);
  if (kind == AB_A) { *h = c.Ah + x.rs[i] + x.cs[j] * c.lda; *ldh = c.lda; }
  else if (kind == AB_U) { *h = c.Uh + x.rs[i] + x.rs[j] * x.m; *ldh = x.m; }
  else { *h = c.Vh + x.cs[i] + x.cs[j] * x.n; *ldh = x.n; }
}

int cache_tile(AbExec& x, int64_t blk, double** ptr, int64_t* ld) {
  auto it = x.cache->where.find(blk);
  if (it == x.cache->where.end()) {
    set_last_error("block cache: a task's block is not resident");
    return RANDUTV_EUNSUPPORTED;
  }
  *ptr = x.cache->base + it->second * x.b * x.b;
  *ld = x.b;
  return 0;
}

bool in_task(const AbTask& a, int64_t blk) {
  for (int t = 0; t < a.nin; ++t)
    if (a.in[t] == blk) return true;
  for (int t = 0; t < a.nout; ++t)
    if (a.out[t] == blk) return true;
  return false;
}

// Frees a slot for the task's block `blk` and fills it (load = true: read
// from the host).  The block's new writer event is the copy (or, for an
// output-only block, the point after which the slot is free).
int cache_place(AbExec& x, const AbTask& a, int64_t blk, bool load) {
  TileCache& c = *x.cache;
  Dataflow& df = x.df;
  int64_t s = -1;
  for (int64_t t = 0; t < c.nslots && s < 0; ++t)
    if (c.blk[t] < 0) s = t;
  if (s < 0) {
    for (int64_t t = 0; t < c.nslots; ++t)
      if (!in_task(a, c.blk[t]) && (s < 0 || c.last[t] < c.last[s])) s = t;
    if (s < 0) {
      set_last_error("block cache: fewer slots than one task's blocks");
      return RANDUTV_EUNSUPPORTED;
    }
  }
  double* slot = c.base + s * x.b * x.b;
  // the copy stream waits for every user of the slot's old block
  if (c.blk[s] >= 0) {
    const int64_t old = c.blk[s];
    BlockState& os = df.state[old];
    if (c.dirty[s]) {  // write the old block back to its host home
      double* h; int64_t ldh, rr, cc;
      host_tile(x, old, &h, &ldh, &rr, &cc);
      if (os.writer >= 0) RUTV_CK(cudaStreamWaitEvent(c.d2h, df.pool.ev[os.writer], 0));
      RUTV_CK(cudaMemcpy2DAsync(h, (size_t)ldh * 8, slot, (size_t)x.b * 8, (size_t)rr * 8,
                                (size_t)cc, cudaMemcpyDeviceToHost, c.d2h));
      ++c.writes;
      c.bytes += 8.0 * rr * cc;
      int e = -1;
      RUTV_TRY(df.pool.get(&e));
      RUTV_CK(cudaEventRecord(df.pool.ev[e], c.d2h));
      // the old block's home now follows this copy
      if (os.writer >= 0) df.pool.drop(os.writer);
      os.writer = e;
      df.pool.hold(e);
    }
    if (os.writer >= 0) RUTV_CK(cudaStreamWaitEvent(c.h2d, df.pool.ev[os.writer], 0));
    for (int r : os.readers) {
      RUTV_CK(cudaStreamWaitEvent(c.h2d, df.pool.ev[r], 0));
      df.pool.drop(r);
    }
    os.readers.clear();
    c.where.erase(old);
  }
  // the new block: its host home must be final (an earlier write-back)
  BlockState& ns = df.state[blk];
  if (ns.writer >= 0) RUTV_CK(cudaStreamWaitEvent(c.h2d, df.pool.ev[ns.writer], 0));
  for (int r : ns.readers) df.pool.drop(r);
  ns.readers.clear();
  if (load) {
    double* h; int64_t ldh, rr, cc;
    host_tile(x, blk, &h, &ldh, &rr, &cc);
    RUTV_CK(cudaMemcpy2DAsync(slot, (size_t)x.b * 8, h, (size_t)ldh * 8, (size_t)rr * 8,
                              (size_t)cc, cudaMemcpyHostToDevice, c.h2d));
    ++c.reads;
    c.bytes += 8.0 * rr * cc;
    if (ab_kind(blk) == AB_A && !c.checked[blk]) {
      c.checked[blk] = 1;
      ab_check_finite_kernel<<<grid_of(rr * cc), 256, 0, c.h2d>>>(rr, cc, slot, x.b, x.status);
      note_launch();
      RUTV_CK(cudaGetLastError());
    }
  }
  int e = -1;
  RUTV_TRY(df.pool.get(&e));
  RUTV_CK(cudaEventRecord(df.pool.ev[e], c.h2d));
  if (ns.writer >= 0) df.pool.drop(ns.writer);
  ns.writer = e;
  df.pool.hold(e);
  c.blk[s] = blk;
  c.dirty[s] = 0;
  c.where[blk] = s;
  return 0;
}

int cache_prepare(AbExec& x, const AbTask& a) {
  TileCache& c = *x.cache;
  auto matrix = [](int64_t blk) {
    const int k = ab_kind(blk);
    return k == AB_A || k == AB_U || k == AB_V;
  };
  for (int t = 0; t < a.nin; ++t)
    if (matrix(a.in[t]) && !c.where.count(a.in[t])) RUTV_TRY(cache_place(x, a, a.in[t], true));
  for (int t = 0; t < a.nout; ++t)
    if (matrix(a.out[t]) && !c.where.count(a.out[t])) RUTV_TRY(cache_place(x, a, a.out[t], false));
  ++c.tick;
  for (int t = 0; t < a.nin; ++t) {
    auto it = c.where.find(a.in[t]);
    if (it != c.where.end()) c.last[it->second] = c.tick;
  }
  for (int t = 0; t < a.nout; ++t) {
    auto it = c.where.find(a.out[t]);
    if (it != c.where.end()) {
      c.last[it->second] = c.tick;
      c.dirty[it->second] = 1;
    }
  }
  return 0;
}

// Writes every modified block back to its host home.
int cache_flush(AbExec& x) {
  TileCache& c = *x.cache;
  for (int64_t s = 0; s < c.nslots; ++s) {
    if (c.blk[s] < 0 || !c.dirty[s]) continue;
    double* h; int64_t ldh, rr, cc;
    host_tile(x, c.blk[s], &h, &ldh, &rr, &cc);
    const int w = x.df.writer_of(c.blk[s]);
    if (w >= 0) RUTV_CK(cudaStreamWaitEvent(c.d2h, x.df.pool.ev[w], 0));
    RUTV_CK(cudaMemcpy2DAsync(h, (size_t)ldh * 8, c.base + s * x.b * x.b, (size_t)x.b * 8,
                              (size_t)rr * 8, (size_t)cc, cudaMemcpyDeviceToHost, c.d2h));
    ++c.writes;
    c.bytes += 8.0 * rr * cc;
    c.dirty[s] = 0;
  }
  return 0;
}

}  // namespace
}  // namespace rutv

// ------------------------------------------------------------ the driver
namespace rutv {
namespace {

struct AbStreams {
  cudaStream_t st[kMaxStreams] = {};
  cudaStream_t h2d = nullptr, d2h = nullptr;
  cudaEvent_t join = nullptr, fin[kMaxStreams + 2] = {};
  bool ok = false;
};
AbStreams g_ab[64];

int ab_streams(AbStreams** out) {
  int dev = 0;
  RUTV_CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return RANDUTV_EUNSUPPORTED;
  AbStreams& s = g_ab[dev];
  if (!s.ok) {
    for (auto& x : s.st) RUTV_CK(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking));
    RUTV_CK(cudaStreamCreateWithFlags(&s.h2d, cudaStreamNonBlocking));
    RUTV_CK(cudaStreamCreateWithFlags(&s.d2h, cudaStreamNonBlocking));
    RUTV_CK(cudaEventCreateWithFlags(&s.join, cudaEventDisableTiming));
    for (auto& e : s.fin) RUTV_CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    s.ok = true;
  }
  *out = &s;
  return 0;
}

size_t gemm_bytes_of(int64_t b) { return (size_t)16 * (size_t)b * (size_t)b * 8; }

// Device bytes of everything but the tiles of A, U, V: the sketch tiles, the
// WY and SVD factors, and per stream the tile temporaries and kernel scratch.
size_t ab_fixed_bytes(int64_t Mt, int64_t Nt, int64_t steps, int64_t b, int nst) {
  const size_t bb = (size_t)b * (size_t)b * 8;
  const size_t mx = (size_t)std::max(Mt, Nt);
  size_t s = 0;
  auto add = [&](size_t x) { s += (x + 255) & ~size_t(255); };
  add(3 * mx * bb);                      // G, Y, Z
  add(3 * (size_t)Nt * bb);              // B blocks
  add(3 * (size_t)Mt * bb);              // C blocks
  add(2 * (size_t)steps * bb);           // P, Q
  add((size_t)steps * (size_t)b * 8);    // D
  for (int i = 0; i < nst; ++i) {
    add(bb);                             // t
    add(2 * bb);                         // stack
    add(2 * bb);                         // W
    add((size_t)b * 8);                  // tau
    add(bb);                             // Gm
    add(householder_scratch_bytes(b));
    add(gemm_bytes_of(b));
    add(small_svd_scratch_bytes((int)b));
    add(gemm_bytes_of(b));
    add(256);                            // barrier words
  }
  return s + 4096;
}

int ab_setup(AbExec& x, Arena& ar, int nst, AbStreams* ss) {
  const size_t bb = (size_t)x.b * (size_t)x.b * 8;
  const int64_t steps = (x.p + x.b - 1) / x.b, mx = std::max(x.Mt, x.Nt);
  x.G = (double*)ar.take(mx * bb);
  x.Y = (double*)ar.take(mx * bb);
  x.Z = (double*)ar.take(mx * bb);
  x.Bs = (double*)ar.take(3 * (size_t)x.Nt * bb);
  x.Cs = (double*)ar.take(3 * (size_t)x.Mt * bb);
  x.P = (double*)ar.take((size_t)steps * bb);
  x.Q = (double*)ar.take((size_t)steps * bb);
  x.D = (double*)ar.take((size_t)steps * x.b * 8);
  x.nst = nst;
  for (int i = 0; i < nst; ++i) {
    StreamRes& r = x.res[i];
    r.st = ss->st[i];
    r.t = (double*)ar.take(bb);
    r.stack = (double*)ar.take(2 * bb);
    r.W = (double*)ar.take(2 * bb);
    r.tau = (double*)ar.take((size_t)x.b * 8);
    r.Gm = (double*)ar.take(bb);
    r.qr = (char*)ar.take(householder_scratch_bytes(x.b));
    r.gemm_bytes = gemm_bytes_of(x.b);
    r.gemm = (double*)ar.take(r.gemm_bytes);
    r.svd = (char*)ar.take(small_svd_scratch_bytes((int)x.b));
    r.svd_gemm_bytes = gemm_bytes_of(x.b);
    r.svd_gemm = (double*)ar.take(r.svd_gemm_bytes);
    r.bar = (unsigned*)ar.take(256);
  }
  return 0;
}

// Runs the task list; the compute streams and the copy streams start after
// the work queued on `caller` and `caller` continues after all of them.
int ab_run(AbExec& x, AbStreams* ss, cudaStream_t caller) {
  RUTV_CK(cudaEventRecord(ss->join, caller));
  for (int i = 0; i < x.nst; ++i) RUTV_CK(cudaStreamWaitEvent(ss->st[i], ss->join, 0));
  RUTV_CK(cudaStreamWaitEvent(ss->h2d, ss->join, 0));
  RUTV_CK(cudaStreamWaitEvent(ss->d2h, ss->join, 0));
  const std::vector<AbTask> tasks = ab_analyze(x.m, x.n, x.b, x.q, x.U != nullptr ||
                                               (x.cache && x.cache->Uh), x.V != nullptr ||
                                               (x.cache && x.cache->Vh));
  for (const AbTask& a : tasks) {
    // every block keeps to one stream: its successive writers need no event
    const uint64_t h = (uint64_t)a.out[0] * 0x9E3779B97F4A7C15ull;
    StreamRes& r = x.res[(h >> 32) % (uint64_t)x.nst];
    if (x.cache) RUTV_TRY(cache_prepare(x, a));
    RUTV_TRY(x.df.wait_for(r.st, a));
    RUTV_TRY(run_task(x, r, a));
    RUTV_TRY(x.df.done(r.st, a));
  }
  if (x.cache) RUTV_TRY(cache_flush(x));
  for (int i = 0; i < x.nst; ++i) {
    RUTV_CK(cudaEventRecord(ss->fin[i], ss->st[i]));
    RUTV_CK(cudaStreamWaitEvent(caller, ss->fin[i], 0));
  }
  RUTV_CK(cudaEventRecord(ss->fin[kMaxStreams], ss->h2d));
  RUTV_CK(cudaStreamWaitEvent(caller, ss->fin[kMaxStreams], 0));
  RUTV_CK(cudaEventRecord(ss->fin[kMaxStreams + 1], ss->d2h));
  RUTV_CK(cudaStreamWaitEvent(caller, ss->fin[kMaxStreams + 1], 0));
  return 0;
}

void ab_geometry(AbExec& x, int64_t m, int64_t n, int64_t b, int q, uint64_t seed) {
  x.m = m;
  x.n = n;
  x.p = std::min(m, n);
  x.b = std::min<int64_t>(b, x.p);
  x.q = q;
  x.seed = seed;
  x.rs = ab_tile_starts(m, x.p, x.b);
  x.cs = ab_tile_starts(n, x.p, x.b);
  x.Mt = (int64_t)x.rs.size() - 1;
  x.Nt = (int64_t)x.cs.size() - 1;
}

}  // namespace
}  // namespace rutv

using namespace rutv;

extern "C" {

int randutv_factor_ab(int64_t m, int64_t n, const double* A, int64_t lda, int b, int q,
                      uint64_t seed, double* U, double* T, double* V, int nstreams, void* stream) {
  if (m < 1) return -1;
  if (n < 1) return -2;
  if (!A) return -3;
  if (lda < m) return -4;
  if (b < 1 || b > 256) return -5;
  if (q < 0 || q > 16) return -6;
  if (!T) return -9;
  if (nstreams < 1 || nstreams > kMaxStreams) return -11;
  if (std::max(m, n) / std::min<int64_t>(b, std::min(m, n)) + 2 >= (1 << 20))
    return RANDUTV_EUNSUPPORTED;
  cudaStream_t st = (cudaStream_t)stream;
  AbStreams* ss = nullptr;
  RUTV_TRY(ab_streams(&ss));
  AbExec x;
  ab_geometry(x, m, n, b, q, seed);
  Arena ar;
  RUTV_TRY(scratch_reserve(ab_fixed_bytes(x.Mt, x.Nt, (x.p + x.b - 1) / x.b, x.b, nstreams), &ar));
  RUTV_TRY(status_words(&x.status));
  RUTV_TRY(ab_setup(x, ar, nstreams, ss));
  x.T = T;
  x.U = U;
  x.V = V;
  RUTV_CK(cudaMemsetAsync(x.status, 0, 64 * sizeof(unsigned), st));
  if (T != A)
    RUTV_CK(cudaMemcpy2DAsync(T, (size_t)m * 8, A, (size_t)lda * 8, (size_t)m * 8, (size_t)n,
                              cudaMemcpyDeviceToDevice, st));
  ab_check_finite_kernel<<<grid_of(m * n), 256, 0, st>>>(m, n, T, m, x.status);
  if (U) ab_identity_kernel<<<grid_of(m * m), 256, 0, st>>>(m, m, U, m);
  if (V) ab_identity_kernel<<<grid_of(n * n), 256, 0, st>>>(n, n, V, n);
  note_launch(1 + (U ? 1 : 0) + (V ? 1 : 0));
  RUTV_CK(cudaGetLastError());
  // a matrix with NaN or Inf is not factored
  unsigned h = 0;
  RUTV_CK(cudaMemcpyAsync(&h, x.status, sizeof h, cudaMemcpyDeviceToHost, st));
  RUTV_CK(cudaStreamSynchronize(st));
  if (h != 0) return 0;  // the status stays in the device word (randutv_stream_status)
  return ab_run(x, ss, st);
}

size_t randutv_ooc_ab_min_device_bytes(int64_t m, int64_t n, int b, int nstreams) {
  if (m < 1 || n < 1 || b < 1 || nstreams < 1 || nstreams > kMaxStreams) return 0;
  AbExec x;
  ab_geometry(x, m, n, b, 0, 0);
  return ab_fixed_bytes(x.Mt, x.Nt, (x.p + x.b - 1) / x.b, x.b, nstreams) +
         (size_t)8 * (size_t)x.b * (size_t)x.b * 8 + 8192;
}

int randutv_factor_ooc_ab(int64_t m, int64_t n, double* A, int64_t lda, int b, int q,
                          uint64_t seed, double* U, double* V, size_t device_bytes, int nstreams,
                          int64_t* io, void* stream) {
  if (m < 1) return -1;
  if (n < 1) return -2;
  if (!A) return -3;
  if (lda < m) return -4;
  if (b < 1 || b > 256) return -5;
  if (q < 0 || q > 16) return -6;
  if (nstreams < 1 || nstreams > kMaxStreams) return -11;
  if (device_bytes < randutv_ooc_ab_min_device_bytes(m, n, b, nstreams)) return -10;
  if (std::max(m, n) / std::min<int64_t>(b, std::min(m, n)) + 2 >= (1 << 20))
    return RANDUTV_EUNSUPPORTED;
  cudaStream_t st = (cudaStream_t)stream;
  AbStreams* ss = nullptr;
  RUTV_TRY(ab_streams(&ss));
  AbExec x;
  ab_geometry(x, m, n, b, q, seed);
  const size_t fixed = ab_fixed_bytes(x.Mt, x.Nt, (x.p + x.b - 1) / x.b, x.b, nstreams);
  const size_t slot = (size_t)x.b * (size_t)x.b * 8;
  TileCache c;
  c.nslots = (int64_t)((device_bytes - fixed - 8192) / slot);
  Arena ar;
  RUTV_TRY(scratch_reserve(fixed + (size_t)c.nslots * slot + 8192, &ar));
  RUTV_TRY(status_words(&x.status));
  RUTV_TRY(ab_setup(x, ar, nstreams, ss));
  c.base = (double*)ar.take((size_t)c.nslots * slot);
  c.blk.assign(c.nslots, -1);
  c.last.assign(c.nslots, -1);
  c.dirty.assign(c.nslots, 0);
  c.Ah = A;
  c.Uh = U;
  c.Vh = V;
  c.lda = lda;
  c.h2d = ss->h2d;
  c.d2h = ss->d2h;
  x.cache = &c;
  RUTV_CK(cudaMemsetAsync(x.status, 0, 64 * sizeof(unsigned), st));
  RUTV_CK(cudaStreamSynchronize(st));
  // U = I, V = I in their host homes
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
  RUTV_TRY(ab_run(x, ss, st));
  RUTV_CK(cudaStreamSynchronize(st));
  if (io) {
    io[0] = c.reads;
    io[1] = c.writes;
    io[2] = (int64_t)c.bytes;
  }
  unsigned h = 0;
  RUTV_CK(cudaMemcpy(&h, x.status, sizeof h, cudaMemcpyDeviceToHost));
  return (int)h;
}

}  // extern "C"
