// Host driver and C-ABI of the randUTV library.
//
// One block step (§3.1 steps 1-6; update list of Fig. 2), all in FP64 on the
// device, with k the offset of the block, bi = min(b, min(m,n) - k) its width,
// rm = m - k and rn = n - k:
//   right transform (when rn > bi):
//     G = sketch(seed, step)                  rm x bi       philox_normal
//     Y = T22^T G, then q times Y = T22^T (T22 Y)            dgemm
//     [W, tau] = QR(Y); S = wy(W, tau)                      householder, wy_factor
//     T(:, k:) -= (T(:, k:) W) (W S^T)^T, likewise V(:, k:)  dgemm (all m rows)
//   left transform (when rm > bi):
//     [W, tau] = QR(T(k:, k:k+bi)) in place (R, exact zeros); S = wy(W, tau)
//     T(k:, k+bi:) -= (W S^T) (T(k:, k+bi:)^T W)^T           dgemm (applies Q^T)
//     U(:, k:) -= (U(:, k:) W) (W S^T)^T                     dgemm
//   small SVD of T(k:k+bi, k:k+bi) = Us D Vs^T and fold-back:
//     T(0:k, blk) = T(0:k, blk) Vs; T(blk, k+bi:) = Us^T T(blk, k+bi:);
//     V(:, blk) = V(:, blk) Vs; U(:, blk) = U(:, blk) Us; T(blk, blk) = diag(D)
// The right update touches all m rows, as T^(i) = U^(i)^T T^(i-1) V^(i)
// requires; the left update applies Q^T (the formula printed in Fig. 2 is
// dimensionally garbled).  W S^T serves both transforms: T Q = T - (T W)(W S^T)^T
// and Q^T T = T - (W S^T)(W^T T).
#include <atomic>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace rutv {

// ------------------------------------------------------------ bookkeeping

static thread_local char g_last_error[512] = "";
static std::atomic<uint64_t> g_launches{0};

void set_last_error(const char* msg) { snprintf(g_last_error, sizeof g_last_error, "%s", msg); }

int cuda_fail(cudaError_t e, const char* what) {
  snprintf(g_last_error, sizeof g_last_error, "%s: %s (%s)", what, cudaGetErrorName(e),
           cudaGetErrorString(e));
  return RANDUTV_ECUDA;
}

void note_launch(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }

namespace {
struct ProfRec {
  int cls;
  double flops, bytes;
  cudaEvent_t e0, e1;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfRec> g_prof;   // records of the current window
size_t g_prof_used = 0;
}  // namespace

ProfScope::ProfScope(int cls, double flops, double bytes, cudaStream_t s) : slot(-1), st(s) {
  if (!g_prof_on) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (g_prof_used == g_prof.size()) {
    ProfRec r{};
    if (cudaEventCreate(&r.e0) != cudaSuccess || cudaEventCreate(&r.e1) != cudaSuccess) return;
    g_prof.push_back(r);
  }
  ProfRec& r = g_prof[g_prof_used];
  r.cls = cls;
  r.flops = flops;
  r.bytes = bytes;
  slot = (int)g_prof_used++;
  cudaEventRecord(r.e0, st);
}

ProfScope::~ProfScope() {
  if (slot < 0) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  cudaEventRecord(g_prof[slot].e1, st);
}

namespace {
constexpr int kMaxDev = 64;
std::mutex g_mu;
DevInfo g_info[kMaxDev];
bool g_info_ok[kMaxDev];
struct DevScratch {
  char* base = nullptr;
  size_t cap = 0;
  unsigned* status = nullptr;  // 64 words, persistent
  char* stage = nullptr;       // host-call staging
  size_t stage_cap = 0;
};
DevScratch g_scr[kMaxDev];

int current_device() {
  int d = 0;
  cudaGetDevice(&d);
  return d;
}
}  // namespace

const DevInfo& dev_info() {
  const int d = current_device();
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_info_ok[d]) {
    cudaDeviceGetAttribute(&g_info[d].sms, cudaDevAttrMultiProcessorCount, d);
    cudaDeviceGetAttribute(&g_info[d].smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, d);
    if (g_info[d].sms <= 0) g_info[d].sms = 1;
    g_info_ok[d] = true;
  }
  return g_info[d];
}

int status_words(unsigned** out) {
  const int d = current_device();
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scr[d].status) {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, 64 * sizeof(unsigned));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(status)");
    e = cudaMemset(p, 0, 64 * sizeof(unsigned));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemset(status)");
    g_scr[d].status = (unsigned*)p;
  }
  *out = g_scr[d].status;
  return 0;
}

int scratch_reserve(size_t bytes, Arena* out) {
  const int d = current_device();
  std::lock_guard<std::mutex> lk(g_mu);
  DevScratch& s = g_scr[d];
  if (s.cap < bytes) {
    if (s.base) {
      cudaError_t e = cudaDeviceSynchronize();
      if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
      cudaFree(s.base);
      s.base = nullptr;
      s.cap = 0;
    }
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
      cuda_fail(e, "cudaMalloc(scratch)");
      return RANDUTV_ENOMEM;
    }
    s.base = (char*)p;
    s.cap = bytes;
  }
  out->base = s.base;
  out->cap = s.cap;
  out->used = 0;
  return 0;
}

namespace {
struct FuncAttr {
  const void* func;
  size_t smem;
  bool nonportable;
};
std::vector<FuncAttr> g_attr[kMaxDev];

FuncAttr& func_attr(int d, const void* func) {
  for (FuncAttr& a : g_attr[d])
    if (a.func == func) return a;
  g_attr[d].push_back(FuncAttr{func, 0, false});
  return g_attr[d].back();
}
}  // namespace

int ensure_smem(const void* func, size_t bytes) {
  const int d = current_device();
  std::lock_guard<std::mutex> lk(g_mu);
  FuncAttr& a = func_attr(d, func);
  if (a.smem < bytes) {
    RUTV_CK(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    a.smem = bytes;
  }
  return 0;
}

int ensure_nonportable_cluster(const void* func) {
  const int d = current_device();
  std::lock_guard<std::mutex> lk(g_mu);
  FuncAttr& a = func_attr(d, func);
  if (!a.nonportable) {
    RUTV_CK(cudaFuncSetAttribute(func, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    a.nonportable = true;
  }
  return 0;
}

static int stage_reserve(size_t bytes, char** out) {
  const int d = current_device();
  std::lock_guard<std::mutex> lk(g_mu);
  DevScratch& s = g_scr[d];
  if (s.stage_cap < bytes) {
    if (s.stage) {
      cudaError_t e = cudaDeviceSynchronize();
      if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
      cudaFree(s.stage);
      s.stage = nullptr;
      s.stage_cap = 0;
    }
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
      cuda_fail(e, "cudaMalloc(staging)");
      return RANDUTV_ENOMEM;
    }
    s.stage = (char*)p;
    s.stage_cap = bytes;
  }
  *out = s.stage;
  return 0;
}

// ---------------------------------------------------------- small kernels

namespace {

__global__ void set_identity_kernel(int64_t rows, int64_t cols, double* X, int64_t ld) {
  const int64_t total = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % rows, j = e / rows;
    X[i + j * ld] = (i == j) ? 1.0 : 0.0;
  }
}

__global__ void check_finite_kernel(int64_t rows, int64_t cols, const double* X, int64_t ld,
                                    unsigned* err) {
  const int64_t total = rows * cols;
  int bad = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % rows, j = e / rows;
    bad |= !isfinite(X[i + j * ld]);
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) {
    if (atomicCAS(err, 0u, (unsigned)RANDUTV_ENONFINITE) == 0u) atomicExch(err + 1, 100u);
  }
}

// T(blk, blk) = diag(D), exact zeros elsewhere in the block.
__global__ void set_diag_block_kernel(int64_t bi, const double* D, double* T, int64_t ldt) {
  const int64_t total = bi * bi;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % bi, j = e / bi;
    T[i + j * ldt] = (i == j) ? D[i] : 0.0;
  }
}

// One CTA at a barrier for two CTAs (the failure-detection self-test).
__global__ void lone_barrier_kernel(unsigned* bar, unsigned* err) {
  unsigned epoch = 0;
  grid_barrier(bar, 2u, err, 901u, epoch);
}

int grid_for(int64_t total, int threads = 256) {
  int64_t blocks = (total + threads - 1) / threads;
  const int64_t cap = (int64_t)dev_info().sms * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  return (int)blocks;
}

int set_identity(int64_t rows, int64_t cols, double* X, int64_t ld, cudaStream_t st) {
  if (rows * cols == 0) return 0;
  set_identity_kernel<<<grid_for(rows * cols), 256, 0, st>>>(rows, cols, X, ld);
  note_launch();
  RUTV_CK(cudaGetLastError());
  return 0;
}

int copy2d(double* dst, int64_t ldd, const double* src, int64_t lds, int64_t rows, int64_t cols,
           cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return 0;
  RUTV_CK(cudaMemcpy2DAsync(dst, (size_t)ldd * sizeof(double), src, (size_t)lds * sizeof(double),
                            (size_t)rows * sizeof(double), (size_t)cols, cudaMemcpyDeviceToDevice,
                            st));
  return 0;
}

// ------------------------------------------------------------- workspace

struct Plan {
  int64_t m, n, b, big;
  size_t bytes;
};

Plan make_plan(int64_t m, int64_t n, int64_t b) {
  Plan p;
  p.m = m;
  p.n = n;
  p.b = b;
  p.big = (m > n ? m : n);
  const size_t big = (size_t)p.big * (size_t)b * sizeof(double);
  const size_t small = (size_t)b * (size_t)b * sizeof(double);
  size_t bytes = 0;
  auto add = [&](size_t s) { bytes += (s + 255) & ~size_t(255); };
  add(big);  // G
  add(big);  // Y
  add(big);  // Z
  add(big);  // W
  add(big);  // WS
  add(big);  // X
  add(big);  // tmp
  add((size_t)b * sizeof(double));  // tau
  add((size_t)b * sizeof(double));  // D
  add(small);  // Gram
  add(small);  // S
  add(small);  // Us
  add(small);  // Vs
  add(householder_scratch_bytes(b));
  add(small_svd_scratch_bytes(b));
  add(dgemm_scratch_bytes(p.big, b));
  add(big);                             // tmp of the SVD stream
  add(dgemm_scratch_bytes(b, b));       // dgemm scratch of the SVD stream (K = b products)
  p.bytes = bytes + 4096;
  return p;
}

struct Work {
  double *G, *Y, *Z, *W, *WS, *X, *tmp, *tau, *D, *Gm, *S, *Us, *Vs;
  char* qr;
  char* svd;
  double* gemm;
  size_t gemm_bytes;
  double* tmp2;   // SVD stream: fold-back products
  double* gemm2;  // SVD stream: dgemm scratch
  size_t gemm2_bytes;
};

Work carve(Arena& ar, const Plan& p) {
  Work w;
  const size_t big = (size_t)p.big * (size_t)p.b * sizeof(double);
  const size_t small = (size_t)p.b * (size_t)p.b * sizeof(double);
  w.G = (double*)ar.take(big);
  w.Y = (double*)ar.take(big);
  w.Z = (double*)ar.take(big);
  w.W = (double*)ar.take(big);
  w.WS = (double*)ar.take(big);
  w.X = (double*)ar.take(big);
  w.tmp = (double*)ar.take(big);
  w.tau = (double*)ar.take((size_t)p.b * sizeof(double));
  w.D = (double*)ar.take((size_t)p.b * sizeof(double));
  w.Gm = (double*)ar.take(small);
  w.S = (double*)ar.take(small);
  w.Us = (double*)ar.take(small);
  w.Vs = (double*)ar.take(small);
  w.qr = (char*)ar.take(householder_scratch_bytes(p.b));
  w.svd = (char*)ar.take(small_svd_scratch_bytes(p.b));
  w.gemm_bytes = dgemm_scratch_bytes(p.big, p.b);
  w.gemm = (double*)ar.take(w.gemm_bytes);
  w.tmp2 = (double*)ar.take(big);
  w.gemm2_bytes = dgemm_scratch_bytes(p.b, p.b);
  w.gemm2 = (double*)ar.take(w.gemm2_bytes);
  return w;
}



// ---------------------------------------------------------------- the step

struct Ctx {
  int64_t m, n, ldt;
  int b, q;
  uint64_t seed;
  uint32_t matrix_id;
  double *U, *T, *V;
  Work w;
  unsigned* status;  // [0] err, [1] site, [2..3] barrier
  cudaStream_t st;
  SideStream* side;
  bool fold_pending = false;  // row fold of an earlier block still to apply
  int64_t fold_k = 0, fold_bi = 0;
};

int gemm(Ctx& c, bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha, const double* A,
         int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc) {
  return launch_dgemm(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, c.w.gemm,
                      c.w.gemm_bytes, c.st);
}

// W (r x bi, ld r) and tau -> S (bi x bi), then WS = W S^T (r x bi, ld r).
int wy_and_ws(Ctx& c, int64_t r, int64_t bi) {
  Work& w = c.w;
  RUTV_TRY(gemm(c, true, false, bi, bi, r, 1.0, w.W, r, w.W, r, 0.0, w.Gm, bi));
  RUTV_TRY(launch_wy_factor(bi, w.Gm, w.tau, w.S, c.st));
  RUTV_TRY(gemm(c, false, true, r, bi, bi, 1.0, w.W, r, w.S, bi, 0.0, w.WS, r));
  return 0;
}

// Waits for the side stream's SVD and applies the pending row fold
// T(blk, k+b:) <- Us^T T(blk, k+b:) of that block on the main stream.
int flush_fold(Ctx& c) {
  if (!c.fold_pending) return 0;
  c.fold_pending = false;
  RUTV_CK(cudaStreamWaitEvent(c.st, c.side->svd, 0));
  const int64_t k = c.fold_k, bi = c.fold_bi, nc = c.n - k - bi;
  if (nc <= 0) return 0;
  double* Tr = c.T + k + (k + bi) * c.ldt;  // T(blk, k+bi:)
  RUTV_TRY(gemm(c, true, false, bi, nc, bi, 1.0, c.w.Us, bi, Tr, c.ldt, 0.0, c.w.tmp, bi));
  RUTV_TRY(copy2d(Tr, c.ldt, c.w.tmp, bi, bi, nc, c.st));
  return 0;
}

int side_gemm(Ctx& c, bool ta, bool tb, int64_t M, int64_t N, int64_t K, const double* A,
              int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc) {
  return launch_dgemm(ta, tb, M, N, K, 1.0, A, lda, B, ldb, 0.0, C, ldc, c.w.gemm2,
                      c.w.gemm2_bytes, c.side->st);
}

int block_step(Ctx& c, int step, int64_t k, int64_t bi) {
  const int64_t m = c.m, n = c.n, ldt = c.ldt;
  const int64_t rm = m - k, rn = n - k;
  Work& w = c.w;
  double* T = c.T;
  double* T22 = T + k + k * ldt;
  // ---- right transform: block of V from the sketch
  if (rn > bi) {
    RUTV_TRY(launch_philox_normal(c.seed, (uint32_t)step, c.matrix_id, 0u, rm, bi, w.G, rm, c.st));
    RUTV_TRY(gemm(c, true, false, rn, bi, rm, 1.0, T22, ldt, w.G, rm, 0.0, w.Y, rn));
    for (int it = 0; it < c.q; ++it) {
      RUTV_TRY(gemm(c, false, false, rm, bi, rn, 1.0, T22, ldt, w.Y, rn, 0.0, w.Z, rm));
      RUTV_TRY(gemm(c, true, false, rn, bi, rm, 1.0, T22, ldt, w.Z, rm, 0.0, w.Y, rn));
    }
    // the previous block's SVD may still hold SMs: leave them to it
    RUTV_TRY(launch_householder_qr(rn, bi, w.Y, rn, w.W, w.tau, w.qr, c.status + 2, c.status,
                                   c.st, c.fold_pending ? kSvdSms : 0));
    RUTV_TRY(wy_and_ws(c, rn, bi));
    RUTV_TRY(flush_fold(c));
    double* Tk = T + k * ldt;
    RUTV_TRY(gemm(c, false, false, m, bi, rn, 1.0, Tk, ldt, w.W, rn, 0.0, w.X, m));
    RUTV_TRY(gemm(c, false, true, m, rn, bi, -1.0, w.X, m, w.WS, rn, 1.0, Tk, ldt));
    if (c.V) {
      double* Vk = c.V + k * n;
      RUTV_TRY(gemm(c, false, false, n, bi, rn, 1.0, Vk, n, w.W, rn, 0.0, w.X, n));
      RUTV_TRY(gemm(c, false, true, n, rn, bi, -1.0, w.X, n, w.WS, rn, 1.0, Vk, n));
    }
  }
  // ---- left transform: block of U from the QR of the new column panel
  if (rm > bi) {
    RUTV_TRY(launch_householder_qr(rm, bi, T22, ldt, w.W, w.tau, w.qr, c.status + 2, c.status,
                                   c.st));
    RUTV_TRY(wy_and_ws(c, rm, bi));
    if (rn > bi) {
      double* T2 = T + k + (k + bi) * ldt;
      const int64_t nc = rn - bi;
      RUTV_TRY(gemm(c, true, false, nc, bi, rm, 1.0, T2, ldt, w.W, rm, 0.0, w.X, nc));
      RUTV_TRY(gemm(c, false, true, rm, nc, bi, -1.0, w.WS, rm, w.X, nc, 1.0, T2, ldt));
    }
    if (c.U) {
      double* Uk = c.U + k * m;
      RUTV_TRY(gemm(c, false, false, m, bi, rm, 1.0, Uk, m, w.W, rm, 0.0, w.X, m));
      RUTV_TRY(gemm(c, false, true, m, rm, bi, -1.0, w.X, m, w.WS, rm, 1.0, Uk, m));
    }
  }
  // ---- small SVD of the diagonal block and its fold-back, on the side stream
  RUTV_TRY(flush_fold(c));  // the previous block's row fold precedes this SVD's folds
  cudaStream_t ss = c.side->st;
  RUTV_CK(cudaEventRecord(c.side->panel, c.st));
  RUTV_CK(cudaStreamWaitEvent(ss, c.side->panel, 0));
  RUTV_TRY(launch_small_svd((int)bi, T22, ldt, w.D, w.Us, w.Vs, c.status + 8, w.svd, w.gemm2,
                            w.gemm2_bytes, ss));
  if (k > 0) {
    double* Tc = T + k * ldt;  // T(0:k, blk)
    RUTV_TRY(side_gemm(c, false, false, k, bi, bi, Tc, ldt, w.Vs, bi, w.tmp2, k));
    RUTV_TRY(copy2d(Tc, ldt, w.tmp2, k, k, bi, ss));
  }
  if (c.V) {
    double* Vb = c.V + k * n;
    RUTV_TRY(side_gemm(c, false, false, n, bi, bi, Vb, n, w.Vs, bi, w.tmp2, n));
    RUTV_TRY(copy2d(Vb, n, w.tmp2, n, n, bi, ss));
  }
  if (c.U) {
    double* Ub = c.U + k * m;
    RUTV_TRY(side_gemm(c, false, false, m, bi, bi, Ub, m, w.Us, bi, w.tmp2, m));
    RUTV_TRY(copy2d(Ub, m, w.tmp2, m, m, bi, ss));
  }
  set_diag_block_kernel<<<grid_for(bi * bi), 256, 0, ss>>>(bi, w.D, T22, ldt);
  note_launch();
  RUTV_CK(cudaGetLastError());
  RUTV_CK(cudaEventRecord(c.side->svd, ss));
  c.fold_pending = true;  // T(blk, k+bi:) <- Us^T T(blk, k+bi:) (empty when rn == bi)
  c.fold_k = k;
  c.fold_bi = bi;
  return 0;
}

}  // namespace
}  // namespace rutv

namespace rutv {

// The small SVD of a block and its fold-back run on a second stream, beside
// the next block step: nothing of step k+1 before its right update reads
// what they write.  One fold, T(blk, k+b:) <- Us^T T(blk, k+b:), writes
// entries that step k+1's right update also writes; the main stream applies
// it itself, after waiting for the SVD, just before that update (or before
// the next SVD starts, or at the end of the call).  Every entry thus sees the
// same operations in the same order as in a serial run, and the results are
// bitwise the same.  The side stream is non-blocking (no implicit ordering
// with the legacy default stream) and of the highest priority; one per
// device, with its two events.
std::mutex g_side_mu;
SideStream g_side[64];

int side_stream(SideStream** out) {
  int dev = 0;
  RUTV_CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return RANDUTV_EUNSUPPORTED;
  std::lock_guard<std::mutex> lk(g_side_mu);
  SideStream& s = g_side[dev];
  if (!s.st) {
    int least = 0, greatest = 0;
    RUTV_CK(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    RUTV_CK(cudaStreamCreateWithPriority(&s.st, cudaStreamNonBlocking, greatest));
    RUTV_CK(cudaEventCreateWithFlags(&s.panel, cudaEventDisableTiming));
    RUTV_CK(cudaEventCreateWithFlags(&s.svd, cudaEventDisableTiming));
  }
  *out = &s;
  return 0;
}

}  // namespace rutv

// ================================================================= C-ABI

using namespace rutv;

extern "C" {

const char* randutv_strerror(int status) {
  if (status < 0) return "invalid argument";
  switch (status) {
    case RANDUTV_OK: return "success";
    case RANDUTV_ECUDA: return "CUDA runtime error";
    case RANDUTV_ENONFINITE: return "input holds NaN or Inf";
    case RANDUTV_ETIMEOUT: return "a bounded device-side wait ran out";
    case RANDUTV_ENOMEM: return "scratch allocation failed";
    case RANDUTV_EUNSUPPORTED: return "arguments outside what this build supports";
    default: return "unknown status";
  }
}

const char* randutv_last_error(void) { return g_last_error; }

void randutv_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof_on = on != 0;
  g_prof_used = 0;
}

int randutv_profile_read(double* out, int nclass) {
  if (!out) return -1;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  const int nc = nclass < K_NCLASS ? nclass : K_NCLASS;
  for (int c = 0; c < nc * 4; ++c) out[c] = 0.0;
  for (size_t i = 0; i < g_prof_used; ++i) {
    ProfRec& r = g_prof[i];
    cudaError_t e = cudaEventSynchronize(r.e1);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize(profile)");
    float ms = 0.f;
    e = cudaEventElapsedTime(&ms, r.e0, r.e1);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventElapsedTime(profile)");
    if (r.cls < nc) {
      out[r.cls * 4 + 0] += 1.0;
      out[r.cls * 4 + 1] += ms;
      out[r.cls * 4 + 2] += r.flops;
      out[r.cls * 4 + 3] += r.bytes;
    }
  }
  g_prof_used = 0;
  return K_NCLASS;
}

const char* randutv_profile_class_name(int cls) {
  static const char* names[K_NCLASS] = {"philox_normal", "dgemm", "householder_panel",
                                        "wy_factor", "jacobi_svd", "other", "bgemm_tcgen05",
                                        "convert", "jacobi_svd_fp32", "reorth_pass",
                                        "qr_adjoint"};
  return (cls >= 0 && cls < K_NCLASS) ? names[cls] : "?";
}

// Failure detection self-test: one CTA arrives at a grid barrier sized for
// two, so the counter it waits on never completes; the bounded wait gives
// up after kWaitLimitNs and records RANDUTV_ETIMEOUT with site 901.
int randutv_selftest_wait_timeout(void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  unsigned* status = nullptr;
  RUTV_TRY(status_words(&status));
  RUTV_CK(cudaMemsetAsync(status, 0, 64 * sizeof(unsigned), st));
  lone_barrier_kernel<<<1, 32, 0, st>>>(status + 2, status);
  note_launch();
  RUTV_CK(cudaGetLastError());
  RUTV_CK(cudaStreamSynchronize(st));
  unsigned h[2] = {0, 0};
  RUTV_CK(cudaMemcpy(h, status, sizeof h, cudaMemcpyDeviceToHost));
  if (h[0] == (unsigned)RANDUTV_ETIMEOUT && h[1] == 901u) return (int)h[0];
  if (h[0] != 0u) {
    // some other device status: report it as it is, with the site it came from
    char msg[96];
    snprintf(msg, sizeof msg, "selftest: device status %u at site %u", h[0], h[1]);
    set_last_error(msg);
    return (int)h[0];
  }
  set_last_error("selftest: the wait completed without a timeout being recorded");
  return -100;
}

uint64_t randutv_launch_count(int reset) {
  if (reset) return g_launches.exchange(0);
  return g_launches.load();
}

size_t randutv_workspace_bytes(int64_t m, int64_t n, int b, int prec) {
  (void)prec;
  if (m < 1 || n < 1 || b < 1) return 0;
  int64_t p = m < n ? m : n;
  int64_t bb = b < p ? b : p;
  return make_plan(m, n, bb).bytes;
}

void randutv_finalize(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  int cur = 0;
  cudaGetDevice(&cur);
  for (int d = 0; d < kMaxDev; ++d) {
    DevScratch& s = g_scr[d];
    if (!s.base && !s.status && !s.stage) continue;
    cudaSetDevice(d);
    cudaDeviceSynchronize();
    if (s.base) cudaFree(s.base);
    if (s.status) cudaFree(s.status);
    if (s.stage) cudaFree(s.stage);
    s = DevScratch();
  }
  cudaSetDevice(cur);
}

int randutv_stream_status(void* stream) {
  unsigned* st = nullptr;
  RUTV_TRY(status_words(&st));
  RUTV_CK(cudaStreamSynchronize((cudaStream_t)stream));
  unsigned h[2] = {0, 0};
  RUTV_CK(cudaMemcpy(h, st, sizeof h, cudaMemcpyDeviceToHost));
  return (int)h[0];
}

int randutv_factor_ex(int64_t m, int64_t n, const double* A, int64_t lda, int b, int q,
                      uint64_t seed, double* U, double* T, double* V, int max_steps,
                      void* stream, int first_step) {
  if (m < 1) return -1;
  if (n < 1) return -2;
  if (!A && first_step == 0) return -3;
  if (lda < m) return -4;
  if (b < 1 || b > 256) return -5;
  if (q < 0 || q > 16) return -6;
  if (!T) return -9;
  if (first_step < 0) return -13;
  if (T == A && lda != m) return -9;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t p = m < n ? m : n;
  const int64_t bb = b < p ? b : p;
  const Plan plan = make_plan(m, n, bb);
  Arena ar;
  RUTV_TRY(scratch_reserve(plan.bytes, &ar));
  unsigned* status = nullptr;
  RUTV_TRY(status_words(&status));
  RUTV_CK(cudaMemsetAsync(status, 0, 64 * sizeof(unsigned), st));

  Ctx c;
  c.m = m;
  c.n = n;
  c.ldt = m;
  c.b = (int)bb;
  c.q = q;
  c.seed = seed;
  c.matrix_id = 0;
  c.U = U;
  c.T = T;
  c.V = V;
  c.w = carve(ar, plan);
  c.status = status;
  c.st = st;

  if (first_step == 0) {
    check_finite_kernel<<<grid_for(m * n), 256, 0, st>>>(m, n, A, lda, status);
    note_launch();
    RUTV_CK(cudaGetLastError());
    if (T != A) RUTV_TRY(copy2d(T, m, A, lda, m, n, st));
    if (U) RUTV_TRY(set_identity(m, m, U, m, st));
    if (V) RUTV_TRY(set_identity(n, n, V, n, st));
  }
  RUTV_TRY(side_stream(&c.side));
  int step = 0;
  for (int64_t k = 0; k < p; k += bb, ++step) {
    const int64_t bi = (bb < p - k) ? bb : p - k;
    if (step < first_step) continue;
    if (max_steps >= 0 && step >= max_steps) break;
    RUTV_TRY(block_step(c, step, k, bi));
  }
  RUTV_TRY(flush_fold(c));  // also joins the side stream into the caller's stream
  return 0;
}

int randutv_factor(int64_t m, int64_t n, const double* A, int64_t lda, int b, int q,
                   uint64_t seed, double* U, double* T, double* V) {
  int r = randutv_factor_ex(m, n, A, lda, b, q, seed, U, T, V, -1, nullptr, 0);
  if (r != 0) return r;
  return randutv_stream_status(nullptr);
}

int randutv_factor_host(int64_t m, int64_t n, const double* A_host, int64_t lda, int b, int q,
                        uint64_t seed, double* U_host, double* T_host, double* V_host) {
  if (m < 1) return -1;
  if (n < 1) return -2;
  if (!A_host) return -3;
  if (lda < m) return -4;
  if (!T_host) return -9;
  const size_t e = sizeof(double);
  const size_t bytes = ((size_t)m * n + (U_host ? (size_t)m * m : 0) +
                        (V_host ? (size_t)n * n : 0)) * e + 1024;
  char* base = nullptr;
  RUTV_TRY(stage_reserve(bytes, &base));
  double* dT = (double*)base;
  double* dU = U_host ? dT + (size_t)m * n : nullptr;
  double* dV = V_host ? (dU ? dU + (size_t)m * m : dT + (size_t)m * n) : nullptr;
  RUTV_CK(cudaMemcpy2D(dT, (size_t)m * e, A_host, (size_t)lda * e, (size_t)m * e, (size_t)n,
                       cudaMemcpyHostToDevice));
  int r = randutv_factor(m, n, dT, m, b, q, seed, dU, dT, dV);
  if (r != 0) return r;
  RUTV_CK(cudaMemcpy(T_host, dT, (size_t)m * n * e, cudaMemcpyDeviceToHost));
  if (U_host) RUTV_CK(cudaMemcpy(U_host, dU, (size_t)m * m * e, cudaMemcpyDeviceToHost));
  if (V_host) RUTV_CK(cudaMemcpy(V_host, dV, (size_t)n * n * e, cudaMemcpyDeviceToHost));
  return 0;
}

// ------------------------------------------------------------ components

int randutv_philox_normal(uint64_t seed, uint32_t step, uint32_t matrix_id, uint32_t stream_id,
                          int64_t rows, int64_t cols, double* G, void* stream) {
  if (rows < 0) return -5;
  if (cols < 0) return -6;
  if (!G && rows * cols > 0) return -7;
  return launch_philox_normal(seed, step, matrix_id, stream_id, rows, cols, G, rows,
                              (cudaStream_t)stream);
}

int randutv_philox_normal_f32(uint64_t seed, uint32_t step, uint32_t matrix_id,
                              uint32_t stream_id, int64_t rows, int64_t cols, float* G,
                              void* stream) {
  if (rows < 0) return -5;
  if (cols < 0) return -6;
  if (!G && rows * cols > 0) return -7;
  return launch_philox_normal_f32(seed, step, matrix_id, stream_id, rows, cols, G, rows,
                                  (cudaStream_t)stream);
}

int randutv_philox_words(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                         int64_t count, uint32_t* out, void* stream) {
  if (count < 0) return -6;
  if (!out && count > 0) return -7;
  return launch_philox_words(seed, make_uint4(c0, c1, c2, c3), count, out, (cudaStream_t)stream);
}

int randutv_householder_qr(int64_t r, int64_t c, double* panel, int64_t ld, double* W,
                           double* tau, void* stream) {
  if (r < 1) return -1;
  if (c < 1 || c > r || c > 256) return -2;
  if (!panel) return -3;
  if (ld < r) return -4;
  if (!W) return -5;
  if (!tau) return -6;
  Arena ar;
  RUTV_TRY(scratch_reserve(householder_scratch_bytes(c) + 4096, &ar));
  unsigned* status = nullptr;
  RUTV_TRY(status_words(&status));
  cudaStream_t st = (cudaStream_t)stream;
  RUTV_CK(cudaMemsetAsync(status, 0, 64 * sizeof(unsigned), st));
  return launch_householder_qr(r, c, panel, ld, W, tau, (char*)ar.take(householder_scratch_bytes(c)),
                               status + 2, status, st);
}

int randutv_wy_factor(int64_t r, int64_t c, const double* W, const double* tau, double* S,
                      void* stream) {
  if (r < 1) return -1;
  if (c < 1 || c > r || c > 256) return -2;
  if (!W) return -3;
  if (!tau) return -4;
  if (!S) return -5;
  cudaStream_t st = (cudaStream_t)stream;
  Arena ar;
  const size_t gbytes = dgemm_scratch_bytes(c, c);
  RUTV_TRY(scratch_reserve((size_t)c * c * sizeof(double) + gbytes + 4096, &ar));
  double* Gm = (double*)ar.take((size_t)c * c * sizeof(double));
  double* gs = (double*)ar.take(gbytes);
  RUTV_TRY(launch_dgemm(true, false, c, c, r, 1.0, W, r, W, r, 0.0, Gm, c, gs, gbytes, st));
  return launch_wy_factor(c, Gm, tau, S, st);
}

int randutv_small_svd(int64_t b, const double* B, int64_t ldb, double* D, double* Us, double* Vs,
                      void* stream) {
  if (b < 1 || b > 256) return -1;
  if (!B) return -2;
  if (ldb < b) return -3;
  if (!D) return -4;
  if (!Us) return -5;
  if (!Vs) return -6;
  unsigned* status = nullptr;
  RUTV_TRY(status_words(&status));
  const size_t sb = small_svd_scratch_bytes((int)b), gb = dgemm_scratch_bytes(b, b);
  Arena ar;
  RUTV_TRY(scratch_reserve(sb + gb + 1024, &ar));
  void* svd = ar.take(sb);
  double* gs = (double*)ar.take(gb);
  return launch_small_svd((int)b, B, ldb, D, Us, Vs, status + 8, svd, gs, gb,
                          (cudaStream_t)stream);
}

int randutv_dgemm(char transa, char transb, int64_t M, int64_t N, int64_t K, double alpha,
                  const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
                  double* C, int64_t ldc, void* stream) {
  const bool ta = (transa == 'T' || transa == 't'), tb = (transb == 'T' || transb == 't');
  if (!ta && !(transa == 'N' || transa == 'n')) return -1;
  if (!tb && !(transb == 'N' || transb == 'n')) return -2;
  if (M < 0) return -3;
  if (N < 0) return -4;
  if (K < 0) return -5;
  if (lda < (ta ? (K > 1 ? K : 1) : (M > 1 ? M : 1))) return -8;
  if (ldb < (tb ? (N > 1 ? N : 1) : (K > 1 ? K : 1))) return -10;
  if (ldc < (M > 1 ? M : 1)) return -13;
  Arena ar;
  const size_t gbytes = dgemm_scratch_bytes(M, N);
  RUTV_TRY(scratch_reserve(gbytes + 4096, &ar));
  double* gs = (double*)ar.take(gbytes);
  return launch_dgemm(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, gs, gbytes,
                      (cudaStream_t)stream);
}

}  // extern "C"
