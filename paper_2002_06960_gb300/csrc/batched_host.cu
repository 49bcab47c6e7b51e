// Host side of the batched randUTV: plans (descriptors, queue order,
// workspace) and the capturable run.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <numeric>
#include <vector>

#include "common.cuh"

namespace rutv {

size_t batched_work_floats(int64_t mmax);
size_t batched_smem_bytes();
int launch_batched(const void* desc_dev, const int* order_dev, int count, int* next_dev,
                   int* info_dev, uint64_t seed, float* work, int64_t work_stride, int64_t mmax,
                   int grid, cudaStream_t st);
int batched_max_ctas_per_sm(int* out);
int batched_desc_bytes();

namespace {

// must match the device-side BatchDesc
struct BatchDescHost {
  int64_t m, n, lda;
  const float* A;
  float* T;
  float* U;
  float* V;
  int b, q;
  int matrix_id, pad;
};

// Block size per size class (class c covers max(m, n) in (128 c, 128 (c+1)]),
// written by the autotuner; 0 entries fall back to kDefaultB.
constexpr int kClasses = 8;
constexpr int kDefaultB = 32;
std::mutex g_tune_mu;
int g_b_table[kClasses] = {0};
int g_ctas_per_sm = 0;  // 0 = occupancy limit

int b_for(int64_t m, int64_t n) {
  const int64_t big = m > n ? m : n;
  int c = (int)((big - 1) / 128);
  if (c < 0) c = 0;
  if (c >= kClasses) c = kClasses - 1;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  return g_b_table[c] > 0 ? g_b_table[c] : kDefaultB;
}

}  // namespace

struct BatchedPlan {
  int count = 0;
  int grid = 0;
  int64_t mmax = 0;
  uint64_t seed = 0;
  void* desc = nullptr;   // device
  int* order = nullptr;   // device
  int* next = nullptr;    // device
  float* work = nullptr;  // device
  int64_t work_stride = 0;
  double flops = 0.0;
};

}  // namespace rutv

using namespace rutv;

extern "C" {

int randutv_batched_set_tuning(const int* b_for_class, int nclasses, int ctas_per_sm) {
  if (nclasses < 0 || nclasses > kClasses) return -2;
  if (ctas_per_sm < 0 || ctas_per_sm > 16) return -3;
  int table[kClasses];
  for (int c = 0; c < kClasses; ++c) {  // validate all first: an error changes nothing
    const int b = (b_for_class && c < nclasses) ? b_for_class[c] : 0;
    if (b != 0 && b != 16 && b != 32 && b != 64) return -1;
    table[c] = b;
  }
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (int c = 0; c < kClasses; ++c) g_b_table[c] = table[c];
  g_ctas_per_sm = ctas_per_sm;
  return 0;
}

int randutv_batched_plan_create(void** plan_out, int batch, const int64_t* m, const int64_t* n,
                                const float* const* A, const int64_t* lda, int b, int q,
                                uint64_t seed, float* const* U, float* const* T,
                                float* const* V) {
  if (!plan_out) return -1;
  if (batch < 1) return -2;
  if (!m) return -3;
  if (!n) return -4;
  if (!A) return -5;
  if (!lda) return -6;
  if (!(b == 0 || b == 16 || b == 32 || b == 64)) return -7;
  if (q < 0 || q > 16) return -8;
  if (!T) return -11;
  std::vector<BatchDescHost> d((size_t)batch);
  int64_t mmax = 1;
  double flops = 0.0;
  std::vector<double> cost((size_t)batch);
  for (int i = 0; i < batch; ++i) {
    if (m[i] < 1 || m[i] > 1024 || n[i] < 1 || n[i] > 1024) return RANDUTV_EUNSUPPORTED;
    if (lda[i] < m[i]) return -6;
    if (!A[i] || !T[i]) return -5;
    d[i].m = m[i];
    d[i].n = n[i];
    d[i].lda = lda[i];
    d[i].A = A[i];
    d[i].T = T[i];
    d[i].U = U ? U[i] : nullptr;
    d[i].V = V ? V[i] : nullptr;
    d[i].b = b ? b : b_for(m[i], n[i]);
    d[i].q = q;
    d[i].matrix_id = i;
    d[i].pad = 0;
    mmax = std::max<int64_t>(mmax, std::max(m[i], n[i]));
    const double p = (double)std::min(m[i], n[i]);
    cost[i] = (double)m[i] * (double)n[i] * p;
    flops += cost[i];
  }
  // largest first, so that the tail of the launch is made of small matrices
  std::vector<int> order((size_t)batch);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return cost[a] > cost[c]; });

  int per_sm = 0;
  RUTV_TRY(batched_max_ctas_per_sm(&per_sm));
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (g_ctas_per_sm > 0 && g_ctas_per_sm < per_sm) per_sm = g_ctas_per_sm;
  }
  if (per_sm < 1) per_sm = 1;
  int grid = dev_info().sms * per_sm;
  if (grid > batch) grid = batch;

  BatchedPlan* P = new BatchedPlan();
  P->count = batch;
  P->grid = grid;
  P->mmax = mmax;
  P->seed = seed;
  P->work_stride = (int64_t)batched_work_floats(mmax);
  P->flops = flops;
  const size_t desc_bytes = sizeof(BatchDescHost) * (size_t)batch;
  cudaError_t e = cudaMalloc(&P->desc, desc_bytes);
  if (e == cudaSuccess) e = cudaMalloc((void**)&P->order, sizeof(int) * (size_t)batch);
  if (e == cudaSuccess) e = cudaMalloc((void**)&P->next, 256);
  if (e == cudaSuccess)
    e = cudaMalloc((void**)&P->work, sizeof(float) * (size_t)P->work_stride * (size_t)grid);
  if (e == cudaSuccess) e = cudaMemcpy(P->desc, d.data(), desc_bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(P->order, order.data(), sizeof(int) * (size_t)batch, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(P->desc);
    cudaFree(P->order);
    cudaFree(P->next);
    cudaFree(P->work);
    delete P;
    cuda_fail(e, "randutv_batched_plan_create");
    return RANDUTV_ENOMEM;
  }
  (void)batched_desc_bytes;
  *plan_out = P;
  return 0;
}

int randutv_batched_run(void* plan, int* info, void* stream) {
  if (!plan) return -1;
  if (!info) return -2;
  BatchedPlan* P = (BatchedPlan*)plan;
  return launch_batched(P->desc, P->order, P->count, P->next, info, P->seed, P->work,
                        P->work_stride, P->mmax, P->grid, (cudaStream_t)stream);
}

int randutv_batched_plan_destroy(void* plan) {
  if (!plan) return 0;
  BatchedPlan* P = (BatchedPlan*)plan;
  cudaError_t e = cudaDeviceSynchronize();
  cudaFree(P->desc);
  cudaFree(P->order);
  cudaFree(P->next);
  cudaFree(P->work);
  delete P;
  return e == cudaSuccess ? 0 : cuda_fail(e, "randutv_batched_plan_destroy");
}

int randutv_factor_batched(int batch, const int64_t* m, const int64_t* n, const float* const* A,
                           const int64_t* lda, int b, int q, uint64_t seed, float* const* U,
                           float* const* T, float* const* V, int* info, void* stream) {
  void* plan = nullptr;
  RUTV_TRY(randutv_batched_plan_create(&plan, batch, m, n, A, lda, b, q, seed, U, T, V));
  int r = randutv_batched_run(plan, info, stream);
  if (r == 0) {
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) r = cuda_fail(e, "randutv_factor_batched");
  }
  randutv_batched_plan_destroy(plan);
  return r;
}

}  // extern "C"
