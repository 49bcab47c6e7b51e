// Launchers of the device kernels (one translation unit each).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace rutv {

int launch_philox_normal(uint64_t seed, uint32_t step, uint32_t mid, uint32_t sid, int64_t rows,
                         int64_t cols, double* G, int64_t ldg, cudaStream_t st);
int launch_philox_normal_f32(uint64_t seed, uint32_t step, uint32_t mid, uint32_t sid,
                             int64_t rows, int64_t cols, float* G, int64_t ldg, cudaStream_t st);
int launch_philox_normal_rows(uint64_t seed, uint32_t step, uint32_t mid, uint32_t sid,
                              int64_t rows_total, int64_t row0, int64_t nrows, int64_t cols,
                              double* G, int64_t ldg, cudaStream_t st);
int launch_philox_words(uint64_t seed, uint4 c, int64_t count, uint32_t* out, cudaStream_t st);

size_t dgemm_scratch_bytes(int64_t M, int64_t N);
// lower: compute only the 64 x 64 tiles of C that meet or lie below the
// diagonal (for a symmetric product whose reader takes its lower triangle);
// the others are left as they were.
int launch_dgemm(bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha, const double* A,
                 int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc,
                 double* scratch, size_t scratch_bytes, cudaStream_t st, bool lower = false);

size_t householder_scratch_bytes(int64_t c);
// SMs that the small SVD may hold while it runs beside a block step.
constexpr int kSvdSms = 16;
// reserve_sms: SMs to leave free (the grid then uses at most SMs - reserve_sms CTAs).
int launch_householder_qr(int64_t r, int64_t c, double* A, int64_t lda, double* W, double* tau,
                          char* scratch, unsigned* bar, unsigned* err, cudaStream_t st,
                          int reserve_sms = 0);
// S (c x c, ld c) from the Gram matrix of the reflectors (its diagonal and
// strictly lower part are read, leading dimension ldg; 0 means c) and tau.
int launch_wy_factor(int64_t c, const double* Gm, const double* tau, double* S, cudaStream_t st,
                     int64_t ldg = 0);
// M = (I + D_tau striu(Gm))^-1 (c x c, ld c), so that S = M D_tau.
int launch_wy_inverse(int64_t c, const double* Gm, const double* tau, double* M, cudaStream_t st);

// Scratch of launch_small_svd (beside the dgemm scratch it also takes).
size_t small_svd_scratch_bytes(int b);
int launch_small_svd(int b, const double* B, int64_t ldb, double* D, double* Us, double* Vs,
                     unsigned* info, void* scratch, double* gemm_scratch, size_t gemm_bytes,
                     cudaStream_t st);


// Second stream of a device on which the small SVD of a block and its
// fold-back run beside the next block step (non-blocking, highest priority),
// with the two events that order it against the caller's stream.
struct SideStream {
  cudaStream_t st = nullptr;
  cudaEvent_t panel = nullptr;  // main -> side: the block and its factors are final
  cudaEvent_t svd = nullptr;    // side -> main: SVD and folds done
};
int side_stream(SideStream** out);

}  // namespace rutv
