/*
 * randutv.h -- C-ABI of the GB300 randUTV library.
 *
 * randUTV (Heavner, Martinsson & Quintana-Orti, "Computing rank-revealing
 * factorizations of matrices stored out-of-core", arXiv 2002.06960, §3.1 and
 * Fig. 2) factors an m x n matrix as A = U T V^T with U (m x m) and V (n x n)
 * orthogonal and T (m x n) upper triangular, one block of b columns per step:
 * a Gaussian sketch and power iteration give the block of V, a Householder QR
 * of the new column panel gives the block of U, and a b x b SVD makes the
 * diagonal block of T diagonal.  The same library holds the paper's other
 * factorization, HQRRP (§2: column-pivoted QR A P = Q R with pivots chosen on
 * a sketch), and the factorization of a matrix kept in host memory (§3.2).
 *
 * Conventions for every entry point below:
 *  - Matrices are column-major with a leading dimension (ld >= rows).
 *  - Pointers are DEVICE pointers (memory of the current CUDA device) unless
 *    the name ends in _host.  The caller owns every buffer it passes; the
 *    library never frees caller memory.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Each entry point states whether it is asynchronous on its
 *    stream (device errors then come from randutv_stream_status) or
 *    synchronizes before returning.
 *  - Return value: 0 on success; -i if argument i (1-based) is invalid
 *    (LAPACK style); a positive randutv_status otherwise.  No C++ exception
 *    crosses this boundary.
 *  - Scratch memory is allocated by the library on first use per device and
 *    kept until randutv_finalize(); it grows when a larger problem needs it.
 *    All entry points on one device share that scratch (and the library's
 *    side and copy streams), so calls whose device work may overlap, such as
 *    asynchronous calls on different streams or calls from several host
 *    threads, must be serialized by the caller: issue them on one stream,
 *    or wait for one before starting the next.  A batched plan owns its own
 *    workspace.
 *  - Device-side waits are bounded (about two seconds); a wait that runs out
 *    makes the call return RANDUTV_ETIMEOUT and leaves the outputs undefined.
 */
#ifndef RANDUTV_H
#define RANDUTV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RANDUTV_OK = 0,
  RANDUTV_ECUDA = 1,      /* a CUDA runtime call failed (message: randutv_last_error) */
  RANDUTV_ENONFINITE = 2, /* the input holds NaN or Inf */
  RANDUTV_ETIMEOUT = 3,   /* a bounded device-side wait ran out */
  RANDUTV_ENOMEM = 4,     /* scratch allocation failed */
  RANDUTV_EUNSUPPORTED = 5 /* valid arguments outside what this build supports */
} randutv_status;

typedef enum {
  RANDUTV_FP64 = 0 /* every step in FP64 */
} randutv_prec;

/* ---------------------------------------------------------------- factor --
 * Full blocked randUTV, §3.1 steps 1-6 with the update list of Fig. 2.
 *   m, n    (args 1, 2)  sizes, m >= 1, n >= 1.
 *   A       (3)  m x n input, read only, leading dimension lda >= m (4).
 *   b       (5)  block size, 1 <= b <= 256.
 *   q       (6)  power-iteration count, 0 <= q <= 16.
 *   seed    (7)  key of the Philox sketch generator (see randutv_philox_normal).
 *   U       (8)  m x m output, ld m, or NULL to skip U.
 *   T       (9)  m x n output, ld m; may alias A only when lda == m.
 *   V       (10) n x n output, ld n, or NULL to skip V.
 * On return T is upper triangular with exact zeros below the diagonal, every
 * b x b diagonal block is diagonal with non-negative entries in descending
 * order, and A = U T V^T up to rounding.  Returns RANDUTV_ENONFINITE when A
 * holds NaN or Inf (checked before any work).
 */
int randutv_factor(int64_t m, int64_t n, const double* A, int64_t lda, int b, int q,
                   uint64_t seed, double* U, double* T, double* V);

/* As randutv_factor, asynchronous on `stream` (arg 12), with two extras:
 *   max_steps (11)  stop after this many block steps (a partial factorization
 *                   whose first max_steps*b columns of U, V are final); a
 *                   negative value runs to completion.
 *   first_step(13)  resume: treat U, T, V as the state after `first_step`
 *                   steps of an earlier call with the same arguments, and
 *                   continue from there (0 = start from A; A is then unread).
 * Because the sketch of step i depends only on (seed, i), a resumed run gives
 * bitwise the same result as an uninterrupted one.  Errors detected on the
 * device are reported by randutv_stream_status() after the stream completes.
 */
int randutv_factor_ex(int64_t m, int64_t n, const double* A, int64_t lda, int b, int q,
                      uint64_t seed, double* U, double* T, double* V, int max_steps,
                      void* stream, int first_step);

/* randutv_factor with HOST buffers (pageable or pinned): A is copied to the
 * device, factored, and U, T, V copied back; same arguments and layout. */
int randutv_factor_host(int64_t m, int64_t n, const double* A_host, int64_t lda, int b, int q,
                        uint64_t seed, double* U_host, double* T_host, double* V_host);

/* Status word of the last _ex call on `stream` (synchronizes the stream). */
int randutv_stream_status(void* stream);

/* ---------------------------------------------------------- mixed precision --
 * The same block steps (§3.1, Fig. 2) with FP32 input and output, asynchronous
 * on `stream` (arg 12); device errors are read with randutv_stream_status().
 *   A (3)   m x n FP32, leading dimension lda (4); U (8), T (9), V (10) FP32
 *           with ld m, m, n; U or V may be NULL.
 *   b (5)   block size, a multiple of 8 in [8, 256].
 *   max_steps (11) as in randutv_factor_ex.
 * Arithmetic: T, U^T and V^T are held as three BF16 planes each (24
 * significant bits, the precision of FP32 storage).  The sketch and power
 * products take one BF16 product on the tensor cores (FP32 accumulation);
 * every compact-WY update and the fold-back take the six-product BF16 split,
 * which is FP32-accurate; the Householder vectors and norms, the WY factor S
 * and the b x b SVD are FP64.  The sketch is RNE(bf16) of the FP64 sketch
 * of randutv_philox_normal.  A run that completes every step ends with one
 * re-orthogonalisation pass: with E = X^T X - I for X = U, V (its diagonal
 * summed in FP64) and Phi = striu(E) + diag(E)/2, U <- U (I - Phi_U),
 * V <- V (I - Phi_V^T) and T <- (I + Phi_U) T (I + Phi_V), which keeps
 * U T V^T and leaves U and V orthogonal to FP32 rounding; the off-diagonal
 * entries this leaves inside the diagonal blocks of T are zeroed. */
int randutv_factor_mixed(int64_t m, int64_t n, const float* A, int64_t lda, int b, int q,
                         uint64_t seed, float* U, float* T, float* V, int max_steps,
                         void* stream);

/* ----------------------------------------------------------------- batched --
 * Many FP32 matrices of uneven sizes (1 <= m, n <= 1024), each factored by the
 * block steps of §3.1 / Fig. 2, in ONE persistent launch: each CTA takes the
 * next matrix from a device queue ordered by descending cost.  Arithmetic:
 * FP32 storage and FFMA products; Householder norms and scalars in FP64;
 * FP32 one-sided Jacobi for the b x b SVD; the sketch of step i of matrix j
 * is randutv_philox_normal_f32(seed, i, j, 0, ...): the Philox words of
 * randutv_philox_normal with a single-precision Box-Muller.
 *   batch (2)        number of matrices.
 *   m, n, lda (3,4,7) HOST arrays of length batch.
 *   A (5)            HOST array of DEVICE pointers, matrix i is m[i] x n[i].
 *   b (8)            16, 32 or 64 for every matrix, or 0 for the tuned
 *                    per-size table (randutv_batched_set_tuning; default 32).
 *   q (9), seed (10) as in randutv_factor.
 *   U, T, V (11-13)  HOST arrays of DEVICE pointers (ld m[i], m[i], n[i]);
 *                    U or V may be NULL (no factors for any matrix).
 * The plan uploads the descriptors (synchronously) and owns the queue and
 * the per-CTA workspace; randutv_batched_run is one memset and one kernel
 * launch on `stream`, so it can be captured in a CUDA graph and replayed
 * (each replay refactors the same matrices).  info (device, batch ints)
 * receives 0 or RANDUTV_ENONFINITE per matrix. */
int randutv_batched_plan_create(void** plan, int batch, const int64_t* m, const int64_t* n,
                                const float* const* A, const int64_t* lda, int b, int q,
                                uint64_t seed, float* const* U, float* const* T,
                                float* const* V);
int randutv_batched_run(void* plan, int* info, void* stream);
int randutv_batched_plan_destroy(void* plan);

/* One-shot form: plan, run on `stream`, wait, destroy. */
int randutv_factor_batched(int batch, const int64_t* m, const int64_t* n, const float* const* A,
                           const int64_t* lda, int b, int q, uint64_t seed, float* const* U,
                           float* const* T, float* const* V, int* info, void* stream);

/* Autotuner output: block size (16, 32, 64, or 0 = default 32) for each of
 * `nclasses` <= 8 size classes, class c holding max(m, n) in (128c, 128(c+1)],
 * and CTAs per SM for the persistent grid (0 = occupancy limit). */
int randutv_batched_set_tuning(const int* b_for_class, int nclasses, int ctas_per_sm);

/* ------------------------------------------------------------------ HQRRP --
 * Column-pivoted QR A P = Q R by HQRRP (§2.1-2.2): blocks of b pivots, each
 * chosen by b steps of column-pivoted QR of the sketch Y = G R(k:, k:), G of
 * size b x (m - k) with i.i.d. N(0,1) entries, drawn anew at every step, and
 * followed by an unpivoted Householder QR of the chosen columns.  FP64;
 * asynchronous on `stream` (arg 10); all pointers DEVICE.
 *   m, n (1, 2)  m >= n >= 1.
 *   A (3)        m x n with lda (4) >= m, read only (R may be A when lda == m).
 *   b (5)        1 <= b <= 256.
 *   seed (6)     G of step i is the transpose of the m-k x b array that
 *                randutv_philox_normal(seed, i, 0, 6, ...) gives.
 *   Q (7)        m x m (ld m), or NULL.
 *   R (8)        m x n (ld m): R, upper trapezoidal with exact zeros.
 *   perm (9)     n int64: column j of A P is column perm[j] of A.
 * Ties between pivot candidates go to the lowest column position.  Device
 * errors are read with randutv_stream_status(). */
int randutv_hqrrp(int64_t m, int64_t n, const double* A, int64_t lda, int b, uint64_t seed,
                  double* Q, double* R, int64_t* perm, void* stream);

/* ------------------------------------------------------------- out of HBM --
 * The factorization of a matrix that stays in HOST memory (§3.2: the
 * out-of-core setting, here the device's HBM against the host's memory).
 * The same block steps in FP64 as randutv_factor; every pass over a trailing
 * region streams it through the device in panels, with the copies in and out
 * overlapping the arithmetic (two copy streams, three panel buffers).
 *   A (3)      HOST, m x n with lda (4) >= m; overwritten by T.  Pinned
 *              memory (cudaHostAlloc / cudaHostRegister) lets the copies run
 *              asynchronously; pageable memory works, without the overlap.
 *   U (8), V (9)  HOST, m x m (ld m) and n x n (ld n), or NULL.
 *   device_bytes (10)  device memory the call may use (workspace and panel
 *              buffers): at least randutv_ooc_min_device_bytes(m, n, b);
 *              larger panels cost fewer copies per pass.
 *   bytes_moved (11)   HOST, optional: the bytes copied between host and
 *              device by the call.
 *   b, q, seed as in randutv_factor; stream (12): the compute stream.
 * Synchronous: returns after the factorization (0, a device status, or -i).
 * The result is deterministic for a given device_bytes; against
 * randutv_factor (and between budgets) it differs only in rounding, since the
 * panel cut changes the summation order of some products. */
size_t randutv_ooc_min_device_bytes(int64_t m, int64_t n, int b);
int randutv_factor_ooc(int64_t m, int64_t n, double* A, int64_t lda, int b, int q, uint64_t seed,
                       double* U, double* V, size_t device_bytes, double* bytes_moved,
                       void* stream);

/* ---------------------------------------------------- low rank and adjoint --
 * A_k = U(:, 0:k) U(:, 0:k)^T A, the rank-k approximation of §1.1
 * (A_k = U(:,1:k) R(1:k,:) V^*), through the first k/b block steps of §3.1
 * with the sketch fixed by `seed`.  FP64; all pointers DEVICE.
 *   m, n (1, 2); A (3) m x n with lda (4) >= m, read only;
 *   k (5): 1 <= k < min(m, n); b (6): 1 <= b <= 256 and b divides k;
 *   q (7), seed (8) as in randutv_factor.
 * The block SVDs rotate columns inside a block and leave the span of
 * U(:, 0:k) unchanged, so they are not computed.  Synchronous. */
int randutv_lowrank(int64_t m, int64_t n, const double* A, int64_t lda, int k, int b, int q,
                    uint64_t seed, double* Ak /* (9) m x n, ld m */, void* stream);

/* Adjoint (vector-Jacobian product) of randutv_lowrank in A, the sketch held
 * fixed: dA (10, m x n, ld m) = (d A_k / d A)^T dAk (9, m x n, ld m).  The
 * per-step Householder factors are recomputed from A and the seed (nothing
 * is kept from the forward call).  Synchronous; same argument rules. */
int randutv_lowrank_backward(int64_t m, int64_t n, const double* A, int64_t lda, int k, int b,
                             int q, uint64_t seed, const double* dAk, double* dA, void* stream);

/* Tensor-core GEMM of the mixed path, FP32 in and out:
 * C = alpha op(A) B + beta C with op(A) = A (transa 'N', A is M x K, MN-major
 * operand) or A^T (transa 'T', A is K x M, K-major operand), B K x N.  The
 * operands are split into `planes` BF16 planes (1: one BF16 product; 3: the
 * six products of the FP32-accurate split).  Asynchronous on `stream`. */
int randutv_gemm_bf16(char transa, int64_t M, int64_t N, int64_t K, float alpha, const float* A,
                      int64_t lda, const float* B, int64_t ldb, float beta, float* C, int64_t ldc,
                      int planes, void* stream);

/* ------------------------------------------------------------ components --
 * The steps of one block, exposed so that each can be checked on its own.
 * All are asynchronous on `stream` (the last argument); device errors (a
 * bounded wait that ran out) are read with randutv_stream_status().
 */

/* Gaussian sketch of one step (§3.1, construction of V-hat, step 1): G is
 * rows x cols, column-major with ld = rows.  Element l = r + c*rows takes
 * pair p = l >> 1 of Philox4x32-10 with key (lo32(seed), hi32(seed)) and
 * counter (p, step, matrix_id, stream_id); the pair's 53-bit uniforms
 * u1 = (j1 + 1) 2^-53, u2 = j2 2^-53 (j = (x0 >> 5) 2^26 + (x1 >> 6) and
 * likewise from x2, x3) give sqrt(-2 ln u1) cos(2 pi u2) for even l and
 * sqrt(-2 ln u1) sin(2 pi u2) for odd l. */
int randutv_philox_normal(uint64_t seed, uint32_t step, uint32_t matrix_id, uint32_t stream_id,
                          int64_t rows, int64_t cols, double* G, void* stream);

/* The batched form's FP32 sketch (the generator randutv_factor_batched draws
 * with): the same words and element order as randutv_philox_normal, 24-bit
 * uniforms u1 = ((x0 >> 8) + 1) 2^-24 in (0, 1] and u2 = (x2 >> 8) 2^-24 in
 * [0, 1), and sqrt(-2 ln u1) (cos, sin)(2 pi u2) in FP32.  G is rows x cols
 * FP32, ld = rows. */
int randutv_philox_normal_f32(uint64_t seed, uint32_t step, uint32_t matrix_id,
                              uint32_t stream_id, int64_t rows, int64_t cols, float* G,
                              void* stream);

/* Raw Philox4x32-10 words for counters (c0 + i, c1, c2, c3), i = 0..count-1;
 * out is 4*count uint32 (device). */
int randutv_philox_words(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                         int64_t count, uint32_t* out, void* stream);

/* Unpivoted Householder QR of an r x c panel, r >= c, in place (Fig. 2,
 * unpivoted_QR).  On return the upper triangle of the top c x c holds R and
 * the part below the diagonal is exactly zero; W (r x c, ld r) is the unit
 * lower trapezoidal matrix of reflector vectors and tau (c) their scalars,
 * with H_j = I - tau_j w_j w_j^T and panel_in = H_1 ... H_c [R; 0].
 * Reflector convention: for x = (alpha, x2), s = ||x2||; s == 0 gives
 * tau = 0 (H = I); otherwise beta = -sgn(alpha) sqrt(alpha^2 + s^2),
 * sgn(0) = +1, tau = (beta - alpha)/beta, w = (1, x2/(alpha - beta)). */
int randutv_householder_qr(int64_t r, int64_t c, double* panel, int64_t ld, double* W,
                           double* tau, void* stream);

/* randutv_householder_qr without any memory allocation (the paper has no
 * counterpart; this is a service to callers).
 * Some callers cannot let a library allocate device memory: programs whose
 * own allocator or memory pool already owns all of the GPU's memory, where a
 * cudaMalloc from the library would fail or fragment the pool; and latency-
 * bound loops that cannot pay for cudaMalloc/cudaFree, which may block the
 * host and synchronize the device, or handle an allocation failing midway.
 * This entry point serves them: it calls no cudaMalloc, cudaFree or other
 * allocating routine.  Its scratch is a fixed array inside the library
 * (about 388 KiB: partial sums for up to 192 SMs x 256 columns, plus its
 * barrier and status words), which every GPU that loads the library holds
 * until the process exits.
 *   Arguments, layout and results are those of randutv_householder_qr; the
 *   caller still owns panel, W and tau.
 *   c > 256, or a device with more than 192 SMs: returns
 *   RANDUTV_EUNSUPPORTED without launching anything.
 *   The call is synchronous: it waits for the kernel on `stream` and returns
 *   its device status (RANDUTV_ETIMEOUT if a bounded wait ran out).
 *   The first call on a device looks up the array's device address (once
 *   per device, with that device current); make that first call before any
 *   stream capture.
 *   All calls share the one array and it keeps the last call's contents, so
 *   calls that overlap on the GPU (other streams, other host threads) race
 *   and must be serialized by the caller. */
int randutv_householder_qr_noalloc(int64_t r, int64_t c, double* panel, int64_t ld, double* W,
                                   double* tau, void* stream);

/* Compact-WY factor (Fig. 2: T_V, T_U): S (c x c, ld c, upper triangular)
 * with H_1 ... H_c = I - W S W^T, for W (r x c, ld r) and tau from
 * randutv_householder_qr; 1 <= c <= min(r, 256). */
int randutv_wy_factor(int64_t r, int64_t c, const double* W, const double* tau, double* S,
                      void* stream);

/* SVD of a b x b block (Fig. 2: [A11, U_SVD, V_SVD] := SVD(A11)), one-sided
 * Jacobi in FP64: B = Us diag(D) Vs^T with D descending and >= 0; each column
 * of Vs has its entry of largest magnitude (lowest row on ties) positive and
 * the matching column of Us carries the same sign.  B (ld ldb) is read only;
 * Us, Vs are b x b with ld b; 1 <= b <= 256. */
int randutv_small_svd(int64_t b, const double* B, int64_t ldb, double* D, double* Us, double* Vs,
                      void* stream);

/* C = alpha op(A) op(B) + beta C in FP64 (the products of every step);
 * transa/transb are 'N' or 'T'. */
int randutv_dgemm(char transa, char transb, int64_t M, int64_t N, int64_t K, double alpha,
                  const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
                  double* C, int64_t ldc, void* stream);

/* ------------------------------------------------------ randUTV by blocks --
 * The analyzer of §3.2.4: the task list of randUTV_AB for an m x n matrix in
 * blocks of b (tile starts: multiples of b up to p = min(m, n), then p + b t),
 * q power iterations, with U (want_u) and V (want_v) or not.  Each task is an
 * operation (randutv_ab_op_name) of one block step, with up to four blocks
 * read and four written.  A block is kind << 40 | i << 20 | j, kind 0..9 =
 * A, G, Y, Z, B, C, P, Q, U, V (A holds T as it is formed; G, Y, Z the tiles of
 * the sketch and its products; B, C the compact-WY factors of the QRs of the
 * Y tiles and of the A tiles of the block column; P, Q the factors U_s, V_s
 * of the step's small SVD).  Host code only; no device is touched.
 *   ops, steps (cap ints each), operands (8 * cap: in[0..3], out[0..3],
 *   -1 where unused): HOST arrays, filled for the first min(cap, count)
 *   tasks; any may be NULL.  Returns the number of tasks, or -i for a bad
 *   argument i (m, n, b >= 1; 0 <= q <= 16). */
int64_t randutv_ab_tasks(int64_t m, int64_t n, int b, int q, int want_u, int want_v, int32_t* ops,
                         int32_t* steps, int64_t* operands, int64_t cap);

/* Name of an operation of the task list ("Comp_td_QR", ...). */
const char* randutv_ab_op_name(int op);

/* randUTV by blocks in HBM (§3.2.2-3.2.3): the analyzer's task list run on
 * b x b tiles of T (a view of the caller's T), U and V, with every QR done by
 * blocks (a dense QR of the leading block, triangular-dense QRs below it).
 * Tasks are spread over `nstreams` (11, 1..16) library streams and ordered by
 * data flow alone (each waits for the last writer of what it reads and
 * writes and for the readers of what it writes), with no join between block
 * steps.  Arguments 1-10 as in randutv_factor_ex (b <= 256); asynchronous on
 * `stream` (12), device errors from randutv_stream_status().  The result is
 * the by-blocks factorization: the same method with another orthonormal
 * completion of each step's Q, so U, T, V differ from randutv_factor beyond
 * the first block; the first block of U and V spans the same space.
 * Deterministic: each tile's operations run in task order. */
int randutv_factor_ab(int64_t m, int64_t n, const double* A, int64_t lda, int b, int q,
                      uint64_t seed, double* U, double* T, double* V, int nstreams, void* stream);

/* The by-blocks factorization of a matrix in HOST memory (§3.2.4): T (in
 * place of A, arg 3, lda 4), U (8) and V (9) stay in host memory (pinned for
 * the copies to overlap) and their b x b blocks pass through an HBM cache of
 * as many blocks as device_bytes (10) holds beyond the fixed scratch, with
 * least-recently-used replacement and write-back of modified blocks; loads
 * and write-backs run on two copy streams beside the compute streams.
 * device_bytes >= randutv_ooc_ab_min_device_bytes (eight blocks).
 * io (12, HOST int64[3], optional): blocks read, blocks written, bytes
 * copied.  Synchronous; returns 0, a device status or -i. */
size_t randutv_ooc_ab_min_device_bytes(int64_t m, int64_t n, int b, int nstreams);
int randutv_factor_ooc_ab(int64_t m, int64_t n, double* A, int64_t lda, int b, int q,
                          uint64_t seed, double* U, double* V, size_t device_bytes, int nstreams,
                          int64_t* io, void* stream);

/* I/O of the dispatchers of §3.2.4 on the first max_tasks tasks (all when
 * negative) of that list, with every block held in an external store:
 * cache_blocks == 0 is the traditional dispatcher (per task, every input
 * block read and every output block written); cache_blocks > 0 keeps that
 * many blocks with least-recently-used replacement (ties: lowest slot),
 * writing a replaced block back only when it was modified.  reads, writes:
 * HOST int64 outputs.  trace (HOST, max_tasks * cache_blocks, or NULL): the
 * block in every slot after each task (-1 = empty).  Returns 0, -i for a
 * bad argument, or RANDUTV_EUNSUPPORTED when one task needs more blocks than
 * the cache holds. */
int randutv_ab_io(int64_t m, int64_t n, int b, int q, int want_u, int want_v, int64_t max_tasks,
                  int64_t cache_blocks, int64_t* reads, int64_t* writes, int64_t* trace);

/* ------------------------------------------------------------- utilities -- */

/* Bytes of library scratch one factorization of this shape needs. */
size_t randutv_workspace_bytes(int64_t m, int64_t n, int b, int prec);

/* Frees the library's scratch on every device it was allocated on. */
void randutv_finalize(void);

/* Short description of a status code. */
const char* randutv_strerror(int status);

/* Text of the last CUDA error seen by this thread ("" if none). */
const char* randutv_last_error(void);

/* Number of kernel launches issued by this process since the last reset. */
uint64_t randutv_launch_count(int reset);

/* Failure-detection self-test: launches one CTA at a grid barrier sized for
 * two CTAs on `stream`, so that the count it waits on never completes.  The
 * wait is bounded (about two seconds), after which the kernel records
 * RANDUTV_ETIMEOUT and returns, leaving the context usable.  Returns
 * RANDUTV_ETIMEOUT when that happened as designed; any other device status
 * as it is (its site in randutv_last_error); -100 when the wait completed
 * without a timeout being recorded. */
int randutv_selftest_wait_timeout(void* stream);

/* Tracing.  While enabled (on != 0), every kernel launch of the library is
 * bracketed by a pair of CUDA events on its stream and tagged with its kernel
 * class and the algorithmic flops and bytes of that launch.  Enabling clears
 * the records.  Timing adds two event records per launch. */
void randutv_profile_enable(int on);

/* Synchronizes on the recorded events and writes, per kernel class c
 * (0 <= c < nclass), out[4c..4c+3] = {launches, milliseconds, flops, bytes},
 * then clears the records.  Returns the number of classes the library
 * defines (write at most nclass of them), or a status code < 0 / > 0. */
int randutv_profile_read(double* out, int nclass);

/* Name of kernel class `cls` ("dgemm", "jacobi_svd", ...). */
const char* randutv_profile_class_name(int cls);

#ifdef __cplusplus
}
#endif

#endif /* RANDUTV_H */
