// randUTV by blocks (§3.2.2-3.2.4): the task list of randUTV_AB over b x b
// blocks, and the dispatchers that run it.  Host-side declarations shared by
// the analyzer (ab_tasks.cu) and the GPU executor (ab_exec.cu).
#pragma once

#include <stdint.h>

#include <vector>

namespace rutv {

// Kinds of blocks a task reads or writes.  A, U, V: tiles of the matrices
// (A holds T as it is formed).  G, Y, Z: tiles of the sketch, of its range
// product and of the power-iteration product of the current step.  B: the
// compact-WY factor of the QR of one Y tile (the paper's "B" blocks), C: of
// one A tile of the current block column ("C" blocks).  P, Q: the factors
// U_s and V_s of the small SVD of a step.
enum AbKind { AB_A = 0, AB_G, AB_Y, AB_Z, AB_B, AB_C, AB_P, AB_Q, AB_U, AB_V, AB_NKIND };

// A block is one int64: kind << 40 | i << 20 | j (i, j < 2^20).
inline int64_t ab_block(int kind, int64_t i, int64_t j) {
  return ((int64_t)kind << 40) | (i << 20) | j;
}
inline int ab_kind(int64_t blk) { return (int)(blk >> 40); }
inline int64_t ab_bi(int64_t blk) { return (blk >> 20) & 0xFFFFF; }
inline int64_t ab_bj(int64_t blk) { return blk & 0xFFFFF; }

// The operations of the task list (names as in the paper's figures where
// it prints them; the power-iteration product and the fold of U are the
// same kinds of products on other operands).
enum AbOp {
  OP_GEN = 0,     // Generate_normal_random:      G_i
  OP_TN_OZ,       // Gemm_tn_oz:  Y_j  = A_ij^T G_i   (or A_ij^T Z_i)
  OP_TN_OO,       // Gemm_tn_oo:  Y_j += A_ij^T G_i
  OP_NN_OZ,       // Z_i  = A_ij Y_j   (power iteration)
  OP_NN_OO,       // Z_i += A_ij Y_j
  OP_QR_DENSE,    // Comp_dense_QR of X_kk -> X_kk (R and vectors), S
  OP_QR_TD,       // Comp_td_QR of [R in X_kk; X_l] -> X_kk, X_l (vectors), S
  OP_RIGHT_DENSE, // Apply_right_Q_of_dense_QR:  X_rk <- X_rk Q
  OP_RIGHT_TD,    // Apply_right_Q_td_QR:  [X_rk X_rl] <- [X_rk X_rl] Q
  OP_LEFT_DENSE,  // Apply_left_Qt_of_dense_QR:  A_kj <- Q^T A_kj
  OP_LEFT_TD,     // Apply_left_Qt_of_td_QR:  [A_kj; A_ij] <- Q^T [A_kj; A_ij]
  OP_KEEP_UPPER,  // Keep_upper_triang
  OP_SET_ZERO,    // Set_to_zero
  OP_SVD,         // Svd_of_block:  A_kk = P diag(D) Q^T -> A_kk = diag(D), P, Q
  OP_ABTA,        // Gemm_abta:  A = B^T A   (row fold, B = P)
  OP_AABT,        // Gemm_aabt:  A = A Q     (column fold with V_s)
  OP_AAB,         // A = A P                 (fold of U with U_s)
  OP_NOPS
};

const char* ab_op_name(int op);

// Starts of the tiles along one dimension of `extent`, with p = min(m, n):
// multiples of b up to p (the block steps), then p + b t up to `extent`,
// followed by `extent` itself.  Every diagonal block is then one tile.
std::vector<int64_t> ab_tile_starts(int64_t extent, int64_t p, int64_t b);

struct AbTask {
  int op;
  int step;
  int nin, nout;
  int64_t in[4], out[4];
};

// The task list of randUTV_AB for an m x n matrix in blocks of b, q power
// iterations, with or without U and V.  Block steps and the last-block rule
// are those of the blocked algorithm (§3.1): a right transform when columns
// remain after the block, a left QR when rows remain below it, an SVD always.
std::vector<AbTask> ab_analyze(int64_t m, int64_t n, int64_t b, int q, bool want_u, bool want_v);

// I/O of a dispatcher that runs `tasks` with blocks kept in an external
// store.  cache_blocks == 0: the traditional dispatcher (every input read,
// every output written, per task).  cache_blocks > 0: a cache of that many
// blocks with least-recently-used replacement; a replaced block is written
// back only when it was modified.  trace (optional) receives, after each
// task, the block held by every cache slot (-1 for an empty slot).
struct AbIo {
  int64_t reads = 0, writes = 0;
};
AbIo ab_simulate(const std::vector<AbTask>& tasks, int64_t ntasks, int64_t cache_blocks,
                 std::vector<int64_t>* trace);

}  // namespace rutv
