// Mixed-precision path: BF16 planes, the tcgen05 GEMM and its helpers.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace rutv {

// A column-major FP32-level matrix held as three BF16 planes, X = X0+X1+X2.
// ld is a multiple of 8 so every column starts on a 16-byte boundary.
struct Planes {
  __nv_bfloat16* p[3] = {nullptr, nullptr, nullptr};
  int64_t rows = 0, cols = 0, ld = 0;
  __nv_bfloat16* at(int i, int64_t r, int64_t c) const { return p[i] + r + c * ld; }
};

inline int64_t pad8(int64_t x) { return (x + 7) / 8 * 8; }

// One GEMM operand: planes of a column-major source plus the coordinate
// offset (x0 = source row, y0 = source column) of the operand inside it.
// For A: mn_major = 0 means op(A) = X^T (K along source rows),
//        mn_major = 1 means op(A) = X   (M along source rows).
// For B: always K along source rows, N along source columns.
struct BgemmOperand {
  const __nv_bfloat16* planes[3] = {nullptr, nullptr, nullptr};
  int nplanes = 1;
  int64_t rows = 0, cols = 0, ld = 0;  // extent of the source
  int64_t x0 = 0, y0 = 0;
  int mn_major = 0;
};

// Epilogue: mode 0 writes FP32 C = alpha acc + beta C (column-major, ldc);
// mode 1 adds alpha acc to three output planes (column-major, ldp) and
// re-splits the sum.
struct BgemmOut {
  int mode = 0;
  float alpha = 1.f, beta = 0.f;
  float* C = nullptr;
  int64_t ldc = 0;
  __nv_bfloat16* planes[3] = {nullptr, nullptr, nullptr};
  int64_t ldp = 0;
  // mode 0 with beta = 0: split K over up to `ksplit` partial products held
  // in `splitk_ws` (ksplit M x N floats), then summed in a fixed order, for
  // outputs with too few tiles to occupy the SMs; capped by splitk_floats.
  int ksplit = 1;
  float* splitk_ws = nullptr;
  size_t splitk_floats = 0;
};

// Structure of the operands that lets tiles or K steps be skipped:
//   out_upper: only output tiles that reach the diagonal or above are wanted;
//   a_upper:   op(A) is upper triangular;
//   b_upper:   B(k, n) = 0 for k > n;  b_lower: B(k, n) = 0 for k < n.
// With a_upper, b_upper or b_lower a tile whose K range is empty is left as
// it is, which is the product only for mode 0 with beta = 1 (required).
struct BgemmTri {
  int out_upper = 0, a_upper = 0, b_upper = 0, b_lower = 0;
};

// pairs_mode 1: one BF16 product of plane 0 of A and B (accumulated over the
// whole K in tensor memory).  pairs_mode 3: the six products A_i B_j with
// i + j <= 2 of three planes each (FP32 accuracy; the accumulator is
// drained every 64 K into compensated sums).
// max_ctas: upper bound on the persistent grid (0 = one CTA per SM).
int launch_bgemm(const BgemmOperand& A, const BgemmOperand& B, int M, int N, int K,
                 int pairs_mode, const BgemmOut& out, unsigned* err, cudaStream_t st,
                 int max_ctas = 0, const BgemmTri& tri = BgemmTri());

int make_tmap_bf16(CUtensorMap* map, const __nv_bfloat16* base, int64_t rows, int64_t cols,
                   int64_t ld, int box_cols);

// ---- conversions (mixed_util.cu) ----
// dst planes (rows x cols at (r0, c0)) <- split(src), src FP32 column-major;
// trans: dst(i, j) <- src(j, i).
int split_f32(const float* src, int64_t lds, int64_t rows, int64_t cols, int trans,
              const Planes& dst, int64_t r0, int64_t c0, cudaStream_t st);
int split_f64(const double* src, int64_t lds, int64_t rows, int64_t cols, int trans,
              const Planes& dst, int64_t r0, int64_t c0, cudaStream_t st);
// dst (FP32 or FP64, column-major) <- planes block (rows x cols at (r0, c0)); trans as above.
int merge_f32(const Planes& src, int64_t r0, int64_t c0, int64_t rows, int64_t cols, int trans,
              float* dst, int64_t ldd, cudaStream_t st);
int merge_f64(const Planes& src, int64_t r0, int64_t c0, int64_t rows, int64_t cols, int trans,
              double* dst, int64_t ldd, cudaStream_t st);
// BF16 copy of an FP32 matrix scaled by 2^-e, e the exponent of its largest
// magnitude (an exact rescaling that keeps the power iteration in range).
int scaled_bf16(const float* src, int64_t lds, int64_t rows, int64_t cols, __nv_bfloat16* dst,
                int64_t ldd, float* scratch, cudaStream_t st);
int set_identity_planes(const Planes& X, cudaStream_t st);
int launch_check_finite_f32(int64_t rows, int64_t cols, const float* X, int64_t ld, unsigned* err,
                            cudaStream_t st);
int set_diag_planes(const Planes& T, int64_t k, int64_t bi, const double* D, cudaStream_t st);
// Final re-orthogonalisation: d = diag(X^T X) - 1 in FP64 (X FP32, n x n),
// and Phi = striu(E) + diag(d)/2 in BF16 (E FP32, read on and above the
// diagonal), with its transpose PhiT when PhiT is non-null.
int reorth_phi(const float* X, int64_t ldx, int64_t n, const float* E, int64_t lde, double* d,
               __nv_bfloat16* Phi, int64_t ldp, __nv_bfloat16* PhiT, int64_t ldpt,
               cudaStream_t st);
// Zeroes the off-diagonal entries of every b x b diagonal block of T (p = min(m, n)).
int zero_block_offdiag(float* T, int64_t ld, int64_t p, int64_t b, cudaStream_t st);
int philox_normal_bf16(uint64_t seed, uint32_t step, uint32_t mid, uint32_t sid, int64_t rows,
                       int64_t cols, __nv_bfloat16* G, int64_t ldg, cudaStream_t st);

}  // namespace rutv
