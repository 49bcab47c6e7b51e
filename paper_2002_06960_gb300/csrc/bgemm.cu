// Tensor-core GEMM for the mixed-precision path (tcgen05, TMEM, TMA).
//
//   C[M x N] (+)= alpha * sum_{(i,j) in pairs} op(A_i)[M x K] * B_j[K x N]
//
// A_i, B_j are BF16 "planes" of FP32-level matrices: X = X_0 + X_1 + X_2 with
// X_0 = bf16(X), X_1 = bf16(X - X_0), X_2 = bf16(X - X_0 - X_1), 8 significant
// bits each.  One plane gives a BF16 product (the sketch and power products
// of §3.1, V-hat step 2); three planes with the six pairs i + j <= 2 give the
// product to FP32 accuracy (the compact-WY updates of Fig. 2), with FP32
// accumulation in tensor memory throughout.
//
// Operand layout (column-major sources, loaded by TMA with 128-byte swizzle):
//   B is always K-major: B(k, n) = Y[k + n ldy] for a column-major Y.
//   A is K-major when op(A) = X^T (A(m, k) = X[k + m ldx]) and MN-major when
//   op(A) = X (A(m, k) = X[m + k ldx]); both are BF16 (kind::f16), for which
//   the MMA takes either major-ness.
// Tile 128 x 64 x 64 (BM x BN x BK), cta_group::1; tensor memory holds eight
// accumulators of 128 lanes x BN FP32 columns: two for the leading product
// A_0 B_0 (one per K step, alternating) and six chains for the correction
// products of the split (one segment of K steps at a time); a one-pair
// product spreads each tile over all eight, so that every FP32 accumulation
// in TMEM stays short.  Warp 0 issues TMA loads (and owns the TMEM
// allocation), warp 1 issues the MMAs, and warps 2-9 drain the accumulators,
// two warps per 32-lane quadrant, each on half the columns; in plane updates
// each of them also loads and stores its own 32 x 32 block of the output
// planes by TMA.  An FP32 output with few tiles can split K into chunks run
// as extra tiles, whose partial products a second kernel sums in a fixed
// order.
// Every mbarrier wait is bounded; on timeout the kernel records
// RANDUTV_ETIMEOUT, lets its copies in flight land, frees TMEM and returns.
#include <algorithm>
#include <cstring>

#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "common.cuh"
#include "mixed.h"
#include "tcgen05.cuh"

namespace rutv {

namespace {

constexpr int BM = 128, BN = 64, BK = 64;
constexpr int EPI_WARPS = 8;              // two per TMEM lane quadrant
constexpr int EPI_COLS = BN * 4 / EPI_WARPS;  // columns drained by one epilogue warp
constexpr int THREADS = 64 + 32 * EPI_WARPS;
constexpr int CSEG = 16;                  // K steps per correction segment
constexpr int A_TILE = BM * BK * 2;  // 16 KiB
constexpr int B_TILE = BN * BK * 2;  // 8 KiB
constexpr int kCorChains = 6;        // six pairs: correction accumulators
constexpr int kOneChains = 8;        // one pair: accumulators of a tile
constexpr int kTmemCols = 8 * BN;    // eight accumulators of BN columns (all of TMEM)
constexpr int C_ELEMS = BM * BN;     // one output plane tile (mode 1)
constexpr int C_TILE = C_ELEMS * 2;  // its bytes
constexpr int C_ROWS = 32;           // rows of one quadrant's slice (load box C_ROWS x BN)
constexpr int C_SLICE = C_ROWS * BN; // elements of a slice, column-major (ld C_ROWS); each
                                     // epilogue warp stores its half (box C_ROWS x EPI_COLS)

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

// Instruction descriptor, kind::f16: BF16 x BF16 -> FP32, M = 128, N = 128.
__device__ __forceinline__ uint32_t instr_desc(int a_mn_major) {
  uint32_t d = 0;
  d |= 1u << 4;                    // D format F32
  d |= 1u << 7;                    // A format BF16
  d |= 1u << 10;                   // B format BF16
  d |= (uint32_t)a_mn_major << 15; // A major-ness (0 = K, 1 = MN)
  d |= 0u << 16;                   // B K-major
  d |= (uint32_t)(BN >> 3) << 17;  // N / 8
  d |= (uint32_t)(BM >> 4) << 24;  // M / 16
  return d;
}

// TMA store of a 2-D box from shared memory (bulk-group completion).
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, const void* src, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(
          (uint64_t)map),
      "r"(smem_u32(src)), "r"(x), "r"(y)
      : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// wait until the committed bulk stores have finished reading shared memory
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
// wait until the committed bulk stores are complete
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// Error-free transformation of a sum: s + e == a + b exactly (Knuth's two-sum).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float z = s - a;
  e = (a - (s - z)) + (b - z);
}

struct BgemmParams {
  CUtensorMap ta[3];
  CUtensorMap tb[3];
  CUtensorMap tcs[3];  // mode 1: the output planes, box C_ROWS x EPI_COLS, no swizzle
  int M, N, K;
  int tiles_n, ntiles, ksteps;
  int ksplit, kchunk;      // split K: tile t = (output tile) * ksplit + chunk, kchunk K steps each
  int64_t split_stride;    // elements between the partial products of two chunks (mode 0)
  int na, nb, npairs;   // planes of A and B, and pairs (the kernel's template argument)
  int a_mn;            // A MN-major
  int a_x0, a_y0;      // coordinate offsets of A's source (x = source row, y = source col)
  int b_x0, b_y0;
  int stages;
  int out_upper;       // skip tiles wholly below the diagonal (their C is not wanted)
  int a_upper;         // op(A) upper triangular: K from the tile's first row
  int b_upper;         // B(k, n) = 0 for k > n: K up to the tile's last column
  int b_lower;         // B(k, n) = 0 for k < n: K from the tile's first column
  int mode;            // 0: C = alpha acc + beta C (FP32); 1: planes += alpha acc
  float alpha, beta;
  float* C;            // mode 0
  int64_t ldc;
  unsigned* err;
};

// Output tile `tile` of the persistent order (with split K: output tile
// tile / ksplit, K chunk tile % ksplit): its corner and its K steps [kb, ke);
// false when the tile is skipped (wholly below the diagonal with out_upper, or
// no K step that can contribute).
__device__ __forceinline__ bool tile_range(const BgemmParams& p, int tile, int& m0, int& n0,
                                           int& kb, int& ke) {
  const int z = tile % p.ksplit;
  tile /= p.ksplit;
  m0 = (tile / p.tiles_n) * BM;
  n0 = (tile % p.tiles_n) * BN;
  if (p.out_upper && m0 >= n0 + BN) return false;
  kb = z * p.kchunk;
  ke = min(p.ksteps, kb + p.kchunk);
  if (p.a_upper) kb = max(kb, m0 / BK);
  if (p.b_lower) kb = max(kb, n0 / BK);
  if (p.b_upper) ke = min(ke, (n0 + BN + BK - 1) / BK);
  return kb < ke;
}

// Persistent over output tiles (tile t -> rows (t / tiles_n) BM, columns
// (t % tiles_n) BN).
//
// Six pairs (FP32-level products): the leading product A_0 B_0 starts a fresh
// TMEM accumulator every K step of BK, alternating between two, and the
// epilogue warps add each step's result into a running sum held in registers
// as an unevaluated FP32 pair (s, c) with a two-sum.  The accumulation inside
// the tensor core adds each K = 16 product into FP32 with a bias, so its
// error grows like (K / 16) ulp; drained every 64 it stays within a few ulp,
// and the running sum is exact to about FP32^2.  The five correction
// products, about 2^-8 of the leading one, accumulate in TMEM over segments
// of up to CSEG K steps (K = 1024) spread over six chains, so each chain adds
// about 55 terms and its error stays below 2^-8 x 64 ulp of the result; the
// epilogue drains them once per segment into the compensation c.
//
// One pair (BF16 products): eight chains per tile over all of K, summed once.
//
// The epilogue's output of one tile overlaps the main loop of the next.
// Planes of the split in pair q of the six (i + j <= 2): A_i and B_j.
__device__ constexpr int pair_a(int q) { return q == 2 || q == 3 ? 1 : (q == 5 ? 2 : 0); }
__device__ constexpr int pair_b(int q) { return q == 1 || q == 3 ? 1 : (q == 4 ? 2 : 0); }

// NP = 6 (three planes per operand, six pairs) or 1 (one plane): the pair
// tables, the stage layout and every chain index are compile-time constants,
// so the MMA warp issues a straight run of tcgen05.mma per K step.
template <int NP>
__global__ void __launch_bounds__(THREADS, 1) bgemm_kernel(const __grid_constant__ BgemmParams p) {
  static_assert(NP == 1 || NP == 6, "one or six pairs");
  constexpr int NPL = (NP == 6) ? 3 : 1;          // planes per operand
  constexpr int per_stage = NPL * (A_TILE + B_TILE);
  constexpr bool kOnePair = (NP == 1);
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  // 1024-byte aligned tile area
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  // mode 1: the output tile's three planes (column-major BM x BN each) follow the stages
  __nv_bfloat16* ctile = (__nv_bfloat16*)(smem + (size_t)p.stages * per_stage);
  const size_t ctile_bytes = (p.mode == 1) ? (size_t)C_TILE * 3 : 0;
  uint64_t* full = (uint64_t*)(smem + (size_t)p.stages * per_stage + ctile_bytes);
  uint64_t* empty = full + p.stages;
  uint64_t* acc_full = empty + p.stages;  // [2] lead buffers (six pairs)
  uint64_t* acc_empty = acc_full + 2;     // [2]
  uint64_t* cor_full = acc_empty + 2;     // the chains of a segment (six pairs) or tile (one pair)
  uint64_t* cor_empty = cor_full + 1;
  uint64_t* mma_done = cor_empty + 1;
  uint64_t* cw = mma_done + 1;            // [EPI_WARPS] mode 1: a warp's block of the planes loaded
  uint32_t* tmem_slot = (uint32_t*)(cw + EPI_WARPS);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < p.stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], EPI_WARPS);  // one arrival per epilogue warp
    }
    mbar_init(cor_full, 1);
    mbar_init(cor_empty, EPI_WARPS);
    mbar_init(mma_done, 1);
    for (int e = 0; e < EPI_WARPS; ++e) mbar_init(&cw[e], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      int g = 0;   // K steps issued over all tiles of this CTA
      bool run = true;
      for (int tile = blockIdx.x; run && tile < p.ntiles; tile += gridDim.x) {
        int m0, n0, kb, ke;
        if (!tile_range(p, tile, m0, n0, kb, ke)) continue;
        for (int ks = kb; ks < ke; ++ks, ++g) {
          const int s = g % p.stages;
          const int round = g / p.stages;
          if (round > 0 && !mbar_wait(&empty[s], (uint32_t)((round - 1) & 1), p.err, 11)) {
            run = false;
            break;
          }
          uint8_t* st = smem + (size_t)s * per_stage;
          mbar_expect_tx(&full[s], (uint32_t)per_stage);
          const int k0 = ks * BK;
#pragma unroll
          for (int i = 0; i < NPL; ++i) {
            uint8_t* dst = st + i * A_TILE;
            if (p.a_mn) {
              tma_load_2d(dst, &p.ta[i], &full[s], p.a_x0 + m0, p.a_y0 + k0);
              tma_load_2d(dst + A_TILE / 2, &p.ta[i], &full[s], p.a_x0 + m0 + 64, p.a_y0 + k0);
            } else {
              tma_load_2d(dst, &p.ta[i], &full[s], p.a_x0 + k0, p.a_y0 + m0);
            }
          }
#pragma unroll
          for (int j = 0; j < NPL; ++j) {
            uint8_t* dst = st + NPL * A_TILE + j * B_TILE;
            tma_load_2d(dst, &p.tb[j], &full[s], p.b_x0 + k0, p.b_y0 + n0);
          }
        }
      }
      // let every copy issued land before the CTA can exit
      for (int k = (g > p.stages ? g - p.stages : 0); k < g; ++k) {
        mbar_wait(&full[k % p.stages], (uint32_t)((k / p.stages) & 1), p.err, 12);
      }
    }
  } else if (warp == 1) {
    // ----------------------------------------------------------------- MMA
    // The MMAs of a step go round-robin into several accumulators (chains)
    // that the epilogue sums: six pairs put A_0 B_0 into the step's lead
    // buffer and the 20 correction MMAs into six chains; one pair spreads a
    // tile's MMAs over eight chains.  One thread issues every MMA of the CTA,
    // and per-MMA work in that thread (indexed parameter loads, descriptor
    // arithmetic) held the tensor pipe back, so the issue loop is unrolled
    // with compile-time pairs and chains and each descriptor is one add.
    if (lane == 0) {
      const uint32_t idesc = instr_desc(p.a_mn);
      // descriptor steps of one K = 16 slice (in 16-byte units) and A's leading offset
      const int a_kstep = p.a_mn ? 2048 / 16 : 32 / 16;
      const uint32_t a_lbo = p.a_mn ? (uint32_t)(A_TILE / 2) : 16u;
      int g = 0;   // K steps over all tiles of this CTA
      int sg = 0;  // chain groups committed (segments, or tiles for one pair)
      bool run = true;
      for (int tile = blockIdx.x; run && tile < p.ntiles; tile += gridDim.x) {
        int m0, n0, kb, ke;
        if (!tile_range(p, tile, m0, n0, kb, ke)) continue;
        if constexpr (kOnePair) {
          // chains free once the previous tile's have been drained
          if (sg > 0 && !mbar_wait(cor_empty, (uint32_t)((sg - 1) & 1), p.err, 16)) {
            run = false;
            break;
          }
          for (int ks = kb; ks < ke; ++ks, ++g) {
            const int s = g % p.stages;
            if (!mbar_wait(&full[s], (uint32_t)((g / p.stages) & 1), p.err, 13)) {
              run = false;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t st = smem_u32(smem + (size_t)s * per_stage);
            const uint64_t a0 = smem_desc(st, a_lbo, 1024);
            const uint64_t b0 = smem_desc(st + A_TILE, 16, 1024);
            // MMA i of the tile goes to chain i mod 8: steps alternate between
            // chains 0-3 and 4-7, and the first two steps start them
            const uint32_t half = (uint32_t)((ks - kb) & 1) * 4u;
            const uint32_t acc_on = (ks - kb >= 2) ? 1u : 0u;
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk)
              mma_bf16(tmem + (half + (uint32_t)kk) * (uint32_t)BN, a0 + (uint64_t)(kk * a_kstep),
                       b0 + (uint64_t)(kk * 2), idesc, acc_on);
            mma_commit(&empty[s]);
          }
          if (!run) break;
          mma_commit(cor_full);
          ++sg;
        } else {
          for (int ks = kb; ks < ke; ++ks, ++g) {
            const int buf = g & 1, use = g >> 1;
            const int seg_pos = (ks - kb) % CSEG;
            const bool seg_end = (seg_pos == CSEG - 1) || (ks == ke - 1);
            if (use > 0 && !mbar_wait(&acc_empty[buf], (uint32_t)((use - 1) & 1), p.err, 16)) {
              run = false;
              break;
            }
            if (seg_pos == 0) {
              // the previous segment's chains must have been drained
              if (sg > 0 && !mbar_wait(cor_empty, (uint32_t)((sg - 1) & 1), p.err, 20)) {
                run = false;
                break;
              }
            }
            const int s = g % p.stages;
            if (!mbar_wait(&full[s], (uint32_t)((g / p.stages) & 1), p.err, 13)) {
              run = false;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t st = smem_u32(smem + (size_t)s * per_stage);
            const uint64_t a0 = smem_desc(st, a_lbo, 1024);
            const uint64_t b0 = smem_desc(st + NPL * A_TILE, 16, 1024);
            const uint32_t fresh = (seg_pos == 0) ? 1u : 0u;  // the segment starts its chains
  #pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
  #pragma unroll
              for (int q = 0; q < NP; ++q) {
                const uint64_t ad = a0 + (uint64_t)((pair_a(q) * A_TILE) >> 4) + (uint64_t)(kk * a_kstep);
                const uint64_t bd = b0 + (uint64_t)((pair_b(q) * B_TILE + kk * 32) >> 4);
                if (q == 0) {
                  mma_bf16(tmem + (uint32_t)(buf * BN), ad, bd, idesc, kk > 0 ? 1u : 0u);
                } else {
                  // correction MMA c = 5 kk + q - 1 of the step goes to chain c mod 6
                  const int c = (NP - 1) * kk + q - 1;
                  mma_bf16(tmem + (uint32_t)((2 + c % kCorChains) * BN), ad, bd, idesc,
                           (fresh && c < kCorChains) ? 0u : 1u);
                }
              }
            }
            mma_commit(&acc_full[buf]);  // the step's leading product is ready
            mma_commit(&empty[s]);       // stage s is free once these MMAs have read it
            if (seg_end) {
              mma_commit(cor_full);      // the segment's corrections are ready
              ++sg;
            }
          }
        }
      }
      mma_commit(mma_done);
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int ew = warp - 2;                          // epilogue warp index
    const int qd = warp & 3;                          // TMEM lane quadrant this warp may access
    const int c0 = ((warp - 2) >> 2) * EPI_COLS;      // its columns of the tile (warps 2..)
    const uint32_t lane_base = (uint32_t)(qd * 32) << 16;
    int g = 0, sg = 0;
    int tl = 0;  // tiles of this CTA
    bool ok = true;
    for (int tile = blockIdx.x; ok && tile < p.ntiles; tile += gridDim.x) {
      int m0, n0, kb, ke;
      if (!tile_range(p, tile, m0, n0, kb, ke)) continue;
      // mode 1: this warp's block of the output planes (32 rows x EPI_COLS),
      // loaded now so that the copy overlaps the drain; the previous tile's
      // store has finished reading the buffer (bulk_wait_read below)
      __nv_bfloat16* sl0 = ctile + (size_t)qd * C_SLICE + (size_t)c0 * C_ROWS;
      if (p.mode == 1 && lane == 0) {
        mbar_expect_tx(&cw[ew], (uint32_t)(3 * C_ROWS * EPI_COLS * 2));
        for (int i = 0; i < 3; ++i)
          tma_load_2d(sl0 + (size_t)i * C_ELEMS, &p.tcs[i], &cw[ew], m0 + qd * C_ROWS, n0 + c0);
      }
      const bool cpending = (p.mode == 1);
      float sum[EPI_COLS], cmp[EPI_COLS];
#pragma unroll
      for (int i = 0; i < EPI_COLS; ++i) { sum[i] = 0.f; cmp[i] = 0.f; }
      if (kOnePair) {
        // the chains that received MMAs (fewer than kOneChains when K is short)
        const int nch = min(kOneChains, (BK / 16) * (ke - kb));
        bool w = mbar_wait(cor_full, (uint32_t)(sg & 1), p.err, 14);
        ok = __all_sync(0xffffffffu, w) && ok;
        if (ok) {  // on failure fall through to the check below (copies in flight)
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          for (int ch = 0; ch < nch; ++ch) {
            float v[EPI_COLS];
#pragma unroll
            for (int cc = 0; cc < EPI_COLS; cc += 32)
              tmem_ld32(tmem + lane_base + (uint32_t)(ch * BN + c0 + cc), v + cc);
#pragma unroll
            for (int i = 0; i < EPI_COLS; ++i) sum[i] += v[i];
          }
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          __syncwarp();
          if (lane == 0) mbar_arrive(cor_empty);
          ++sg;
        }
      }
      for (int ks = kb; !kOnePair && ks < ke; ++ks, ++g) {
        const int buf = g & 1, use = g >> 1;
        const int seg_pos = (ks - kb) % CSEG;
        const bool seg_end = (seg_pos == CSEG - 1) || (ks == ke - 1);
        bool w = mbar_wait(&acc_full[buf], (uint32_t)(use & 1), p.err, 14);
        ok = __all_sync(0xffffffffu, w) && ok;
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        float v[EPI_COLS];
#pragma unroll
        for (int cc = 0; cc < EPI_COLS; cc += 32)
          tmem_ld32(tmem + lane_base + (uint32_t)(buf * BN + c0 + cc), v + cc);
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(&acc_empty[buf]);  // the buffer is free again
#pragma unroll
        for (int i = 0; i < EPI_COLS; ++i) {
          float t, e;
          two_sum(sum[i], v[i], t, e);
          sum[i] = t;
          cmp[i] += e;
        }
        if (seg_end) {
          w = mbar_wait(cor_full, (uint32_t)(sg & 1), p.err, 21);
          ok = __all_sync(0xffffffffu, w) && ok;
          if (!ok) break;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          for (int ch = 0; ch < kCorChains; ++ch) {
#pragma unroll
            for (int cc = 0; cc < EPI_COLS; cc += 32)
              tmem_ld32(tmem + lane_base + (uint32_t)((2 + ch) * BN + c0 + cc), v + cc);
#pragma unroll
            for (int i = 0; i < EPI_COLS; ++i) cmp[i] += v[i];
          }
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          __syncwarp();
          if (lane == 0) mbar_arrive(cor_empty);
          ++sg;
        }
      }
      // warp-uniform: the lanes must not split before the next tcgen05.ld
      if (__any_sync(0xffffffffu, !ok || *(volatile unsigned*)p.err != 0)) {
        // let this warp's copy in flight land before the CTA can exit
        if (cpending && lane == 0) mbar_wait(&cw[ew], (uint32_t)(tl & 1), p.err, 18);
        break;
      }
      // the tile's sum, rounded once to FP32
#pragma unroll
      for (int i = 0; i < EPI_COLS; ++i) sum[i] += cmp[i];
      const int row = m0 + qd * 32 + lane;
      if (row < p.M) {
        if (p.mode == 0) {
          // read this row's C first: a store may alias the next column's
          // load, so interleaved they would wait one by one
          float* crow = p.C + (int64_t)(tile % p.ksplit) * p.split_stride + (int64_t)row +
                        (int64_t)(n0 + c0) * p.ldc;
          const int ncol = min(EPI_COLS, p.N - (n0 + c0));
          if (p.beta != 0.f) {
            float cv[EPI_COLS];
#pragma unroll
            for (int i = 0; i < EPI_COLS; ++i) cv[i] = (i < ncol) ? crow[(int64_t)i * p.ldc] : 0.f;
#pragma unroll
            for (int i = 0; i < EPI_COLS; ++i) sum[i] = fmaf(p.beta, cv[i], p.alpha * sum[i]);
          } else {
#pragma unroll
            for (int i = 0; i < EPI_COLS; ++i) sum[i] *= p.alpha;
          }
#pragma unroll
          for (int i = 0; i < EPI_COLS; ++i)
            if (i < ncol) crow[(int64_t)i * p.ldc] = sum[i];
        }
      }
      if (p.mode == 1) {
        // this warp's 32 rows x EPI_COLS columns of the tile's planes, in shared
        // memory (zero past the matrix edge); each warp stores its own block
        // back, so the epilogue warps never wait on one another
        const bool w = mbar_wait(&cw[ew], (uint32_t)(tl & 1), p.err, 19);
        if (__any_sync(0xffffffffu, !w)) break;
#pragma unroll
        for (int i = 0; i < EPI_COLS; ++i) {
          const int o = i * C_ROWS + lane;
          // X + alpha acc carried as hi + lo, then split into three planes
          const float x0 = __bfloat162float(sl0[o]);
          const float xr = __bfloat162float(sl0[C_ELEMS + o]) + __bfloat162float(sl0[2 * C_ELEMS + o]);
          float hi, lo;
          two_sum(x0, p.alpha * sum[i], hi, lo);
          lo += xr;
          float y, ey;
          two_sum(hi, lo, y, ey);
          const __nv_bfloat16 h0 = __float2bfloat16_rn(y);
          const float rr = (y - __bfloat162float(h0)) + ey;
          const __nv_bfloat16 h1 = __float2bfloat16_rn(rr);
          const __nv_bfloat16 h2 = __float2bfloat16_rn(rr - __bfloat162float(h1));
          sl0[o] = h0;
          sl0[C_ELEMS + o] = h1;
          sl0[2 * C_ELEMS + o] = h2;
        }
        fence_proxy_async();  // the writes above are read by the TMA stores below
        __syncwarp();
        if (lane == 0) {
          for (int i = 0; i < 3; ++i)
            tma_store_2d(&p.tcs[i], sl0 + (size_t)i * C_ELEMS, m0 + qd * C_ROWS, n0 + c0);
          bulk_commit();
          bulk_wait_read();  // this block may be overwritten from here on
        }
        __syncwarp();
      }
      ++tl;
    }
    // this warp's last stores must be complete before the CTA exits
    if (p.mode == 1 && lane == 0) bulk_wait_all();
  }

  // teardown: all MMAs must have completed before TMEM is released
  __syncthreads();
  if (warp == 0) {
    mbar_wait(mma_done, 0, p.err, 15);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols));
  }
}

// C = alpha sum_z P_z (the split-K partial products, M x N each, ld M), in
// the order z = 0, 1, ...; columns by grid.y.
__global__ void splitk_sum_kernel(int M, int N, int ks, const float* __restrict__ P, float alpha,
                                  float* __restrict__ C, int64_t ldc) {
  const int64_t MN = (int64_t)M * N;
  for (int j = blockIdx.y; j < N; j += gridDim.y)
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x) {
      const int64_t o = i + (int64_t)j * M;
      float s = 0.f;
      for (int z = 0; z < ks; ++z) s += P[z * MN + o];
      C[i + (int64_t)j * ldc] = alpha * s;
    }
}

// ---------------------------------------------------------------- host side

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

int get_encode() {
  if (g_encode) return 0;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  RUTV_CK(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                           cudaEnableDefault, &q));
  if (q != cudaDriverEntryPointSuccess || !fn) return RANDUTV_ECUDA;
  g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  return 0;
}

}  // namespace

// Tensor map of a column-major BF16 matrix (rows x cols, ld elements), box
// {64 rows, box_cols columns}, 128-byte swizzle.  ld must be a multiple of 8.
namespace {
int make_tmap_box(CUtensorMap* map, const __nv_bfloat16* base, int64_t rows, int64_t cols,
                  int64_t ld, int box_rows, int box_cols, CUtensorMapSwizzle swz) {
  RUTV_TRY(get_encode());
  if (((uintptr_t)base & 15) || (ld % 8) != 0) return RANDUTV_EUNSUPPORTED;
  cuuint64_t dims[2] = {(cuuint64_t)rows, (cuuint64_t)cols};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {(cuuint32_t)box_rows, (cuuint32_t)box_cols};
  cuuint32_t estr[2] = {1u, 1u};
  CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)base, dims, strides, box,
                        estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_last_error("cuTensorMapEncodeTiled failed");
    return RANDUTV_ECUDA;
  }
  return 0;
}
}  // namespace

int make_tmap_bf16(CUtensorMap* map, const __nv_bfloat16* base, int64_t rows, int64_t cols,
                   int64_t ld, int box_cols) {
  RUTV_TRY(get_encode());
  if (((uintptr_t)base & 15) || (ld % 8) != 0) return RANDUTV_EUNSUPPORTED;
  cuuint64_t dims[2] = {(cuuint64_t)rows, (cuuint64_t)cols};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {64u, (cuuint32_t)box_cols};
  cuuint32_t estr[2] = {1u, 1u};
  CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)base, dims, strides, box,
                        estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_last_error("cuTensorMapEncodeTiled failed");
    return RANDUTV_ECUDA;
  }
  return 0;
}

int launch_bgemm(const BgemmOperand& A, const BgemmOperand& B, int M, int N, int K, int pairs_mode,
                 const BgemmOut& out, unsigned* err, cudaStream_t st, int max_ctas,
                 const BgemmTri& tri) {
  if (M <= 0 || N <= 0) return 0;
  if (K <= 0) return RANDUTV_EUNSUPPORTED;  // no product to accumulate
  if ((tri.a_upper || tri.b_upper || tri.b_lower) && !(out.mode == 0 && out.beta == 1.f))
    return RANDUTV_EUNSUPPORTED;  // skipped K ranges leave C as it is
  BgemmParams p;
  memset(&p, 0, sizeof p);
  p.na = A.nplanes;
  p.nb = B.nplanes;
  for (int i = 0; i < p.na; ++i) {
    // A K-major: source X (K rows x M cols), box {64 K, 128 M}
    // A MN-major: source X (M rows x K cols), box {64 M, 64 K}
    RUTV_TRY(make_tmap_bf16(&p.ta[i], A.planes[i], A.rows, A.cols, A.ld, A.mn_major ? 64 : 128));
  }
  for (int j = 0; j < p.nb; ++j) {
    RUTV_TRY(make_tmap_bf16(&p.tb[j], B.planes[j], B.rows, B.cols, B.ld, BN));
  }
  p.M = M;
  p.N = N;
  p.K = K;
  if (pairs_mode == 3 && p.na == 3 && p.nb == 3) {
    p.npairs = 6;  // the pairs i + j <= 2 (pair_a, pair_b)
  } else {
    p.npairs = 1;
    p.na = p.nb = 1;
  }
  p.a_mn = A.mn_major;
  p.a_x0 = (int)A.x0;
  p.a_y0 = (int)A.y0;
  p.b_x0 = (int)B.x0;
  p.b_y0 = (int)B.y0;
  const int per_stage = p.na * A_TILE + p.nb * B_TILE;
  // mode 1 keeps the output tile's three planes in shared memory (TMA in and out)
  const size_t ctile_bytes = (out.mode == 1) ? (size_t)3 * C_TILE : 0;
  int stages = (int)((216 * 1024 - ctile_bytes) / per_stage);
  if (stages > 8) stages = 8;
  if (stages < 1) stages = 1;
  p.stages = stages;
  p.mode = out.mode;
  if (out.mode == 1) {
    for (int i = 0; i < 3; ++i)
      RUTV_TRY(make_tmap_box(&p.tcs[i], out.planes[i], M, N, out.ldp, C_ROWS, EPI_COLS,
                             CU_TENSOR_MAP_SWIZZLE_NONE));
  }
  p.alpha = out.alpha;
  p.beta = out.beta;
  p.C = out.C;
  p.ldc = out.ldc;
  p.err = err;
  const int tiles_m = (M + BM - 1) / BM;
  p.tiles_n = (N + BN - 1) / BN;
  p.ntiles = tiles_m * p.tiles_n;
  p.ksteps = (K + BK - 1) / BK;
  p.ksplit = 1;
  p.kchunk = p.ksteps;
  p.split_stride = 0;
  float* const c_final = out.C;
  if (out.mode == 0 && out.beta == 0.f && out.ksplit > 1 && out.splitk_ws &&
      !(tri.out_upper || tri.a_upper || tri.b_upper || tri.b_lower)) {
    int64_t ks = std::min<int64_t>(out.ksplit, p.ksteps);
    ks = std::min<int64_t>(ks, (int64_t)(out.splitk_floats / ((size_t)M * (size_t)N)));
    if (ks > 1) {
      p.kchunk = (int)((p.ksteps + ks - 1) / ks);
      p.ksplit = (p.ksteps + p.kchunk - 1) / p.kchunk;  // every chunk non-empty
      p.ntiles *= p.ksplit;
      p.C = out.splitk_ws;  // partial products, M x N each (ld M), summed below
      p.ldc = M;
      p.alpha = 1.f;
      p.split_stride = (int64_t)M * N;
    }
  }
  p.out_upper = tri.out_upper;
  p.a_upper = tri.a_upper;
  p.b_upper = tri.b_upper;
  p.b_lower = tri.b_lower;
  // MMA flops of the tiles and K steps that run (for tracing)
  double mma_flops = 2.0 * M * (double)N * K * p.npairs;
  if (tri.out_upper || tri.a_upper || tri.b_upper || tri.b_lower) {
    mma_flops = 0.0;
    for (int t = 0; t < tiles_m * p.tiles_n; ++t) {
      const int m0 = (t / p.tiles_n) * BM, n0 = (t % p.tiles_n) * BN;
      if (tri.out_upper && m0 >= n0 + BN) continue;
      int kb = 0, ke = p.ksteps;
      if (tri.a_upper) kb = std::max(kb, m0 / BK);
      if (tri.b_lower) kb = std::max(kb, n0 / BK);
      if (tri.b_upper) ke = std::min(ke, (n0 + BN + BK - 1) / BK);
      if (kb >= ke) continue;
      const double rows = std::min(BM, M - m0), cols = std::min(BN, N - n0);
      const double kk = std::min(ke * BK, K) - kb * BK;
      mma_flops += 2.0 * rows * cols * kk * p.npairs;
    }
  }
  // barriers: full and empty per stage, two lead, the chains' pair, mma_done,
  // one per epilogue warp; then the TMEM address
  const size_t smem =
      1024 + (size_t)stages * per_stage + ctile_bytes + (2 * stages + 7 + EPI_WARPS) * 8 + 16;
  const void* fn = (p.npairs == 6) ? (const void*)bgemm_kernel<6> : (const void*)bgemm_kernel<1>;
  RUTV_TRY(ensure_smem(fn, smem));
  // persistent: at most one CTA per SM (the shared memory allows no more)
  int cap = dev_info().sms;
  if (max_ctas > 0 && max_ctas < cap) cap = max_ctas;
  const int grid = p.ntiles < cap ? p.ntiles : cap;
  ProfScope prof(K_BGEMM, mma_flops,
                 2.0 * ((double)M * K * p.na + (double)K * N * p.nb) +
                     (out.mode == 0 ? 4.0 : 12.0) * M * (double)N,
                 st);
  if (p.npairs == 6) bgemm_kernel<6><<<grid, THREADS, smem, st>>>(p);
  else bgemm_kernel<1><<<grid, THREADS, smem, st>>>(p);
  note_launch();
  RUTV_CK(cudaGetLastError());
  if (p.ksplit > 1) {
    const int64_t bx = std::min<int64_t>((M + 255) / 256, 64);
    splitk_sum_kernel<<<dim3((unsigned)bx, (unsigned)std::min(N, 65535)), 256, 0, st>>>(
        M, N, p.ksplit, out.splitk_ws, out.alpha, c_final, out.ldc);
    note_launch();
    RUTV_CK(cudaGetLastError());
  }
  return 0;
}

}  // namespace rutv
