// SVD of the b x b diagonal block (Fig. 2: [A11, U_SVD, V_SVD] := SVD(A11);
// §3.1 step 3) by one-sided Jacobi (Hestenes 1958; Demmel & Veselic 1992 for
// the rotation and the stopping rule), in two phases:
//
//   1. FP32 sweeps on B (scaled by a power of two into the FP32 range) until
//      its columns are orthogonal to FP32 accuracy, the rotations accumulated
//      in V32.  FP32 runs at 64 times the FP64 rate of this part, and the
//      sweeps that take a dense block to near-orthogonal columns are most of
//      the work.  They run by blocks of columns (block_jacobi_f32_kernel),
//      so that a cluster barrier comes once per block pair rather than twice
//      per round of column pairs.
//   2. V32 is made orthogonal to FP64 accuracy by two Newton-Schulz steps
//      V <- V (3I - V^T V) / 2 (FP64 products), C = B V in FP64, and FP64
//      sweeps on C that start from V finish the job.  The columns of C are
//      already orthogonal to about 1e-6, so Jacobi's quadratic convergence
//      reaches FP64 accuracy within two or three sweeps.  Stopping rule and
//      outputs are those of a plain FP64 one-sided Jacobi, so the result does
//      not depend on phase 1 beyond rounding.
// Blocks of at most 32 columns skip phase 1.
//
// Phase 2 runs jacobi_kernel (templated on the arithmetic type) on one
// thread-block cluster of C CTAs.  CTA k holds rows [k R, (k+1) R) of the
// working matrix and of V in shared memory.  A sweep is b-1 rounds of the
// round-robin (circle) ordering, each rotating b/2 disjoint column pairs:
//   * every CTA writes the partial inner products (|a_p|^2, |a_q|^2, a_p.a_q)
//     of its rows for all pairs; cluster barrier;
//   * CTA k owns pairs [k ceil(npairs/C), (k+1) ceil(npairs/C)): it sums their
//     C partials in a fixed order through distributed shared memory, computes
//     the rotations and stores them into every CTA; cluster barrier;
//   * every CTA applies all the rotations to its own rows.
// Each rotation is computed once, so it is bitwise identical in every CTA, and
// each CTA moves O(npairs) words through the cluster per round (pulling every
// pair's partials into every CTA would move O(npairs C)).
//
// After phase 2: D_j = |c_j|, columns sorted by descending D (lowest index
// first on ties), U_j = c_j / D_j, and each column of V signed so that its
// entry of largest magnitude (lowest row on ties) is positive, U_j with it.
// Exactly-zero singular values get their U columns from a separate
// completion kernel (Gram-Schmidt of unit vectors).
#include <cooperative_groups.h>

#include "common.cuh"
#include "kernels.h"

namespace cg = cooperative_groups;

namespace rutv {

namespace {
constexpr int SVD_THREADS = 256;      // FP64 phase (few rows per CTA)
constexpr int SVD_THREADS_FP32 = 512; // FP32 phase (one to four CTAs)
constexpr int SVD_MAX_THREADS = 512;
constexpr int SVD_MAX_B = 256;
constexpr int SVD_DIRECT_B = 32;  // blocks up to this size skip the FP32 phase

struct JacArgs {
  int b;
  const double* B;   // input block (FP64), column-major
  int64_t ldb;
  const double* Vin; // initial V (b x b, ld b), or null for the identity
  float* V32;        // phase 1 output: V (b x b, ld b)
  double* D;         // phase 2 outputs
  double* Us;
  double* Vs;
  int max_sweeps;
  double tol;        // rotate while |a_p.a_q| > tol |a_p| |a_q|
  unsigned* info;    // phase 2: sweeps taken
};

template <typename Real>
size_t jac_smem_bytes(int b, int ncl) {
  const int P = (b + 1) & ~1, npairs = P / 2, R = (b + ncl - 1) / ncl, LDR = R + 1;
  return 4 * (size_t)P * sizeof(double)                                  // norms, vmax, vbest, D
         + (2 * (size_t)P * LDR + 5 * (size_t)npairs) * sizeof(Real)     // B, V, partials, rotations
         + 2 * (size_t)P * sizeof(int) + 64;                             // vrow, rankof
}

__device__ __forceinline__ double fmar(double x, double y, double z) { return fma(x, y, z); }

// Pair t of round `round` of the circle ordering on P columns (0 <= t < P/2,
// 0 <= round < P-1).
__device__ __forceinline__ void rr_pair(int round, int t, int P, int* p, int* q) {
  int a, c;
  if (t == 0) {
    a = P - 1;
    c = round;
  } else {
    a = round + t;
    if (a >= P - 1) a -= P - 1;
    c = round - t;
    if (c < 0) c += P - 1;
  }
  *p = a < c ? a : c;
  *q = a < c ? c : a;
}

__device__ double block_max(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double m = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
  __syncthreads();
  return m;
}

// Barrier across the cluster, or across the CTA when the cluster is one CTA.
__device__ __forceinline__ void cluster_barrier(cg::cluster_group& cl, int ncl) {
  if (ncl == 1) __syncthreads();
  else cl.sync();
}

// Rotation angle of a pair (Rutishauser's formula), in the phase's precision.
__device__ __forceinline__ void jac_rotation(double al, double be, double ga, double* c,
                                             double* s) {
  const double zeta = (be - al) / (2.0 * ga);
  const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + hypot(1.0, zeta));
  *c = 1.0 / sqrt(fma(t, t, 1.0));
  *s = *c * t;
}

template <typename Real, bool kFinal>
__global__ void __launch_bounds__(SVD_MAX_THREADS) jacobi_kernel(const JacArgs a) {
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int ncl = (int)cl.num_blocks();
  const int b = a.b, P = (b + 1) & ~1, npairs = P / 2;
  const int R = (b + ncl - 1) / ncl, LDR = R + 1;
  const int r0 = rank * R;
  const int nr = max(0, min(b, r0 + R) - r0);
  const int tid = threadIdx.x, nth = blockDim.x;

  extern __shared__ double smem[];
  double* npart = smem;               // [P] column norms^2 of own rows
  double* vmax = npart + P;           // [P] signed entry of largest |V| in own rows
  double* vbest = vmax + P;           // [P] same, over the cluster
  double* Dfull = vbest + P;          // [P]
  Real* Bl = reinterpret_cast<Real*>(Dfull + P);  // column j, local row i at Bl[j*LDR + i]
  Real* Vl = Bl + (size_t)P * LDR;
  Real* part = Vl + (size_t)P * LDR;  // [npairs][3]
  Real* rot = part + (size_t)npairs * 3;  // [npairs][2]: (c, s)
  int* vrow = reinterpret_cast<int*>(rot + (size_t)npairs * 2);
  int* rankof = vrow + P;
  __shared__ int s_rotated;
  __shared__ double s_red[SVD_MAX_THREADS / 32];

  // Phase 1 works on B 2^-e, e the exponent of max |B| (exact, and inside
  // the FP32 range whatever the scale of the block).
  double scale = 1.0;
  if (!kFinal) {
    double mx = 0.0;
    for (int e = tid; e < b * b; e += nth)
      mx = fmax(mx, fabs(a.B[(e % b) + (int64_t)(e / b) * a.ldb]));
    mx = block_max(mx, s_red);
    if (mx > 0.0) {
      int ex = 0;
      frexp(mx, &ex);
      scale = ldexp(1.0, -ex);
    }
  }
  for (int e = tid; e < P * LDR; e += nth) {
    const int j = e / LDR, i = e % LDR;
    const int gi = r0 + i;
    double bv = 0.0, vv = 0.0;
    if (i < nr && j < b) {
      bv = a.B[gi + (int64_t)j * a.ldb] * scale;
      vv = a.Vin ? a.Vin[gi + (int64_t)j * b] : ((gi == j) ? 1.0 : 0.0);
    }
    Bl[e] = (Real)bv;
    Vl[e] = (Real)vv;
  }
  if (tid == 0) s_rotated = 0;
  cl.sync();

  // Lanes per pair: a group of tpp consecutive lanes covers consecutive rows
  // of one column, and each group walks the pairs g = group, group + ngroups,
  // ...  (the trip count is the same for every group, so the shuffles run in
  // whole warps).  One CTA with many rows per pair: tpp = min(32, R), which
  // keeps a warp's shared-memory accesses conflict-free.  A cluster, with few
  // rows per CTA: as many pairs in flight as the block allows, so that a
  // round is one short pass rather than a chain of reductions.
  int tpp = 1;
  if (ncl == 1) {
    while (tpp < 32 && tpp < R) tpp *= 2;
  } else {
    while (tpp < 32 && tpp * 2 * npairs <= nth) tpp *= 2;
  }
  const int group = tid / tpp, sub = tid % tpp, ngroups = nth / tpp;
  const int pair_iters = (npairs + ngroups - 1) / ngroups;
  int NS = 1;
  while (NS < ncl) NS <<= 1;
  const int ppc = (npairs + ncl - 1) / ncl;  // pairs owned per CTA; ppc * NS <= 2 npairs <= nth
  const int own_pl = tid / NS, own_src = tid % NS;
  const int own_pair = rank * ppc + own_pl;
  const bool own_lane = tid < ppc * NS && own_pair < npairs;
  const double tol = a.tol;
  const Real tol_r = (Real)tol;

  int sweep = 0;
  for (; sweep < a.max_sweeps; ++sweep) {
    if (ncl == 1) {
      // One CTA holds every row: each group reduces its pair's sums by
      // shuffles (bit-identical in all its lanes), takes the rotation and
      // applies it; one block barrier per round.
      for (int round = 0; round < P - 1; ++round) {
        for (int it = 0; it < pair_iters; ++it) {
          const int g = group + it * ngroups;
          const bool act = g < npairs;
          int p = 0, q = 0;
          Real sa = 0, sb = 0, sc = 0;
          if (act) {
            rr_pair(round, g, P, &p, &q);
            const Real* bp = Bl + (size_t)p * LDR;
            const Real* bq = Bl + (size_t)q * LDR;
#pragma unroll 4
            for (int i = sub; i < nr; i += tpp) {
              const Real x = bp[i], y = bq[i];
              sa = fmar(x, x, sa);
              sb = fmar(y, y, sb);
              sc = fmar(x, y, sc);
            }
          }
          for (int o = tpp >> 1; o > 0; o >>= 1) {
            sa += __shfl_xor_sync(0xffffffffu, sa, o);
            sb += __shfl_xor_sync(0xffffffffu, sb, o);
            sc += __shfl_xor_sync(0xffffffffu, sc, o);
          }
          if (act && q < b && sc != (Real)0 && sc * sc > tol_r * tol_r * sa * sb) {
            Real c, s;
            jac_rotation(sa, sb, sc, &c, &s);
            if (sub == 0) s_rotated = 1;
            Real* bp = Bl + (size_t)p * LDR;
            Real* bq = Bl + (size_t)q * LDR;
            Real* vp = Vl + (size_t)p * LDR;
            Real* vq = Vl + (size_t)q * LDR;
#pragma unroll 4
            for (int i = sub; i < nr; i += tpp) {
              const Real x = bp[i], y = bq[i];
              bp[i] = fmar(c, x, -s * y);
              bq[i] = fmar(s, x, c * y);
              const Real u = vp[i], w = vq[i];
              vp[i] = fmar(c, u, -s * w);
              vq[i] = fmar(s, u, c * w);
            }
          }
        }
        __syncthreads();
      }
      const int any = s_rotated;
      __syncthreads();
      if (tid == 0) s_rotated = 0;
      __syncthreads();
      if (!any) break;
      continue;
    }
    for (int round = 0; round < P - 1; ++round) {
      // partial inner products over own rows, every pair
      for (int it = 0; it < pair_iters; ++it) {
        const int g = group + it * ngroups;
        const bool act = g < npairs;
        Real sa = 0, sb = 0, sc = 0;
        if (act) {
          int p, q;
          rr_pair(round, g, P, &p, &q);
          const Real* bp = Bl + (size_t)p * LDR;
          const Real* bq = Bl + (size_t)q * LDR;
          for (int i = sub; i < nr; i += tpp) {
            const Real x = bp[i], y = bq[i];
            sa = fmar(x, x, sa);
            sb = fmar(y, y, sb);
            sc = fmar(x, y, sc);
          }
        }
        for (int o = tpp >> 1; o > 0; o >>= 1) {
          sa += __shfl_xor_sync(0xffffffffu, sa, o);
          sb += __shfl_xor_sync(0xffffffffu, sb, o);
          sc += __shfl_xor_sync(0xffffffffu, sc, o);
        }
        if (act && sub == 0) {
          part[(size_t)g * 3] = sa;
          part[(size_t)g * 3 + 1] = sb;
          part[(size_t)g * 3 + 2] = sc;
        }
      }
      cluster_barrier(cl, ncl);
      // owned pairs: sum the partials of all CTAs (fixed shuffle tree, so every
      // lane of the group ends with the same sums) and broadcast the rotation
      {
        double al = 0.0, be = 0.0, ga = 0.0;
        if (own_lane && own_src < ncl) {
          const Real* rp =
              (ncl == 1 ? part : cl.map_shared_rank(part, own_src)) + (size_t)own_pair * 3;
          al = (double)rp[0];
          be = (double)rp[1];
          ga = (double)rp[2];
        }
        for (int o = NS >> 1; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          ga += __shfl_xor_sync(0xffffffffu, ga, o);
        }
        Real c = 1, s = 0;
        if (own_lane) {
          int pp, qq;
          rr_pair(round, own_pair, P, &pp, &qq);
          if (qq < b && ga != 0.0 && ga * ga > tol * tol * al * be)
            jac_rotation((Real)al, (Real)be, (Real)ga, &c, &s);
        }
        if (own_lane && own_src < ncl) {
          Real* rr = (ncl == 1 ? rot : cl.map_shared_rank(rot, own_src)) + (size_t)own_pair * 2;
          rr[0] = c;
          rr[1] = s;
          if (own_src == 0 && s != (Real)0) s_rotated = 1;
        }
      }
      cluster_barrier(cl, ncl);
      for (int it = 0; it < pair_iters; ++it) {
        const int g = group + it * ngroups;
        if (g >= npairs) break;  // no shuffles below: groups may leave early
        const Real c = rot[(size_t)g * 2], s = rot[(size_t)g * 2 + 1];
        if (s != (Real)0) {
          int p, q;
          rr_pair(round, g, P, &p, &q);
          Real* bp = Bl + (size_t)p * LDR;
          Real* bq = Bl + (size_t)q * LDR;
          Real* vp = Vl + (size_t)p * LDR;
          Real* vq = Vl + (size_t)q * LDR;
          for (int i = sub; i < nr; i += tpp) {
            const Real x = bp[i], y = bq[i];
            bp[i] = fmar(c, x, -s * y);
            bq[i] = fmar(s, x, c * y);
            const Real u = vp[i], w = vq[i];
            vp[i] = fmar(c, u, -s * w);
            vq[i] = fmar(s, u, c * w);
          }
        }
      }
      __syncthreads();
    }
    // every CTA reads every owner's flag: the same decision everywhere
    int any = 0;
    for (int k = 0; k < ncl; ++k) any |= *cl.map_shared_rank(&s_rotated, k);
    cl.sync();  // all flags read before any is reset
    if (tid == 0) s_rotated = 0;
    if (!any) break;
  }

  if (!kFinal) {
    if (rank == 0 && tid == 0 && a.info) a.info[0] = (unsigned)sweep;
    for (int e = tid; e < b * nr; e += nth) {
      const int j = e / nr, i = e % nr;
      a.V32[(r0 + i) + (int64_t)j * b] = (float)Vl[(size_t)j * LDR + i];
    }
    return;  // no CTA reads another's shared memory after the last cluster barrier
  }

  // column norms and the signed entry of largest |V| per column (own rows)
  for (int j = tid; j < P; j += nth) {
    double s2 = 0.0, bestabs = -1.0;
    int bi = 0;
    for (int i = 0; i < nr; ++i) {
      const double x = (double)Bl[(size_t)j * LDR + i];
      s2 = fma(x, x, s2);
      const double av = fabs((double)Vl[(size_t)j * LDR + i]);
      if (av > bestabs) {  // strict: lowest row wins ties
        bestabs = av;
        bi = i;
      }
    }
    npart[j] = s2;
    vmax[j] = (nr > 0) ? (double)Vl[(size_t)j * LDR + bi] : 0.0;
    vrow[j] = r0 + bi;
  }
  cl.sync();
  for (int j = tid; j < P; j += nth) {
    // The running maximum keeps its magnitude and its owner explicitly; the
    // signed value is fetched from the owning CTA once the winner is known.
    double s2 = 0.0, bestabs = -1.0;
    int bestk = 0;
    for (int k = 0; k < ncl; ++k) {
      s2 += cl.map_shared_rank(npart, k)[j];
      const double av = fabs(cl.map_shared_rank(vmax, k)[j]);
      if (av > bestabs) {  // strict: lower rows (CTAs) win ties
        bestabs = av;
        bestk = k;
      }
    }
    Dfull[j] = (j < b) ? sqrt(s2) : -1.0;
    vbest[j] = cl.map_shared_rank(vmax, bestk)[j];
  }
  cl.sync();  // every CTA has finished reading the others' vmax/npart
  for (int j = tid; j < b; j += nth) {
    const double dj = Dfull[j];
    int rk = 0;
    for (int l = 0; l < b; ++l) {
      const double dl = Dfull[l];
      rk += (dl > dj) || (dl == dj && l < j);
    }
    rankof[j] = rk;
  }
  __syncthreads();
  // write outputs: column j goes to position rankof[j]
  for (int e = tid; e < b * nr; e += nth) {
    const int j = e / nr, i = e % nr;
    const int pos = rankof[j];
    const double sg = (vbest[j] < 0.0) ? -1.0 : 1.0;
    const double dj = Dfull[j];
    const int64_t gi = r0 + i;
    a.Vs[gi + (int64_t)pos * b] = sg * (double)Vl[(size_t)j * LDR + i];
    a.Us[gi + (int64_t)pos * b] = (dj > 0.0) ? sg * ((double)Bl[(size_t)j * LDR + i] / dj) : 0.0;
  }
  if (rank == 0) {
    for (int j = tid; j < b; j += nth) a.D[rankof[j]] = Dfull[j];
    if (tid == 0 && a.info) a.info[0] = (unsigned)sweep;
  }
}

// ---- Phase 1 by blocks ---------------------------------------------------
// One-sided block Jacobi (the block-cyclic orderings of one-sided Jacobi,
// e.g. Hari & Vesely; each block pair gets one inner sweep): the columns,
// padded with zero columns, form nblk = 2 C blocks of w.  In each of the
// nblk - 1 rounds of an outer sweep (circle ordering of the blocks) CTA k of
// the cluster takes one pair of blocks, loads their 2w columns of B and V
// (every row) from the work arrays into shared memory, runs one inner sweep
// of one-sided Jacobi over them (2w - 1 rounds of w disjoint column pairs,
// one warp per pair, one block barrier per round) and writes them back; a
// cluster barrier (release / acquire) separates the outer rounds.  An outer
// sweep visits every pair of columns in different blocks once, so a round of
// the cluster does w times the work of one scalar round for one cluster
// barrier instead of two.
struct BlkArgs {
  int b, w, nblk;   // columns, block width, blocks (twice the cluster size)
  const double* B;  // input block (FP64), column-major
  int64_t ldb;
  float* Bw;        // work arrays: b rows x nblk w columns, ld b
  float* Vw;
  float* V32;       // output: V (b x b, ld b)
  int max_sweeps;
  float tol;        // rotate while |a_p.a_q| > tol |a_p| |a_q|
  unsigned* info;   // outer sweeps taken
};

size_t blk_smem_bytes(int b, int w) { return (size_t)4 * w * b * sizeof(float); }
constexpr int kRowsPerLane = SVD_MAX_B / 32;  // rows of a column per lane (b <= 256)
constexpr int kLd = 8;                        // loads in flight per thread

// Rotation of phase 1 (Rutishauser's formula) with the hardware's
// approximate divide and reciprocal square root: phase 1 only preconditions
// (its V is made orthogonal in FP64 afterwards and phase 2 restarts from
// C = B V), so a rotation orthogonal to a few FP32 ulp is enough, and the
// rotation is on the critical path of every inner round.  zeta^2 overflows
// only where t is below FP32 resolution, and then t = 0.
__device__ __forceinline__ void blk_rotation(float al, float be, float ga, float* c, float* s) {
  const float zeta = __fdividef(be - al, 2.f * ga);
  const float t = __fdividef(copysignf(1.f, zeta), fabsf(zeta) + __fsqrt_rn(fmaf(zeta, zeta, 1.f)));
  *c = rsqrtf(fmaf(t, t, 1.f));
  *s = *c * t;
}

__global__ void __launch_bounds__(SVD_MAX_THREADS) block_jacobi_f32_kernel(const BlkArgs a) {
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank(), ncl = (int)cl.num_blocks();
  const int b = a.b, w = a.w, nblk = a.nblk, ncol = nblk * w;
  const int tid = threadIdx.x, nth = blockDim.x, warp = tid >> 5, lane = tid & 31;
  extern __shared__ float fsm[];
  float* Bs = fsm;                      // local column l (0..2w-1), row i at Bs[l b + i]
  float* Vs = Bs + (size_t)2 * w * b;
  __shared__ int s_rot;
  __shared__ double s_red[SVD_MAX_THREADS / 32];

  // B 2^-e, e the exponent of max |B| (exact, inside the FP32 range)
  double mx = 0.0;
  for (int e = tid; e < b * b; e += nth)
    mx = fmax(mx, fabs(a.B[(e % b) + (int64_t)(e / b) * a.ldb]));
  mx = block_max(mx, s_red);
  double scale = 1.0;
  if (mx > 0.0) {
    int ex = 0;
    frexp(mx, &ex);
    scale = ldexp(1.0, -ex);
  }
  // this CTA's share of the work arrays: columns rank, rank + C, ...
  for (int j = rank; j < ncol; j += ncl)
    for (int i = tid; i < b; i += nth) {
      a.Bw[i + (int64_t)j * b] = (j < b) ? (float)(a.B[i + (int64_t)j * a.ldb] * scale) : 0.f;
      a.Vw[i + (int64_t)j * b] = (i == j) ? 1.f : 0.f;
    }
  if (tid == 0) s_rot = 0;
  cl.sync();

  const float tol = a.tol;
  int sweep = 0;
  for (; sweep < a.max_sweeps; ++sweep) {
    for (int round = 0; round < nblk - 1; ++round) {
      int bp, bq;
      rr_pair(round, rank, nblk, &bp, &bq);
      // the two blocks are contiguous in the work arrays (ld b): batches of
      // kLd loads in flight per thread before they are stored
      for (int e0 = 0; e0 < 2 * w * b; e0 += kLd * nth) {
        float xb[kLd], xv[kLd];
#pragma unroll
        for (int k = 0; k < kLd; ++k) {
          const int e = e0 + k * nth + tid;
          if (e < 2 * w * b) {
            const int64_t g = (e < w * b) ? (int64_t)bp * w * b + e : (int64_t)bq * w * b + (e - w * b);
            xb[k] = __ldcg(a.Bw + g);
            xv[k] = __ldcg(a.Vw + g);
          }
        }
#pragma unroll
        for (int k = 0; k < kLd; ++k) {
          const int e = e0 + k * nth + tid;
          if (e < 2 * w * b) {
            Bs[e] = xb[k];
            Vs[e] = xv[k];
          }
        }
      }
      __syncthreads();
      for (int ir = 0; ir < 2 * w - 1; ++ir) {
        if (warp < w) {
          int p, q;
          rr_pair(ir, warp, 2 * w, &p, &q);
          float* bpc = Bs + (size_t)p * b;
          float* bqc = Bs + (size_t)q * b;
          float sa = 0.f, sb = 0.f, sc = 0.f;
#pragma unroll
          for (int k = 0; k < kRowsPerLane; ++k) {
            const int i = lane + 32 * k;
            if (i < b) {
              const float x = bpc[i], y = bqc[i];
              sa = fmaf(x, x, sa);
              sb = fmaf(y, y, sb);
              sc = fmaf(x, y, sc);
            }
          }
          for (int o = 16; o > 0; o >>= 1) {  // xor tree: the same sums in every lane
            sa += __shfl_xor_sync(0xffffffffu, sa, o);
            sb += __shfl_xor_sync(0xffffffffu, sb, o);
            sc += __shfl_xor_sync(0xffffffffu, sc, o);
          }
          if (sc != 0.f && sc * sc > tol * tol * sa * sb) {
            float c, s;
            blk_rotation(sa, sb, sc, &c, &s);
            if (lane == 0) s_rot = 1;
            float* vpc = Vs + (size_t)p * b;
            float* vqc = Vs + (size_t)q * b;
            // every load before any store: the four columns' rows would
            // otherwise be read one row at a time behind possibly aliasing stores
            float x[kRowsPerLane], y[kRowsPerLane], u[kRowsPerLane], v[kRowsPerLane];
#pragma unroll
            for (int k = 0; k < kRowsPerLane; ++k) {
              const int i = lane + 32 * k;
              if (i < b) {
                x[k] = bpc[i];
                y[k] = bqc[i];
                u[k] = vpc[i];
                v[k] = vqc[i];
              }
            }
#pragma unroll
            for (int k = 0; k < kRowsPerLane; ++k) {
              const int i = lane + 32 * k;
              if (i < b) {
                bpc[i] = fmaf(c, x[k], -s * y[k]);
                bqc[i] = fmaf(s, x[k], c * y[k]);
                vpc[i] = fmaf(c, u[k], -s * v[k]);
                vqc[i] = fmaf(s, u[k], c * v[k]);
              }
            }
          }
        }
        __syncthreads();
      }
      for (int e = tid; e < 2 * w * b; e += nth) {
        const int l = e / b, i = e % b;
        const int64_t gc = (l < w) ? (int64_t)bp * w + l : (int64_t)bq * w + (l - w);
        a.Bw[i + gc * b] = Bs[e];
        a.Vw[i + gc * b] = Vs[e];
      }
      cl.sync();  // the next round reads what this one wrote
    }
    // every CTA reads every flag: the same decision everywhere
    int any = 0;
    for (int k = 0; k < ncl; ++k) any |= *cl.map_shared_rank(&s_rot, k);
    cl.sync();  // all flags read before any is reset
    if (tid == 0) s_rot = 0;
    if (!any) break;
  }
  if (rank == 0 && tid == 0 && a.info) a.info[0] = (unsigned)sweep;
  for (int j = rank; j < b; j += ncl)
    for (int i = tid; i < b; i += nth) a.V32[i + (int64_t)j * b] = __ldcg(a.Vw + i + (int64_t)j * b);
}

// Completes the columns of Us whose singular value is exactly zero: modified
// Gram-Schmidt (twice) of unit vectors e_0, e_1, ... against the columns
// already present, taking the first with a residual norm above 1/2.
__global__ void complete_basis_kernel(int b, const double* __restrict__ D, double* Us) {
  __shared__ double red[SVD_THREADS / 32];
  __shared__ double u[SVD_MAX_B];
  int nz = 0;
  for (int j = 0; j < b; ++j) nz += (D[j] > 0.0);
  if (nz == b) return;
  int cand = 0;
  for (int j = nz; j < b; ++j) {
    for (; cand < b; ++cand) {
      for (int i = threadIdx.x; i < b; i += blockDim.x) u[i] = (i == cand) ? 1.0 : 0.0;
      __syncthreads();
      for (int pass = 0; pass < 2; ++pass) {
        for (int l = 0; l < j; ++l) {
          double d = 0.0;
          for (int i = threadIdx.x; i < b; i += blockDim.x) d = fma(Us[i + (int64_t)l * b], u[i], d);
          d = block_sum(d, red);
          for (int i = threadIdx.x; i < b; i += blockDim.x) u[i] = fma(-d, Us[i + (int64_t)l * b], u[i]);
          __syncthreads();
        }
      }
      double nn = 0.0;
      for (int i = threadIdx.x; i < b; i += blockDim.x) nn = fma(u[i], u[i], nn);
      nn = sqrt(block_sum(nn, red));
      if (nn > 0.5) {
        for (int i = threadIdx.x; i < b; i += blockDim.x) Us[i + (int64_t)j * b] = u[i] / nn;
        __syncthreads();
        ++cand;
        break;
      }
    }
  }
}

// V <- (double) V32 and H <- I (both b x b, ld b)
__global__ void svd_prep_kernel(int b, const float* __restrict__ V32, double* __restrict__ V,
                                double* __restrict__ H) {
  const int64_t total = (int64_t)b * b;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (V32) V[e] = (double)V32[e];
    H[e] = (e % b == e / b) ? 1.0 : 0.0;
  }
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

template <typename Real, bool kFinal>
int configure(int b, int ncl, size_t* smem_out) {
  RUTV_TRY(ensure_nonportable_cluster((const void*)jacobi_kernel<Real, kFinal>));
  const size_t smem = jac_smem_bytes<Real>(b, ncl);
  RUTV_TRY(ensure_smem((const void*)jacobi_kernel<Real, kFinal>, smem));
  *smem_out = smem;
  return 0;
}

template <typename Real, bool kFinal>
int launch_jacobi(const JacArgs& a, int ncl, cudaStream_t st) {
  size_t smem = 0;
  RUTV_TRY((configure<Real, kFinal>(a.b, ncl, &smem)));
  ProfScope prof(kFinal ? K_SVD : K_SVD32, 0.0, 2.0 * sizeof(Real) * (double)a.b * a.b, st);
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)ncl;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3((unsigned)ncl);
  cfg.blockDim = dim3(kFinal ? SVD_THREADS : SVD_THREADS_FP32);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  RUTV_CK(cudaLaunchKernelEx(&cfg, jacobi_kernel<Real, kFinal>, a));
  note_launch();
  RUTV_CK(cudaGetLastError());
  return 0;
}

// Cluster size of the FP64 phase: 16 CTAs (a non-portable size) where the
// device can place them, else the portable 8.
int fp64_cluster() {
  static int ncl = 0;
  if (ncl) return ncl;
  size_t smem = 0;
  if (configure<double, true>(SVD_MAX_B, 16, &smem) != 0) return 8;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 16;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(16);
  cfg.blockDim = dim3(SVD_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int nclusters = 0;
  if (cudaOccupancyMaxActiveClusters(&nclusters, (void*)jacobi_kernel<double, true>, &cfg) ==
          cudaSuccess &&
      nclusters > 0)
    ncl = 16;
  else
    ncl = 8;
  cudaGetLastError();
  return ncl;
}

// Phase 1 by blocks on a cluster of fp64_cluster() CTAs (16 where the device
// places them): blocks of w = ceil(b / 2C) columns; the work arrays hold
// b x 2C w floats each.
int launch_block_jacobi(BlkArgs a, cudaStream_t st) {
  const int ncl = fp64_cluster();
  a.nblk = 2 * ncl;
  a.w = (a.b + a.nblk - 1) / a.nblk;
  const size_t smem = blk_smem_bytes(a.b, a.w);
  RUTV_TRY(ensure_nonportable_cluster((const void*)block_jacobi_f32_kernel));
  RUTV_TRY(ensure_smem((const void*)block_jacobi_f32_kernel, smem));
  ProfScope prof(K_SVD32, 0.0, 8.0 * (double)a.b * a.b, st);
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)ncl;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3((unsigned)ncl);
  cfg.blockDim = dim3((unsigned)(32 * (a.w > 4 ? a.w : 4)));
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  RUTV_CK(cudaLaunchKernelEx(&cfg, block_jacobi_f32_kernel, a));
  note_launch();
  RUTV_CK(cudaGetLastError());
  return 0;
}
}  // namespace

size_t small_svd_scratch_bytes(int b) {
  return align256((size_t)b * b * sizeof(float)) + 2 * align256((size_t)b * b * sizeof(double));
}

int launch_small_svd(int b, const double* B, int64_t ldb, double* D, double* Us, double* Vs,
                     unsigned* info, void* scratch, double* gemm_scratch, size_t gemm_bytes,
                     cudaStream_t st) {
  if (b < 1 || b > SVD_MAX_B) return RANDUTV_EUNSUPPORTED;
  JacArgs a = {};
  a.b = b;
  a.D = D;
  a.Us = Us;
  a.Vs = Vs;
  a.info = info;
  a.max_sweeps = 40;
  a.tol = (double)b * 0x1.0p-53;
  if (b <= SVD_DIRECT_B) {
    a.B = B;
    a.ldb = ldb;
    a.Vin = nullptr;
    RUTV_TRY((launch_jacobi<double, true>(a, fp64_cluster(), st)));
  } else {
    char* s = (char*)scratch;
    float* V32 = (float*)s;
    double* H = (double*)(s + align256((size_t)b * b * sizeof(float)));
    double* Vb = (double*)((char*)H + align256((size_t)b * b * sizeof(double)));
    // phase 1: FP32 block sweeps down to the FP32 noise level; the work arrays
    // borrow H and Vb (2 b^2 floats each, unused until phase 1 is done)
    BlkArgs a1 = {};
    a1.b = b;
    a1.B = B;
    a1.ldb = ldb;
    a1.Bw = (float*)H;
    a1.Vw = (float*)Vb;
    a1.V32 = V32;
    a1.max_sweeps = 20;
    a1.tol = (float)(2.0 * (double)b * 0x1.0p-24);
    a1.info = info ? info + 1 : nullptr;
    RUTV_TRY(launch_block_jacobi(a1, st));
    // two Newton-Schulz steps: V <- V H, H = 1.5 I - 0.5 V^T V (FP64)
    const int grid = (b * b + 255) / 256;
    svd_prep_kernel<<<grid, 256, 0, st>>>(b, V32, Vs, H);
    note_launch();
    RUTV_CK(cudaGetLastError());
    RUTV_TRY(launch_dgemm(true, false, b, b, b, -0.5, Vs, b, Vs, b, 1.5, H, b, gemm_scratch,
                          gemm_bytes, st));
    RUTV_TRY(launch_dgemm(false, false, b, b, b, 1.0, Vs, b, H, b, 0.0, Vb, b, gemm_scratch,
                          gemm_bytes, st));
    svd_prep_kernel<<<grid, 256, 0, st>>>(b, nullptr, nullptr, H);
    note_launch();
    RUTV_CK(cudaGetLastError());
    RUTV_TRY(launch_dgemm(true, false, b, b, b, -0.5, Vb, b, Vb, b, 1.5, H, b, gemm_scratch,
                          gemm_bytes, st));
    RUTV_TRY(launch_dgemm(false, false, b, b, b, 1.0, Vb, b, H, b, 0.0, Vs, b, gemm_scratch,
                          gemm_bytes, st));
    // C = B V into Us; phase 2 reads C and V from Us and Vs and writes its
    // outputs over them (every CTA reads and writes only its own rows)
    RUTV_TRY(launch_dgemm(false, false, b, b, b, 1.0, B, ldb, Vs, b, 0.0, Us, b, gemm_scratch,
                          gemm_bytes, st));
    a.B = Us;
    a.ldb = b;
    a.Vin = Vs;
    RUTV_TRY((launch_jacobi<double, true>(a, fp64_cluster(), st)));
  }
  complete_basis_kernel<<<1, SVD_THREADS, 0, st>>>(b, D, Us);
  note_launch();
  RUTV_CK(cudaGetLastError());
  return 0;
}

}  // namespace rutv
