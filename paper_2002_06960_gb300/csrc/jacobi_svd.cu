// SVD of the b x b diagonal block (Fig. 2: [A11, U_SVD, V_SVD] := SVD(A11);
// §3.1 step 3), one-sided Jacobi in FP64 (Hestenes 1958; Demmel & Veselic
// 1992 for the rotation and the stopping rule).
//
// Layout: one thread-block cluster of C CTAs (16 where the device can place
// that non-portable size, else 8).  CTA k holds rows [k R, (k+1) R) of both
// the working matrix B (which converges to U diag(D)) and the accumulated
// rotation V, R = ceil(b/C), in shared memory.  A sweep is b-1 rounds of the
// round-robin (circle) ordering, each round rotating b/2 disjoint column
// pairs.  Per round every CTA writes the partial inner products
// (|a_p|^2, |a_q|^2, a_p.a_q) of its rows, a cluster barrier follows, and
// every CTA combines the C partials of each pair in a fixed order through
// distributed shared memory.  The rotation parameters are therefore bitwise
// identical in all CTAs, which apply them to their own rows, and all CTAs
// take the same convergence decision.  FP64 throughput per SM is low on this
// part (two DFMA per clock), which is why the rows are spread over C SMs.
//
// After convergence: D_j = |b_j|, columns sorted by descending D (lowest
// index first on ties), U_j = b_j / D_j, and each column of V signed so that
// its entry of largest magnitude (lowest row on ties) is positive, U_j with
// it.  Exactly-zero singular values get their U columns from a separate
// completion kernel (Gram-Schmidt of unit vectors).
#include <cooperative_groups.h>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace rutv {

namespace {
constexpr int SVD_CL = 8;
constexpr int SVD_THREADS = 256;
constexpr int SVD_MAX_B = 256;

struct SvdSmem {
  int b, P, npairs, R, LDR;
  size_t bytes() const {
    size_t d = 2 * (size_t)P * LDR          // Bl, Vl
               + 2 * (size_t)npairs * 3     // partials, double buffered
               + (size_t)P                  // column norms (partial)
               + (size_t)P                  // max |V| per column, signed (partial)
               + (size_t)P                  // max |V| per column, signed (cluster)
               + (size_t)P;                 // D (full)
    return d * sizeof(double) + (size_t)P * sizeof(int) * 2 + 64;
  }
};

__device__ __forceinline__ void rr_pair(int round, int t, int P, int* p, int* q) {
  int a, c;
  if (t == 0) {
    a = P - 1;
    c = round;
  } else {
    a = (round + t) % (P - 1);
    c = (round - t + (P - 1)) % (P - 1);
  }
  *p = a < c ? a : c;
  *q = a < c ? c : a;
}

__global__ void __launch_bounds__(SVD_THREADS)
jacobi_svd_kernel(int b, const double* __restrict__ Bg, int64_t ldb, double* __restrict__ D,
                  double* __restrict__ Us, double* __restrict__ Vs, int max_sweeps,
                  unsigned* __restrict__ info) {
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  SvdSmem L;
  L.b = b;
  L.P = (b + 1) & ~1;
  L.npairs = L.P / 2;
  const int ncl = (int)cl.num_blocks();  // 16 where the device allows it, else 8
  L.R = (b + ncl - 1) / ncl;
  L.LDR = L.R + 1;
  const int P = L.P, npairs = L.npairs, R = L.R, LDR = L.LDR;
  const int r0 = rank * R;
  const int nr = max(0, min(b, r0 + R) - r0);

  extern __shared__ double smem[];
  double* Bl = smem;                       // column j, local row i at Bl[j*LDR + i]
  double* Vl = Bl + (size_t)P * LDR;
  double* part = Vl + (size_t)P * LDR;     // [2][npairs][3]
  double* npart = part + 2 * npairs * 3;   // [P]
  double* vmax = npart + P;                // [P]
  double* vbest = vmax + P;                // [P]
  double* Dfull = vbest + P;               // [P]
  int* vrow = (int*)(Dfull + P);           // [P]
  int* rankof = vrow + P;                  // [P]
  __shared__ int s_rotated;

  // load own rows of B, V = I (padding column b, if any, is zero)
  for (int e = threadIdx.x; e < P * LDR; e += SVD_THREADS) {
    const int j = e / LDR, i = e % LDR;
    const int gi = r0 + i;
    double bv = 0.0, vv = 0.0;
    if (i < nr && j < b) {
      bv = Bg[gi + (int64_t)j * ldb];
      vv = (gi == j) ? 1.0 : 0.0;
    }
    Bl[e] = bv;
    Vl[e] = vv;
  }
  if (threadIdx.x == 0) s_rotated = 0;
  __syncthreads();

  int tpp = 1;
  while (tpp < 32 && tpp * 2 * npairs <= SVD_THREADS) tpp *= 2;
  const int g = threadIdx.x / tpp, sub = threadIdx.x % tpp;
  const bool active = g < npairs;
  const double tol = (double)(b > 1 ? b : 1) * 0x1.0p-53;

  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    for (int round = 0; round < P - 1; ++round) {
      // Parity of the running round count (a sweep has an odd number of
      // rounds, so the round index alone would reuse a buffer back to back).
      const int buf = (int)(((unsigned)sweep * (unsigned)(P - 1) + (unsigned)round) & 1u);
      int p = 0, q = 0;
      if (active) rr_pair(round, g, P, &p, &q);
      // partial inner products over own rows
      double sa = 0.0, sb = 0.0, sc = 0.0;
      if (active) {
        const double* bp = Bl + (size_t)p * LDR;
        const double* bq = Bl + (size_t)q * LDR;
        for (int i = sub; i < nr; i += tpp) {
          const double x = bp[i], y = bq[i];
          sa = fma(x, x, sa);
          sb = fma(y, y, sb);
          sc = fma(x, y, sc);
        }
      }
      for (int o = tpp >> 1; o > 0; o >>= 1) {
        sa += __shfl_xor_sync(0xffffffffu, sa, o);
        sb += __shfl_xor_sync(0xffffffffu, sb, o);
        sc += __shfl_xor_sync(0xffffffffu, sc, o);
      }
      if (active && sub == 0) {
        double* pp = part + ((size_t)buf * npairs + g) * 3;
        pp[0] = sa; pp[1] = sb; pp[2] = sc;
      }
      cl.sync();
      // cluster sums in CTA order, rotation parameters
      // The threads of the group load the 8 CTAs' partials in parallel and
      // combine them with a fixed shuffle tree: every thread (of every CTA)
      // ends with the same sums and takes the same rotation.
      double c = 1.0, s = 0.0;
      int rot = 0;
      {
        double al = 0.0, be = 0.0, ga = 0.0;
        if (active) {
          for (int k = sub; k < ncl; k += tpp) {
            const double* rp = cl.map_shared_rank(part, k) + ((size_t)buf * npairs + g) * 3;
            al += rp[0];
            be += rp[1];
            ga += rp[2];
          }
        }
        for (int o = tpp >> 1; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          ga += __shfl_xor_sync(0xffffffffu, ga, o);
        }
        if (active && q < b && ga != 0.0 && fabs(ga) > tol * sqrt(al) * sqrt(be)) {
          const double zeta = (be - al) / (2.0 * ga);
          const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + hypot(1.0, zeta));
          c = 1.0 / sqrt(fma(t, t, 1.0));
          s = c * t;
          rot = 1;
        }
      }
      if (active && rot) {
        if (sub == 0) s_rotated = 1;
        double* bp = Bl + (size_t)p * LDR;
        double* bq = Bl + (size_t)q * LDR;
        for (int i = sub; i < nr; i += tpp) {
          const double x = bp[i], y = bq[i];
          bp[i] = fma(c, x, -s * y);
          bq[i] = fma(s, x, c * y);
        }
        double* vp = Vl + (size_t)p * LDR;
        double* vq = Vl + (size_t)q * LDR;
        for (int i = sub; i < nr; i += tpp) {
          const double x = vp[i], y = vq[i];
          vp[i] = fma(c, x, -s * y);
          vq[i] = fma(s, x, c * y);
        }
      }
      __syncthreads();
    }
    const int any = s_rotated;
    __syncthreads();
    if (threadIdx.x == 0) s_rotated = 0;
    __syncthreads();
    if (!any) break;
  }

  // column norms and the signed entry of largest |V| per column (own rows)
  for (int j = threadIdx.x; j < P; j += SVD_THREADS) {
    double s2 = 0.0, bestabs = -1.0;
    int bi = 0;
    for (int i = 0; i < nr; ++i) {
      const double x = Bl[(size_t)j * LDR + i];
      s2 = fma(x, x, s2);
      const double a = fabs(Vl[(size_t)j * LDR + i]);
      if (a > bestabs) {  // strict: lowest row wins ties
        bestabs = a;
        bi = i;
      }
    }
    npart[j] = s2;
    vmax[j] = (nr > 0) ? Vl[(size_t)j * LDR + bi] : 0.0;
    vrow[j] = r0 + bi;
  }
  cl.sync();
  for (int j = threadIdx.x; j < P; j += SVD_THREADS) {
    // The running maximum keeps its magnitude and its owner explicitly; the
    // signed value is fetched from the owning CTA once the winner is known.
    double s2 = 0.0, bestabs = -1.0;
    int bestk = 0;
    for (int k = 0; k < ncl; ++k) {
      s2 += cl.map_shared_rank(npart, k)[j];
      const double a = fabs(cl.map_shared_rank(vmax, k)[j]);
      if (a > bestabs) {  // strict: lower rows (CTAs) win ties
        bestabs = a;
        bestk = k;
      }
    }
    Dfull[j] = (j < b) ? sqrt(s2) : -1.0;
    vbest[j] = cl.map_shared_rank(vmax, bestk)[j];
  }
  cl.sync();  // every CTA has finished reading the others' vmax/npart
  for (int j = threadIdx.x; j < b; j += SVD_THREADS) {
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
  for (int e = threadIdx.x; e < b * nr; e += SVD_THREADS) {
    const int j = e / nr, i = e % nr;
    const int pos = rankof[j];
    const double sg = (vbest[j] < 0.0) ? -1.0 : 1.0;
    const double dj = Dfull[j];
    const int64_t gi = r0 + i;
    Vs[gi + (int64_t)pos * b] = sg * Vl[(size_t)j * LDR + i];
    Us[gi + (int64_t)pos * b] = (dj > 0.0) ? sg * (Bl[(size_t)j * LDR + i] / dj) : 0.0;
  }
  if (rank == 0) {
    for (int j = threadIdx.x; j < b; j += SVD_THREADS) D[rankof[j]] = Dfull[j];
    if (threadIdx.x == 0 && info) info[0] = (unsigned)sweep;
  }
  cl.sync();  // keep shared memory alive until no CTA reads it remotely
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
}  // namespace

int launch_small_svd(int b, const double* B, int64_t ldb, double* D, double* Us, double* Vs,
                     unsigned* info, cudaStream_t st) {
  if (b < 1 || b > SVD_MAX_B) return RANDUTV_EUNSUPPORTED;
  SvdSmem L;
  L.b = b;
  L.P = (b + 1) & ~1;
  L.npairs = L.P / 2;
  // A cluster of 16 CTAs (a non-portable size) halves each CTA's FP64 work
  // per round; fall back to the portable 8 where the device cannot place 16.
  static int ncl = 0;
  static size_t configured = 0;
  if (ncl == 0) {
    RUTV_CK(cudaFuncSetAttribute(jacobi_svd_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed,
                                 1));
    RUTV_CK(cudaFuncSetAttribute(jacobi_svd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 160 * 1024));
    configured = 160 * 1024;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 16;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(16);
    cfg.blockDim = dim3(SVD_THREADS);
    cfg.dynamicSmemBytes = 100 * 1024;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, (void*)jacobi_svd_kernel, &cfg) == cudaSuccess &&
        nclusters > 0)
      ncl = 16;
    else
      ncl = SVD_CL;
    cudaGetLastError();
  }
  L.R = (b + ncl - 1) / ncl;
  L.LDR = L.R + 1;
  const size_t smem = L.bytes();
  if (smem > configured) {
    RUTV_CK(cudaFuncSetAttribute(jacobi_svd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
    configured = smem;
  }
  ProfScope prof(K_SVD, 0.0, 32.0 * (double)b * b, st);
  const int max_sweeps = 40;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)ncl;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3((unsigned)ncl);
  cfg.blockDim = dim3(SVD_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  RUTV_CK(cudaLaunchKernelEx(&cfg, jacobi_svd_kernel, b, B, ldb, D, Us, Vs, max_sweeps, info));
  note_launch();
  RUTV_CK(cudaGetLastError());
  complete_basis_kernel<<<1, SVD_THREADS, 0, st>>>(b, D, Us);
  note_launch();
  RUTV_CK(cudaGetLastError());
  return 0;
}

}  // namespace rutv
