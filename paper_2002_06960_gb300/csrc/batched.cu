// Batched randUTV: many FP32 matrices of uneven sizes in one persistent launch.
//
// Every CTA repeatedly takes the next matrix from a device work queue (the
// host orders it by descending cost) and runs the whole blocked loop of §3.1
// / Fig. 2 on it: the sketch and power products, the two Householder panel
// QRs with their compact-WY updates of T, U and V, and the small SVD with its
// fold-back.  The matrices here are at most 1024 x 1024, so one SM owns one
// matrix and everything runs as CTA-level tiles: FP32 storage and FFMA
// products, Householder norms and scalars in FP64, and a one-sided Jacobi
// SVD (FP32) of the b x b block in shared memory.  The queue is a single
// atomic counter; no CTA ever waits on another, so the launch can be
// captured in a CUDA graph and replayed.
//
// The sketch uses the same Philox4x32-10 words as the other paths (counter
// (pair, step, matrix id, 0)), turned into normals by a single-precision
// Box-Muller: u1 = ((x0 >> 8) + 1) 2^-24, u2 = (x2 >> 8) 2^-24,
// sqrt(-2 ln u1) (cos, sin)(2 pi u2).
#include "common.cuh"
#include "philox.cuh"

namespace rutv {

namespace {

constexpr int BT = 256;          // threads per CTA
constexpr int BMAX = 64;         // largest block size of the batched path
constexpr int GK = 32;           // depth of one CTA GEMM stage
constexpr int GSTAGES = 3;       // CTA GEMM pipeline depth
constexpr int GBUF = GSTAGES * GK * (129 + 33);  // floats of the GEMM operand buffers
constexpr int GCBUF = GSTAGES * 4096;            // floats of the GEMM C-tile buffers
// Below S (which sits at the top of the shared union): room to stage W for
// the WY factor
constexpr int WY_SMEM_FLOATS = GBUF + GCBUF - 2 * BMAX * (BMAX + 1);
constexpr int NWARP = BT / 32;

struct BatchDesc {
  int64_t m, n, lda;
  const float* A;
  float* T;
  float* U;
  float* V;
  int b, q;
  int matrix_id, pad;
};

struct BatchArgs {
  const BatchDesc* desc;
  const int* order;
  int count;
  int* next;
  int* info;
  uint64_t seed;
  float* work;
  int64_t work_stride;
  int64_t mmax;
};

struct Smem {
  // The GEMM tiles and the WY / SVD arrays are never live at the same time.
  union {
    struct {
      float gbuf[GBUF];   // GEMM operands, k-major: A [GSTAGES][GK][TM+1], then B [GSTAGES][GK][TN+1]
      float gcbuf[GCBUF]; // C tiles for beta != 0: [GSTAGES][TN][TM]
    };
    struct {
      float svB[BMAX][BMAX + 1];  // column j at svB[j][i]
      float svV[BMAX][BMAX + 1];
      float svpad[WY_SMEM_FLOATS - 2 * BMAX * (BMAX + 1)];
      double S[BMAX][BMAX + 1];   // S(i, j) at S[j][i], FP64
    };
  };
  double tau[BMAX];
  float wv[BMAX];
  float qscale[BMAX];  // panel QR: 1 / (alpha - beta) of each reflector
  float qbeta[BMAX];   // panel QR: R(j, j)
  float D[BMAX];
  float vbest[BMAX];
  int rankof[BMAX];
  double red[NWARP];
  double coef[4];
  int flag;
};

// ------------------------------------------------------------ CTA GEMM
// 4-byte asynchronous copy global -> shared (zero fill when !valid), and the
// group commit / wait of the copies a thread has issued.
__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const int n = valid ? 4 : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// C = alpha op(A) op(B) + beta C (FP32, column-major); C must not alias A, B.
// TM x TN output tiles (TM TN = 4096), 4 x 4 per thread: rows tx + (TM/4) i,
// columns ty + (TN/4) j.  K goes in stages of GK, and the stages of all tiles
// form one pipeline through GSTAGES shared-memory buffers filled by
// asynchronous copies: stage s is multiplied while stages s + 1 and s + 2
// (of this tile or the next ones) are in flight, and with beta != 0 the copy
// of a tile's C travels with its last stage.  Every output is one FMA chain over k = 0 .. K-1 in
// order, whatever the tile shape, so the result does not depend on it.
template <bool TA, bool TB, int TM, int TN>
__device__ void cta_gemm_t(int M, int N, int K, float alpha, const float* __restrict__ A,
                           int64_t lda, const float* __restrict__ B, int64_t ldb, float beta,
                           float* C, int64_t ldc, Smem& sm) {
  static_assert(TM * TN == 16 * BT, "4 x 4 outputs per thread");
  constexpr int RX = TM / 4, RY = TN / 4;
  constexpr int PA = TM * GK / BT, PB = TN * GK / BT;  // elements per thread per stage
  static_assert(GSTAGES * GK * (TM + 1) + GSTAGES * GK * (TN + 1) <= GBUF, "tile buffers fit");
  float(*gA)[GK][TM + 1] = reinterpret_cast<float(*)[GK][TM + 1]>(sm.gbuf);
  float(*gB)[GK][TN + 1] =
      reinterpret_cast<float(*)[GK][TN + 1]>(sm.gbuf + GSTAGES * GK * (TM + 1));
  const int tid = threadIdx.x, tx = tid % RX, ty = tid / RX;
  const int tiles_m = (M + TM - 1) / TM, tiles_n = (N + TN - 1) / TN, nk = (K + GK - 1) / GK;
  const int total = tiles_m * tiles_n * nk;
  // element e = tid + BT t of a tile; the fast index follows the contiguous
  // direction of the source, so the global reads coalesce
  auto issue = [&](int s) {
    if (s < total) {
      const int buf = s % GSTAGES;
      const int tile = s / nk, k0 = (s - tile * nk) * GK;
      const int m0 = (tile % tiles_m) * TM, n0 = (tile / tiles_m) * TN;
#pragma unroll
      for (int t = 0; t < PA; ++t) {
        const int e = tid + BT * t;
        int mm, kk;
        if (!TA) { mm = e % TM; kk = e / TM; } else { kk = e % GK; mm = e / GK; }
        const int gm = m0 + mm, gk = k0 + kk;
        const bool v = gm < M && gk < K;
        cp_async4(&gA[buf][kk][mm], v ? (TA ? A + gk + (int64_t)gm * lda : A + gm + (int64_t)gk * lda) : A, v);
      }
#pragma unroll
      for (int t = 0; t < PB; ++t) {
        const int e = tid + BT * t;
        int nn, kb;
        if (!TB) { kb = e % GK; nn = e / GK; } else { nn = e % TN; kb = e / TN; }
        const int gn = n0 + nn, gkb = k0 + kb;
        const bool v = gn < N && gkb < K;
        cp_async4(&gB[buf][kb][nn], v ? (TB ? B + gn + (int64_t)gkb * ldb : B + gkb + (int64_t)gn * ldb) : B, v);
      }
      if (beta != 0.f && k0 + GK >= K) {
        float* gC = sm.gcbuf + buf * 4096;
#pragma unroll 4
        for (int t = 0; t < 4096 / BT; ++t) {
          const int e = tid + BT * t, mm = e % TM, nn = e / TM;
          const int gm = m0 + mm, gn = n0 + nn;
          const bool v = gm < M && gn < N;
          cp_async4(gC + e, v ? C + gm + (int64_t)gn * ldc : C, v);
        }
      }
    }
    cp_async_commit();  // one group per stage index, empty past the end
  };
  issue(0);
  issue(1);
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int s = 0; s < total; ++s) {
    cp_async_wait<1>();  // this thread's copies of stage s have landed
    __syncthreads();     // everyone's have; and stage s - 1 is no longer read
    issue(s + 2);        // into the buffer of stage s - 1
    const int buf = s % GSTAGES;
    const int tile = s / nk;
    const bool last = s - tile * nk == nk - 1;
    const int m0 = (tile % tiles_m) * TM, n0 = (tile / tiles_m) * TN;
#pragma unroll 8
    for (int k = 0; k < GK; ++k) {
      float a[4], bb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = gA[buf][k][tx + RX * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bb[j] = gB[buf][k][ty + RY * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], bb[j], acc[i][j]);
    }
    if (last) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int n = n0 + ty + RY * j;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int m = m0 + tx + RX * i;
          float v = alpha * acc[i][j];
          if (beta != 0.f) v = fmaf(beta, sm.gcbuf[buf * 4096 + (ty + RY * j) * TM + tx + RX * i], v);
          if (m < M && n < N) C[m + (int64_t)n * ldc] = v;
          acc[i][j] = 0.f;
        }
      }
    }
  }
  cp_async_wait<0>();
  __syncthreads();
}

// Tile shape by the output's shape: a narrow side of at most 32 gets the
// 128 x 32 (or 32 x 128) tile instead of half-empty 64 x 64 tiles.
template <bool TA, bool TB>
__device__ void cta_gemm(int M, int N, int K, float alpha, const float* __restrict__ A, int64_t lda,
                         const float* __restrict__ B, int64_t ldb, float beta, float* C,
                         int64_t ldc, Smem& sm) {
  if (N <= 32)
    cta_gemm_t<TA, TB, 128, 32>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, sm);
  else if (M <= 32)
    cta_gemm_t<TA, TB, 32, 128>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, sm);
  else
    cta_gemm_t<TA, TB, 64, 64>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, sm);
}

__device__ void cta_copy(int rows, int cols, const float* src, int64_t lds, float* dst,
                         int64_t ldd) {
  for (int64_t e = threadIdx.x; e < (int64_t)rows * cols; e += BT) {
    const int i = (int)(e % rows), j = (int)(e / rows);
    dst[i + j * ldd] = src[i + j * lds];
  }
  __syncthreads();
}

__device__ void cta_identity(int n, float* X) {
  for (int64_t e = threadIdx.x; e < (int64_t)n * n; e += BT) {
    const int i = (int)(e % n), j = (int)(e / n);
    X[e] = (i == j) ? 1.f : 0.f;
  }
  __syncthreads();
}

__device__ double cta_sum(double v, Smem& sm) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sm.red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < NWARP; ++i) s += sm.red[i];
  __syncthreads();
  return s;
}

// ------------------------------------------------------ Householder QR
// In-place QR of an r x c panel (c <= BMAX): R on and above the diagonal,
// exact zeros below; W (r x c, ld r) explicit; tau in sm.tau (FP64).
// Norms and reflector scalars are FP64 (same convention as the FP64 path).
__device__ void cta_householder(int r, int c, float* Pn, int64_t ldp, float* W, Smem& sm) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int j = 0; j < c; ++j) {
    double ss = 0.0;
    for (int i = j + 1 + tid; i < r; i += BT) {
      const double x = Pn[i + (int64_t)j * ldp];
      ss = fma(x, x, ss);
    }
    ss = cta_sum(ss, sm);
    if (tid == 0) {
      const double alpha = Pn[j + (int64_t)j * ldp];
      double tau, beta, scale;
      if (ss == 0.0) {
        tau = 0.0; beta = alpha; scale = 0.0;
      } else {
        const double nrm = sqrt(fma(alpha, alpha, ss));
        beta = (alpha >= 0.0) ? -nrm : nrm;
        tau = (beta - alpha) / beta;
        scale = 1.0 / (alpha - beta);
      }
      sm.coef[0] = tau; sm.coef[1] = scale; sm.coef[2] = beta;
      sm.tau[j] = tau;
    }
    __syncthreads();
    const double tau = sm.coef[0];
    const float scale = (float)sm.coef[1];
    for (int l = j + 1 + warp; l < c; l += NWARP) {
      float d = 0.f;
      for (int i = j + lane; i < r; i += 32) {
        const float v = (i == j) ? 1.f : Pn[i + (int64_t)j * ldp] * scale;
        d = fmaf(v, Pn[i + (int64_t)l * ldp], d);
      }
      for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
      if (lane == 0) sm.wv[l] = (float)(tau * (double)d);
    }
    __syncthreads();
    if (tau != 0.0) {
      const int rr = r - j;
      for (int64_t e = tid; e < (int64_t)rr * (c - j - 1); e += BT) {
        const int i = j + (int)(e % rr), l = j + 1 + (int)(e / rr);
        const float v = (i == j) ? 1.f : Pn[i + (int64_t)j * ldp] * scale;
        Pn[i + (int64_t)l * ldp] = fmaf(-v, sm.wv[l], Pn[i + (int64_t)l * ldp]);
      }
    }
    __syncthreads();
    for (int i = tid; i < r; i += BT) {
      float w;
      if (i < j) w = 0.f;
      else if (i == j) w = 1.f;
      else w = (tau != 0.0) ? Pn[i + (int64_t)j * ldp] * scale : 0.f;
      W[i + (int64_t)j * r] = w;
      if (i > j) Pn[i + (int64_t)j * ldp] = 0.f;
      if (i == j) Pn[i + (int64_t)j * ldp] = (float)sm.coef[2];
    }
    __syncthreads();
  }
}

// The same factorization with the panel held in shared memory (in the GEMM
// buffers, which are idle here) when r c fits: one read and one write of the
// panel instead of three passes over it per column.  The arithmetic and its
// order are those of cta_householder, so the two give identical bits.
constexpr int QR_SMEM_FLOATS = GBUF + GCBUF;
__device__ void cta_householder_smem(int r, int c, float* Pn, int64_t ldp, float* W, Smem& sm) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  float* P = sm.gbuf;  // column l at P[l * r], contiguous with gcbuf
  for (int64_t e = tid; e < (int64_t)r * c; e += BT) {
    const int i = (int)(e % r), l = (int)(e / r);
    P[e] = Pn[i + (int64_t)l * ldp];
  }
  __syncthreads();
  for (int j = 0; j < c; ++j) {
    const float* pj = P + (int64_t)j * r;
    double ss = 0.0;
    for (int i = j + 1 + tid; i < r; i += BT) {
      const double x = pj[i];
      ss = fma(x, x, ss);
    }
    ss = cta_sum(ss, sm);
    if (tid == 0) {
      const double alpha = pj[j];
      double tau, beta, scale;
      if (ss == 0.0) {
        tau = 0.0; beta = alpha; scale = 0.0;
      } else {
        const double nrm = sqrt(fma(alpha, alpha, ss));
        beta = (alpha >= 0.0) ? -nrm : nrm;
        tau = (beta - alpha) / beta;
        scale = 1.0 / (alpha - beta);
      }
      sm.tau[j] = tau;
      sm.qscale[j] = (float)scale;
      sm.qbeta[j] = (float)beta;
    }
    __syncthreads();
    const double tau = sm.tau[j];
    const float scale = sm.qscale[j];
    // Each warp takes whole columns l > j: the dot w_j^T p_l (every lane ends
    // with the same sum) and then p_l -= w_j (tau w_j^T p_l) on its own.
    if (tau != 0.0) {
      for (int l = j + 1 + warp; l < c; l += NWARP) {
        float* pl = P + (int64_t)l * r;
        float d = 0.f;
        for (int i = j + lane; i < r; i += 32) {
          const float v = (i == j) ? 1.f : pj[i] * scale;
          d = fmaf(v, pl[i], d);
        }
        for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
        const float wl = (float)(tau * (double)d);
        for (int i = j + lane; i < r; i += 32) {
          const float v = (i == j) ? 1.f : pj[i] * scale;
          pl[i] = fmaf(-v, wl, pl[i]);
        }
      }
    }
    __syncthreads();
  }
  // R (with exact zeros below the diagonal) back to the panel; W explicit
  for (int64_t e = tid; e < (int64_t)r * c; e += BT) {
    const int i = (int)(e % r), l = (int)(e / r);
    const float x = P[e];
    float w, y;
    if (i < l) { w = 0.f; y = x; }
    else if (i == l) { w = 1.f; y = sm.qbeta[l]; }
    else { w = (sm.tau[l] != 0.0) ? x * sm.qscale[l] : 0.f; y = 0.f; }
    W[i + (int64_t)l * r] = w;
    Pn[i + (int64_t)l * ldp] = y;
  }
  __syncthreads();
}

__device__ void cta_qr(int r, int c, float* Pn, int64_t ldp, float* W, Smem& sm) {
  if ((int64_t)r * c <= QR_SMEM_FLOATS)
    cta_householder_smem(r, c, Pn, ldp, W, sm);
  else
    cta_householder(r, c, Pn, ldp, W, sm);
}

// Error-free transformation of a sum: s + e == a + b exactly (Knuth's two-sum).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float z = s - a;
  e = (a - (s - z)) + (b - z);
}

// Gm (c x c, ld c, FP64, both triangles) = W^T W for the stored FP32
// reflectors W (r x c, ld r, unit lower trapezoidal).  Compensated dot
// products (Ogita, Rump & Oishi 2005, "Accurate sum and dot product", Dot2):
// every product is split exactly by an FMA and the running sum is carried
// with a two-sum, so the result is as accurate as an FP64 accumulation while
// the arithmetic stays FP32 (one SM's FP64 rate is 1/64 of its FP32 rate).
__device__ void cta_gram64(int r, int c, const float* __restrict__ W, double* __restrict__ Gm) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int j = 0; j < c; ++j) {
    for (int i = warp; i <= j; i += NWARP) {
      float s = 0.f, comp = 0.f;
      for (int k = j + lane; k < r; k += 32) {  // w_j vanishes above row j, and i <= j
        const float a = W[k + (int64_t)i * r], b = W[k + (int64_t)j * r];
        const float p = a * b;
        const float pe = fmaf(a, b, -p);
        float t, te;
        two_sum(s, p, t, te);
        s = t;
        comp += te + pe;
      }
      for (int o = 16; o > 0; o >>= 1) {
        const float s2 = __shfl_xor_sync(0xffffffffu, s, o);
        const float c2 = __shfl_xor_sync(0xffffffffu, comp, o);
        float t, te;
        two_sum(s, s2, t, te);
        s = t;
        comp += c2 + te;
      }
      if (lane == 0) {
        const double g = (double)s + (double)comp;
        Gm[i + (int64_t)j * c] = g;
        Gm[j + (int64_t)i * c] = g;
      }
    }
  }
  __syncthreads();
}

// S (c x c, FP64, in sm.S) with H_1...H_c = I - W S W^T, from the Gram matrix
// Gm = W^T W (c x c, ld c, FP64, global).  tau_j is reset to 2 / |w_j|^2 of the
// stored reflector (0 stays 0), so that each H_j, and I - W S W^T with them,
// is orthogonal to FP64 accuracy for the FP32 W that the updates apply.
__device__ void cta_wy(int c, const double* Gm, Smem& sm) {
  for (int e = threadIdx.x; e < BMAX * (BMAX + 1); e += BT) (&sm.S[0][0])[e] = 0.0;
  if (threadIdx.x < c && sm.tau[threadIdx.x] != 0.0)
    sm.tau[threadIdx.x] = 2.0 / Gm[threadIdx.x + (int64_t)threadIdx.x * c];
  __syncthreads();
  for (int j = 0; j < c; ++j) {
    const double tj = sm.tau[j];
    if (threadIdx.x < j) {
      const int i = threadIdx.x;
      double s = 0.0;
      for (int l = i; l < j; ++l) s = fma(sm.S[l][i], Gm[l + (int64_t)j * c], s);
      sm.S[j][i] = -tj * s;
    }
    if (threadIdx.x == 0) sm.S[j][j] = tj;
    __syncthreads();
  }
}

// ----------------------------------------------------------- small SVD
__device__ __forceinline__ void rr_pair_b(int round, int t, int P, int* p, int* q) {
  int a, c;
  if (t == 0) { a = P - 1; c = round; }
  else { a = (round + t) % (P - 1); c = (round - t + (P - 1)) % (P - 1); }
  *p = a < c ? a : c;
  *q = a < c ? c : a;
}

// One-sided Jacobi sweeps on sm.svB (bi columns), rotations accumulated in
// sm.svV, until a sweep rotates nothing or max_sweeps.
//
// The stopping threshold on |cos| is a few FP32 ulps, independent of bi: the
// orthogonality of U_s = B V / D is that of the converged columns, and it
// enters U and T at every fold-back.  Reaching it needs a_p.a_q without the
// rounding noise of an FP32 dot product (about sqrt(bi) ulp of |a_p||a_q|,
// which near convergence is far above a_p.a_q itself), so that one is a
// compensated dot product.  Every lane of a group ends with bit-identical
// sums, hence every row of the pair gets the same rotation.
__device__ void cta_jacobi_sweeps(int bi, int max_sweeps, Smem& sm) {
  const int tid = threadIdx.x;
  const int P = (bi + 1) & ~1, npairs = P / 2;
  int tpp = 1;
  while (tpp < 32 && tpp * 2 * npairs <= BT) tpp *= 2;
  const int g = tid / tpp, sub = tid % tpp;
  const bool active = g < npairs;
  const float tol = 4.f * 0x1.0p-24f;
  if (tid == 0) sm.flag = 0;
  __syncthreads();
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    for (int round = 0; round < P - 1; ++round) {
      int p = 0, q = 0;
      if (active) rr_pair_b(round, g, P, &p, &q);
      float sa = 0.f, sb = 0.f, sc = 0.f, scc = 0.f;
      if (active)
        for (int i = sub; i < bi; i += tpp) {
          const float x = sm.svB[p][i], y = sm.svB[q][i];
          sa = fmaf(x, x, sa); sb = fmaf(y, y, sb);
          const float pr = x * y, pe = fmaf(x, y, -pr);
          float t, te;
          two_sum(sc, pr, t, te);
          sc = t;
          scc += te + pe;
        }
      for (int o = tpp >> 1; o > 0; o >>= 1) {
        sa += __shfl_xor_sync(0xffffffffu, sa, o);
        sb += __shfl_xor_sync(0xffffffffu, sb, o);
        const float s2 = __shfl_xor_sync(0xffffffffu, sc, o);
        const float c2 = __shfl_xor_sync(0xffffffffu, scc, o);
        float t, te;
        two_sum(sc, s2, t, te);  // t and te do not depend on the operand order
        sc = t;
        scc = (scc + c2) + te;   // nor does this sum
      }
      sc += scc;
      if (active && q < bi && sc != 0.f && fabsf(sc) > tol * sqrtf(sa) * sqrtf(sb)) {
        const float zeta = (sb - sa) / (2.f * sc);
        const float t = (zeta >= 0.f ? 1.f : -1.f) / (fabsf(zeta) + hypotf(1.f, zeta));
        // correctly rounded: an approximate reciprocal square root leaves
        // cs^2 + sn^2 off 1 by a few ulp with a bias, and thousands of
        // rotations then drift the column norms of V (and of B, hence D)
        const float cs = 1.f / sqrtf(fmaf(t, t, 1.f)), sn = cs * t;
        if (sub == 0) sm.flag = 1;
        for (int i = sub; i < bi; i += tpp) {
          const float x = sm.svB[p][i], y = sm.svB[q][i];
          sm.svB[p][i] = fmaf(cs, x, -sn * y);
          sm.svB[q][i] = fmaf(sn, x, cs * y);
          const float u = sm.svV[p][i], w = sm.svV[q][i];
          sm.svV[p][i] = fmaf(cs, u, -sn * w);
          sm.svV[q][i] = fmaf(sn, u, cs * w);
        }
      }
      __syncthreads();
    }
    const int any = sm.flag;
    __syncthreads();
    if (tid == 0) sm.flag = 0;
    __syncthreads();
    if (!any) break;
  }
}

// SVD of the bi x bi block B (column-major, ld ldb): D descending in sm.D,
// Us, Vs (bi x bi, ld bi, global); signs as in the other paths.
//
// FP32 sweeps to convergence leave two errors of the size of the rounding
// accumulated over all the rotations (about sqrt(#rotations) ulp): V is
// not quite orthogonal, and the rotated B is not quite B0 V.  Both are
// removed by a refinement: V64 = V (3I - V^T V)/2 (one Newton-Schulz step,
// Gram compensated, result held in FP64), B1 = B0 V64 (FP64 accumulation),
// and FP32 sweeps on B1 from V = I, which are near-identity rotations with
// correspondingly small rounding.  The output V is V64 V2.
__device__ void cta_svd(int bi, const float* Bg, int64_t ldb, float* Us, float* Vs, Smem& sm) {
  const int tid = threadIdx.x;
  const int P = (bi + 1) & ~1;
  for (int e = tid; e < P * BMAX; e += BT) {
    const int j = e / BMAX, i = e % BMAX;
    sm.svB[j][i] = (j < bi && i < bi) ? Bg[i + (int64_t)j * ldb] : 0.f;
    sm.svV[j][i] = (j < bi && i < bi && i == j) ? 1.f : 0.f;
  }
  __syncthreads();
  cta_jacobi_sweeps(bi, 30, sm);
  // H' = -(V^T V - I) / 2 into svB (FP32: it is of the order of the rounding)
  for (int e = tid; e < bi * bi; e += BT) {
    const int i = e % bi, j = e / bi;
    if (i > j) continue;
    float sg = 0.f, cg = 0.f;
    for (int k = 0; k < bi; ++k) {
      const float x = sm.svV[i][k], y = sm.svV[j][k];
      const float pr = x * y, pe = fmaf(x, y, -pr);
      float t, te;
      two_sum(sg, pr, t, te);
      sg = t;
      cg += te + pe;
    }
    const float h = -0.5f * (((i == j) ? sg - 1.f : sg) + cg);  // sg - 1 is exact
    sm.svB[j][i] = h;
    sm.svB[i][j] = h;
  }
  __syncthreads();
  // V64 = V + V H' (FP64) into sm.S, S(i, j) at S[j][i]
  for (int e = tid; e < bi * bi; e += BT) {
    const int i = e % bi, j = e / bi;
    double acc = 0.0;
    for (int l = 0; l < bi; ++l) acc = fma((double)sm.svV[l][i], (double)sm.svB[j][l], acc);
    sm.S[j][i] = (double)sm.svV[j][i] + acc;
  }
  __syncthreads();
  // B1 = B0 V64 (FP64 accumulation), V2 = I
  for (int e = tid; e < P * BMAX; e += BT) {
    const int j = e / BMAX, i = e % BMAX;
    float v = 0.f;
    if (j < bi && i < bi) {
      double acc = 0.0;
      for (int l = 0; l < bi; ++l) acc = fma((double)Bg[i + (int64_t)l * ldb], sm.S[j][l], acc);
      v = (float)acc;
    }
    sm.svB[j][i] = v;
    sm.svV[j][i] = (j < bi && i < bi && i == j) ? 1.f : 0.f;
  }
  __syncthreads();
  cta_jacobi_sweeps(bi, 10, sm);
  // V = V64 V2 (FP64 accumulation) through Vs, then back into svV
  for (int e = tid; e < bi * bi; e += BT) {
    const int i = e % bi, j = e / bi;
    double acc = 0.0;
    for (int l = 0; l < bi; ++l) acc = fma(sm.S[l][i], (double)sm.svV[j][l], acc);
    Vs[i + j * bi] = (float)acc;
  }
  __syncthreads();
  for (int e = tid; e < bi * bi; e += BT) {
    const int i = e % bi, j = e / bi;
    sm.svV[j][i] = Vs[i + j * bi];
  }
  __syncthreads();
  // norms, order, signs
  if (tid < bi) {
    const int j = tid;
    double s2 = 0.0;
    float best = -1.f;
    int bi_row = 0;
    for (int i = 0; i < bi; ++i) {
      s2 += (double)sm.svB[j][i] * sm.svB[j][i];
      const float a = fabsf(sm.svV[j][i]);
      if (a > best) { best = a; bi_row = i; }
    }
    sm.D[j] = (float)sqrt(s2);
    sm.vbest[j] = sm.svV[j][bi_row];
  }
  __syncthreads();
  if (tid < bi) {
    const int j = tid;
    int rk = 0;
    for (int l = 0; l < bi; ++l) rk += (sm.D[l] > sm.D[j]) || (sm.D[l] == sm.D[j] && l < j);
    sm.rankof[j] = rk;
  }
  __syncthreads();
  for (int e = tid; e < bi * bi; e += BT) {
    const int j = e / bi, i = e % bi, pos = sm.rankof[j];
    const float sg = (sm.vbest[j] < 0.f) ? -1.f : 1.f;
    const float dj = sm.D[j];
    Vs[i + pos * bi] = sg * sm.svV[j][i];
    Us[i + pos * bi] = (dj > 0.f) ? sg * (sm.svB[j][i] / dj) : 0.f;
  }
  __syncthreads();
  // D in order (into wv as scratch, then back)
  if (tid < bi) sm.wv[sm.rankof[tid]] = sm.D[tid];
  __syncthreads();
  if (tid < bi) sm.D[tid] = sm.wv[tid];
  __syncthreads();
  // exactly-zero singular values: complete Us by Gram-Schmidt of unit vectors
  if (tid == 0) {
    int nz = 0;
    while (nz < bi && sm.D[nz] > 0.f) ++nz;
    int cand = 0;
    for (int j = nz; j < bi; ++j) {
      for (; cand < bi; ++cand) {
        for (int i = 0; i < bi; ++i) sm.wv[i] = (i == cand) ? 1.f : 0.f;
        for (int pass = 0; pass < 2; ++pass)
          for (int l = 0; l < j; ++l) {
            float d = 0.f;
            for (int i = 0; i < bi; ++i) d = fmaf(Us[i + l * bi], sm.wv[i], d);
            for (int i = 0; i < bi; ++i) sm.wv[i] = fmaf(-d, Us[i + l * bi], sm.wv[i]);
          }
        float nn = 0.f;
        for (int i = 0; i < bi; ++i) nn = fmaf(sm.wv[i], sm.wv[i], nn);
        nn = sqrtf(nn);
        if (nn > 0.5f) {
          for (int i = 0; i < bi; ++i) Us[i + j * bi] = sm.wv[i] / nn;
          ++cand;
          break;
        }
      }
    }
  }
  __syncthreads();
}

// ------------------------------------------------------------ one matrix
struct Work {
  float *G, *Y, *Z, *W, *WS, *X, *tmp, *Us, *Vs;
  double* Gm;  // BMAX x BMAX, FP64
};

__device__ Work carve(float* base, int64_t mmax) {
  Work w;
  const int64_t big = mmax * BMAX;
  w.G = base;
  w.Y = w.G + big;
  w.Z = w.Y + big;
  w.W = w.Z + big;
  w.WS = w.W + big;
  w.X = w.WS + big;
  w.tmp = w.X + big;
  w.Gm = reinterpret_cast<double*>(w.tmp + big);  // 8-byte aligned: big is even
  w.Us = w.tmp + big + 2 * BMAX * BMAX;
  w.Vs = w.Us + BMAX * BMAX;
  return w;
}

__device__ void cta_sketch(uint64_t seed, int step, int mid, int rows, int cols, float* G) {
  const PhiloxKey key{(uint32_t)seed, (uint32_t)(seed >> 32)};
  const int64_t count = (int64_t)rows * cols, npairs = (count + 1) >> 1;
  for (int64_t p = threadIdx.x; p < npairs; p += BT) {
    const uint4 w = philox4x32_10(make_uint4((uint32_t)p, (uint32_t)step, (uint32_t)mid, 0u), key);
    float z0, z1;
    box_muller_f32(w, &z0, &z1);
    const int64_t l0 = 2 * p;
    G[l0] = z0;  // G is rows x cols with ld = rows: element l at G[l]
    if (l0 + 1 < count) G[l0 + 1] = z1;
  }
  __syncthreads();
}

// W (r x bi) and sm.tau -> sm.S and WS = W S^T (r x bi).  W is read from a
// shared-memory copy when it fits below S (the same arithmetic either way).
__device__ void cta_wy_ws(int r, int bi, Work& w, Smem& sm) {
  const float* W = w.W;
  if ((int64_t)r * bi <= WY_SMEM_FLOATS) {
    for (int64_t e = threadIdx.x; e < (int64_t)r * bi; e += BT) sm.gbuf[e] = w.W[e];
    __syncthreads();
    W = sm.gbuf;
  }
  cta_gram64(r, bi, W, w.Gm);
  cta_wy(bi, w.Gm, sm);
  // WS = W S^T with S in shared memory: S^T(l, j) = S(j, l) = sm.S[l][j]
  for (int64_t e = threadIdx.x; e < (int64_t)r * bi; e += BT) {
    const int i = (int)(e % r), j = (int)(e / r);
    float s = 0.f;
    for (int l = j; l < bi; ++l) s = fmaf(W[i + (int64_t)l * r], (float)sm.S[l][j], s);
    w.WS[i + (int64_t)j * r] = s;
  }
  __syncthreads();
}

__device__ int factor_one(const BatchDesc& d, uint64_t seed, Work& w, Smem& sm) {
  const int m = (int)d.m, n = (int)d.n, b = d.b, q = d.q;
  const int p = m < n ? m : n;
  float* T = d.T;
  const int64_t ldt = m;
  // input check and copy
  int bad = 0;
  for (int64_t e = threadIdx.x; e < (int64_t)m * n; e += BT)
    bad |= !isfinite(d.A[(e % m) + (e / m) * d.lda]);
  if (__syncthreads_or(bad)) return RANDUTV_ENONFINITE;
  if (T != d.A) cta_copy(m, n, d.A, d.lda, T, ldt);
  if (d.U) cta_identity(m, d.U);
  if (d.V) cta_identity(n, d.V);

  int step = 0;
  for (int k = 0; k < p; k += b, ++step) {
    const int bi = (b < p - k) ? b : p - k;
    const int rm = m - k, rn = n - k;
    float* T22 = T + k + (int64_t)k * ldt;
    if (rn > bi) {
      cta_sketch(seed, step, d.matrix_id, rm, bi, w.G);
      cta_gemm<true, false>(rn, bi, rm, 1.f, T22, ldt, w.G, rm, 0.f, w.Y, rn, sm);
      for (int it = 0; it < q; ++it) {
        cta_gemm<false, false>(rm, bi, rn, 1.f, T22, ldt, w.Y, rn, 0.f, w.Z, rm, sm);
        cta_gemm<true, false>(rn, bi, rm, 1.f, T22, ldt, w.Z, rm, 0.f, w.Y, rn, sm);
      }
      cta_qr(rn, bi, w.Y, rn, w.W, sm);
      cta_wy_ws(rn, bi, w, sm);
      float* Tk = T + (int64_t)k * ldt;
      cta_gemm<false, false>(m, bi, rn, 1.f, Tk, ldt, w.W, rn, 0.f, w.X, m, sm);
      cta_gemm<false, true>(m, rn, bi, -1.f, w.X, m, w.WS, rn, 1.f, Tk, ldt, sm);
      if (d.V) {
        float* Vk = d.V + (int64_t)k * n;
        cta_gemm<false, false>(n, bi, rn, 1.f, Vk, n, w.W, rn, 0.f, w.X, n, sm);
        cta_gemm<false, true>(n, rn, bi, -1.f, w.X, n, w.WS, rn, 1.f, Vk, n, sm);
      }
    }
    if (rm > bi) {
      cta_qr(rm, bi, T22, ldt, w.W, sm);
      cta_wy_ws(rm, bi, w, sm);
      if (rn > bi) {
        const int nc = rn - bi;
        float* T2 = T + k + (int64_t)(k + bi) * ldt;
        cta_gemm<true, false>(nc, bi, rm, 1.f, T2, ldt, w.W, rm, 0.f, w.X, nc, sm);
        cta_gemm<false, true>(rm, nc, bi, -1.f, w.WS, rm, w.X, nc, 1.f, T2, ldt, sm);
      }
      if (d.U) {
        float* Uk = d.U + (int64_t)k * m;
        cta_gemm<false, false>(m, bi, rm, 1.f, Uk, m, w.W, rm, 0.f, w.X, m, sm);
        cta_gemm<false, true>(m, rm, bi, -1.f, w.X, m, w.WS, rm, 1.f, Uk, m, sm);
      }
    }
    cta_svd(bi, T22, ldt, w.Us, w.Vs, sm);
    if (k > 0) {
      float* Tc = T + (int64_t)k * ldt;
      cta_gemm<false, false>(k, bi, bi, 1.f, Tc, ldt, w.Vs, bi, 0.f, w.tmp, k, sm);
      cta_copy(k, bi, w.tmp, k, Tc, ldt);
    }
    if (rn > bi) {
      const int nc = rn - bi;
      float* Tr = T + k + (int64_t)(k + bi) * ldt;
      cta_gemm<true, false>(bi, nc, bi, 1.f, w.Us, bi, Tr, ldt, 0.f, w.tmp, bi, sm);
      cta_copy(bi, nc, w.tmp, bi, Tr, ldt);
    }
    if (d.V) {
      float* Vb = d.V + (int64_t)k * n;
      cta_gemm<false, false>(n, bi, bi, 1.f, Vb, n, w.Vs, bi, 0.f, w.tmp, n, sm);
      cta_copy(n, bi, w.tmp, n, Vb, n);
    }
    if (d.U) {
      float* Ub = d.U + (int64_t)k * m;
      cta_gemm<false, false>(m, bi, bi, 1.f, Ub, m, w.Us, bi, 0.f, w.tmp, m, sm);
      cta_copy(m, bi, w.tmp, m, Ub, m);
    }
    for (int e = threadIdx.x; e < bi * bi; e += BT) {
      const int i = e % bi, j = e / bi;
      T22[i + (int64_t)j * ldt] = (i == j) ? sm.D[i] : 0.f;
    }
    __syncthreads();
  }
  return 0;
}

__global__ void __launch_bounds__(BT, 2) batched_kernel(BatchArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  Smem& sm = *reinterpret_cast<Smem*>(smraw);
  __shared__ int s_idx;
  Work w = carve(a.work + (int64_t)blockIdx.x * a.work_stride, a.mmax);
  for (;;) {
    if (threadIdx.x == 0) s_idx = atomicAdd(a.next, 1);
    __syncthreads();
    const int it = s_idx;
    __syncthreads();
    if (it >= a.count) break;
    const int mi = a.order[it];
    const BatchDesc d = a.desc[mi];
    const int st = factor_one(d, a.seed, w, sm);
    if (threadIdx.x == 0) a.info[mi] = st;
    __syncthreads();
  }
}

}  // namespace

size_t batched_work_floats(int64_t mmax) {
  return (size_t)(7 * mmax * BMAX + 4 * BMAX * BMAX) + 64;
}

size_t batched_smem_bytes() { return sizeof(Smem); }

int launch_batched(const void* desc_dev, const int* order_dev, int count, int* next_dev,
                   int* info_dev, uint64_t seed, float* work, int64_t work_stride, int64_t mmax,
                   int grid, cudaStream_t st) {
  BatchArgs a;
  a.desc = (const BatchDesc*)desc_dev;
  a.order = order_dev;
  a.count = count;
  a.next = next_dev;
  a.info = info_dev;
  a.seed = seed;
  a.work = work;
  a.work_stride = work_stride;
  a.mmax = mmax;
  const size_t smem = sizeof(Smem);
  RUTV_TRY(ensure_smem((const void*)batched_kernel, smem));
  RUTV_CK(cudaMemsetAsync(next_dev, 0, sizeof(int), st));
  batched_kernel<<<grid, BT, smem, st>>>(a);
  note_launch();
  RUTV_CK(cudaGetLastError());
  return 0;
}

int batched_max_ctas_per_sm(int* out) {
  RUTV_TRY(ensure_smem((const void*)batched_kernel, sizeof(Smem)));
  RUTV_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, batched_kernel, BT, sizeof(Smem)));
  return 0;
}

int batched_desc_bytes() { return (int)sizeof(BatchDesc); }

}  // namespace rutv
