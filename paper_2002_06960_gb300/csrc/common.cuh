// Shared device/host helpers of the randUTV library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/randutv.h"

namespace rutv {

// ----------------------------------------------------------------- host side

// Records a CUDA error for randutv_last_error() and returns RANDUTV_ECUDA.
int cuda_fail(cudaError_t e, const char* what);

#define RUTV_CK(call)                                     \
  do {                                                    \
    cudaError_t _e = (call);                              \
    if (_e != cudaSuccess) return ::rutv::cuda_fail(_e, #call); \
  } while (0)

#define RUTV_TRY(x)          \
  do {                       \
    int _r = (x);            \
    if (_r != 0) return _r;  \
  } while (0)

// Records a message for randutv_last_error().
void set_last_error(const char* msg);

// Counts kernel launches (the library's own kernels only).
void note_launch(int n = 1);

// Per-kernel-class timing (tracing): when enabled, every launch of the
// library is bracketed by a CUDA event pair on its stream and tagged with the
// algorithmic flops and bytes of that launch.
enum KernelClass { K_PHILOX = 0, K_DGEMM, K_QR, K_WY, K_SVD, K_OTHER, K_BGEMM, K_CONVERT,
                   K_SVD32, K_REORTH, K_ADJOINT, K_NCLASS };  // K_REORTH spans a whole pass (its
                                                  // launches also count in their own class)
struct ProfScope {
  ProfScope(int cls, double flops, double bytes, cudaStream_t st);
  ~ProfScope();
  int slot;
  cudaStream_t st;
};

// Device properties cached per device.
struct DevInfo {
  int sms;
  int smem_optin;
};
const DevInfo& dev_info();

// Scratch: one growing allocation per device, carved into aligned pieces.
struct Arena {
  char* base = nullptr;
  size_t cap = 0;
  size_t used = 0;
  void* take(size_t bytes) {
    size_t off = (used + 255) & ~size_t(255);
    used = off + bytes;
    return base + off;
  }
};
// Makes sure the device scratch holds at least `bytes`; returns status.
int scratch_reserve(size_t bytes, Arena* out);

// The device status words of the current device (64 words, persistent).
int status_words(unsigned** out);

// Raises the dynamic shared-memory limit of kernel `func` on the current
// device to at least `bytes` (the attribute is kept per device, so a process
// that uses several GPUs sets it on each).  Thread-safe.
int ensure_smem(const void* func, size_t bytes);

// Sets cudaFuncAttributeNonPortableClusterSizeAllowed on `func` for the
// current device, once per device.  Thread-safe.
int ensure_nonportable_cluster(const void* func);

// Words of device status shared by the kernels of one call: [0] error code,
// [1] where the error happened, [2..3] barrier counter and generation.
struct StatusWords {
  unsigned* words;  // device, 64 words
};

// Milliseconds a bounded device-side wait may spin before it gives up.
constexpr unsigned long long kWaitLimitNs = 2000000000ull;

// ---------------------------------------------------------------- device side

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_gpu(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void red_release_add_gpu(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier for a cooperatively launched grid (all CTAs resident).
// `bar` points at a counter that is zero when the launch starts.  The k-th
// barrier of every CTA adds 1 to it and waits until it reaches k * nblocks;
// `epoch` is the CTA's count of barriers so far (kept by thread 0 of the
// caller, starting at 0).  A monotonic count needs no reset by a last
// arriver, which halves the latency of a barrier on 152 CTAs.  Every wait
// is bounded: after kWaitLimitNs the waiting CTA sets err[0] =
// RANDUTV_ETIMEOUT (err[1] = `site`) and every CTA then returns false from
// this and every later barrier, so the kernel can leave early.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned nblocks, unsigned* err,
                                             unsigned site, unsigned& epoch) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    // The error word is read only while waiting: a CTA that gives up never
    // arrives, and the others see its error within 64 polls.  The acquiring
    // poll (with the block barrier after it) orders what follows, so no fence
    // is needed after it.
    int ok = 1;
    const unsigned target = nblocks * (++epoch);
    __threadfence();
    red_release_add_gpu(bar, 1u);
    if (ld_acquire_gpu(bar) < target) {
      const unsigned long long t0 = globaltimer_ns();
      unsigned spins = 0;
      while (ld_acquire_gpu(bar) < target) {
        if ((++spins & 63u) == 0) {
          if (ld_acquire_gpu(err) != 0) { ok = 0; break; }
          if (globaltimer_ns() - t0 > kWaitLimitNs) {
            if (atomicCAS(err, 0u, (unsigned)RANDUTV_ETIMEOUT) == 0u) atomicExch(err + 1, site);
            ok = 0;
            break;
          }
        }
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Deterministic block-wide sum (fixed tree); `red` is blockDim.x/32 doubles.
__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < nw; ++i) s += red[i];
  return s;
}

}  // namespace rutv
