// common.cuh -- shared host/device helpers of the CUDA path (context,
// errors, launch accounting, deterministic reductions, bounded grid barrier).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>

#include "rbffd.h"

struct rbffd_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int num_sms = 0;
  size_t budget = 0;  // 0 = no cap
  size_t used = 0;
  int64_t launches = 0;
  // pinned host scratch for small read-backs
  void *pinned = nullptr;
  size_t pinned_bytes = 0;
};

namespace rbffd {

void set_error(const char *fmt, ...);
void clear_error();

#define RBFFD_CK(call)                                                                        \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) {                                                                  \
      ::rbffd::set_error("%s:%d: %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_)); \
      return RBFFD_ECUDA;                                                                     \
    }                                                                                         \
  } while (0)

#define RBFFD_TRY(expr)       \
  do {                        \
    int rc_ = (expr);         \
    if (rc_ != RBFFD_OK) return rc_; \
  } while (0)

// Check the launch that was just issued and count it.
inline int after_launch(rbffd_ctx *ctx, const char *what) {
  ctx->launches++;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("launch of %s failed: %s", what, cudaGetErrorString(e));
    return RBFFD_ECUDA;
  }
  return RBFFD_OK;
}

// Device allocation charged to the context's budget.
int dev_alloc(rbffd_ctx *ctx, void **p, size_t bytes);
void dev_free(rbffd_ctx *ctx, void *p, size_t bytes);
// Small pinned host buffer of at least `bytes` (owned by the context).
int pinned(rbffd_ctx *ctx, size_t bytes, void **out);

inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

// ------------------------------------------------------------------------
// Device helpers

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic block sum: every thread gets the same value; the order of
// additions depends only on blockDim (fixed per launch), never on timing.
template <int NT>
__device__ __forceinline__ double block_sum(double v, double *sh /* NT/32 */) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double t = (l < NT / 32) ? sh[l] : 0.0;
  t = warp_sum(t);
  return t;
}

// Sum of a partials array of length m in a fixed order (lane-strided, then
// a butterfly), computed redundantly by one warp; every block that calls it
// on the same data gets the bit-identical result.
__device__ __forceinline__ double warp_sum_array(const double *a, int m) {
  const int l = threadIdx.x & 31;
  double t = 0.0;
  for (int k = l; k < m; k += 32) t += a[k];
  return warp_sum(t);
}

struct GridBarrier {
  unsigned int count;
  unsigned int gen;
  int err;
  int pad;
};

// Grid-wide barrier for a cooperative launch.  Every wait is bounded: after
// ~2^31 clock cycles (about a second) the block records a timeout in
// bar->err and goes on; callers test the return value and leave the kernel.
__device__ __forceinline__ bool grid_sync(GridBarrier *bar, unsigned int nblocks,
                                          unsigned int &gen) {
  __syncthreads();
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    __threadfence();
    unsigned int arrived = atomicAdd(&bar->count, 1u);
    if (arrived == nblocks - 1) {
      atomicExch(&bar->count, 0u);
      __threadfence();
      atomicExch(&bar->gen, gen + 1);
    } else {
      long long t0 = clock64();
      volatile unsigned int *vg = &bar->gen;
      while (*vg == gen) {
        if (clock64() - t0 > (1ll << 31)) {
          atomicExch(&bar->err, 1);
          break;
        }
        __nanosleep(20);
      }
    }
    __threadfence();
    s_ok = (*(volatile int *)&bar->err) == 0;
  }
  gen++;
  __syncthreads();
  return s_ok != 0;
}

}  // namespace rbffd
