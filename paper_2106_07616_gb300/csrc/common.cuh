// common.cuh -- shared host/device helpers of the CUDA path (context,
// errors, launch accounting, deterministic reductions, bounded grid barrier).
#pragma once
#include <cstddef>

#include <cuda/atomic>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <cstdarg>
#include <cstdio>

#include "rbffd.h"

struct rbffd_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int num_sms = 0;
  size_t budget = 0;  // 0 = no cap
  // device bytes held (dev_reserve / dev_release: the multigrid build's
  // host thread allocates beside the caller)
  std::atomic<size_t> used{0};
  int64_t launches = 0;
  // device-side waits of this context's launches: 2^wait_log2 cycles (0:
  // the default 2^31), rbffd_ctx_set_wait_limit
  int wait_log2 = 0;
  // multigrid hierarchies built on this context get the composed cycle when
  // it pays (rbffd_ctx_set_amg_compose)
  bool amg_compose = true;
  // level 0 of large hierarchies built on the device (rbffd_ctx_set_amg_device_setup)
  bool amg_device_setup = true;
  // flexible GMRES's Gram-Schmidt (rbffd_ctx_set_fgmres_reorth): 0 one
  // pass, 1 two passes a step, 2 two passes with the second delayed
  int fgmres_reorth = 1;
  // pinned host scratch for small read-backs
  void *pinned = nullptr;
  size_t pinned_bytes = 0;
  // problems and batches alive on this context; rbffd_ctx_destroy waits for
  // the last one (Python may finalise objects in any order at exit)
  int refs = 0;
  bool closing = false;
  // live kernel timing (rbffd_ctx_profile)
  bool prof = false;
  cudaEvent_t ev[8] = {};
  rbffd_kernel_stat kst[RBFFD_KSTAT_COUNT] = {};
};

namespace rbffd {

// a - b along an axis that is periodic with length L (L = 0: bounded): the
// difference moved by one period when it exceeds half of one, i.e. the
// nearest periodic image (paper Sec. 3.1: clouds wrap around a periodic
// boundary).  Round-to-nearest steps, no fusion.
__host__ __device__ __forceinline__ double pdiff(double a, double b, double L) {
#ifdef __CUDA_ARCH__
  double d = __dsub_rn(a, b);
  if (L > 0.0) {
    if (d > 0.5 * L) d = __dsub_rn(d, L);
    else if (d < -0.5 * L) d = __dadd_rn(d, L);
  }
#else
  double d = a - b;
  if (L > 0.0) {
    if (d > 0.5 * L) d = d - L;
    else if (d < -0.5 * L) d = d + L;
  }
#endif
  return d;
}

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

// Reference counting of the objects that point at a context.
void ctx_ref(rbffd_ctx *ctx);
void ctx_unref(rbffd_ctx *ctx);

// Device allocation charged to the context's budget.
int dev_alloc(rbffd_ctx *ctx, void **p, size_t bytes);
void dev_free(rbffd_ctx *ctx, void *p, size_t bytes);
// count `bytes` against the context's budget (false: it would exceed it;
// the error text is set) / give them back
bool dev_reserve(rbffd_ctx *ctx, size_t bytes);
void dev_release(rbffd_ctx *ctx, size_t bytes);
// Small pinned host buffer of at least `bytes` (owned by the context).
int pinned(rbffd_ctx *ctx, size_t bytes, void **out);

inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

// Event pair k (0..3) brackets a launch when profiling is on.
inline void prof_begin(rbffd_ctx *ctx, int k) {
  if (ctx->prof) cudaEventRecord(ctx->ev[2 * k], ctx->stream);
}
inline void prof_end(rbffd_ctx *ctx, int k) {
  if (ctx->prof) cudaEventRecord(ctx->ev[2 * k + 1], ctx->stream);
}
// After the stream has been synchronised: add pair k to class `cls`.
inline void prof_collect(rbffd_ctx *ctx, int k, int cls, double units, double bytes) {
  if (!ctx->prof) return;
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, ctx->ev[2 * k], ctx->ev[2 * k + 1]) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  rbffd_kernel_stat &s = ctx->kst[cls];
  s.launches += 1;
  s.ms += ms;
  s.units += units;
  s.bytes += bytes;
}

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
  // bound of every device-side wait of the launch: 2^wait_log2 clock cycles
  // (0: the default 2^31, about a second); set per context
  // (rbffd_ctx_set_wait_limit) when the barrier is reset before a launch
  int wait_log2;
};
static_assert(offsetof(GridBarrier, wait_log2) == offsetof(GridBarrier, err) + sizeof(int),
              "wait_cycles() reads the limit beside the error word");

// The wait bound of a barrier, given its error word (the limit is the next
// word of the same GridBarrier).
__device__ __forceinline__ long long wait_cycles(const int *err) {
  const int s = err[1];
  return 1ll << (s > 0 ? s : 31);
}

// Grid-wide barrier for a cooperative launch: arrive with a release
// fetch_add, the last arriver publishes the next generation with a release
// store, the others poll it with acquire loads.  Every wait is bounded:
// after 2^wait_log2 clock cycles (default 2^31, about a second) the block
// records a timeout in bar->err and goes on; callers test the return value
// and leave the kernel.
__device__ __forceinline__ bool grid_sync(GridBarrier *bar, unsigned int nblocks,
                                          unsigned int &gen) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    cuda::atomic_ref<unsigned int, cuda::thread_scope_device> cnt(bar->count);
    cuda::atomic_ref<unsigned int, cuda::thread_scope_device> g(bar->gen);
    cuda::atomic_ref<int, cuda::thread_scope_device> er(bar->err);
    unsigned int arrived = cnt.fetch_add(1u, cuda::memory_order_acq_rel);
    if (arrived == nblocks - 1) {
      cnt.store(0u, cuda::memory_order_relaxed);
      g.store(gen + 1, cuda::memory_order_release);
    } else {
      long long t0 = clock64();
      while (g.load(cuda::memory_order_acquire) == gen) {
        if (clock64() - t0 > wait_cycles(&bar->err)) {
          er.store(1, cuda::memory_order_relaxed);
          break;
        }
      }
    }
    s_ok = er.load(cuda::memory_order_relaxed) == 0;
  }
  gen++;
  __syncthreads();
  return s_ok != 0;
}

// Zero the barriers bars[0..m) on the context's stream and give them the
// context's wait limit (one kernel, so it can be captured in a graph).
int reset_barriers(rbffd_ctx *ctx, GridBarrier *bars, int m);

}  // namespace rbffd
