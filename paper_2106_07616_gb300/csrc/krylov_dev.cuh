// krylov_dev.cuh -- device building blocks of the persistent Krylov
// kernels: a T-threads-per-row ELL SpMV, block partial sums and the
// grid-wide publish/wait/reduce exchange (an arrival counter).
#pragma once
#include <type_traits>

#include "common.cuh"
#include "inner_arith.cuh"

namespace rbffd {
namespace kdev {

constexpr int CH = 12;                   // gathers batched per lane before the FMAs
constexpr int MAXB = 160;                // blocks a launch may use
constexpr int BPL = (MAXB + 31) / 32;    // flags / partials per lane

template <typename T>
__device__ __forceinline__ T wsum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ ff wsum(ff v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
    v = ff_add(v, ff(__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)));
  return v;
}

// coherent (L2) loads of the partial-sum types
__device__ __forceinline__ double ld_cg(const double *p) { return __ldcg(p); }
__device__ __forceinline__ float ld_cg(const float *p) { return __ldcg(p); }
__device__ __forceinline__ ff ld_cg(const ff *p) {
  const float2 t = __ldcg(reinterpret_cast<const float2 *>(p));
  return ff(t.x, t.y);
}

// ---- windows of gathered vectors staged in shared memory ------------------
// A launch may give its CTAs dynamic shared memory; then every CTA finds,
// once per launch (win_init), the column window [w0, w1) that its own rows'
// ELL entries reach -- the clouds keep it a few lattice lines wide in
// row-major or Morton order -- and every level-0 SpMV stages that window of
// the gathered vector into shared memory first (one coalesced pass from L2,
// after the exchange that published the vector) and gathers from there:
// one 4- or 8-byte shared-memory read per nonzero instead of one 32-byte L2
// sector.  Columns outside the window (a window wider than the buffer keeps
// the part around the CTA's own rows) are read from L2 as before.  Without
// dynamic shared memory the capacity is zero and nothing is staged.
extern __shared__ __align__(16) unsigned char kdev_dyn[];

__device__ __forceinline__ unsigned int dyn_smem_bytes() {
  unsigned int r;
  asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(r));
  return r;
}

// window capacity in entries: room for two FP64 vectors (two right-hand sides)
__device__ __forceinline__ int win_cap() { return (int)(dyn_smem_bytes() / 16u); }

struct RowWindow {
  int w0, w1;
};
__device__ __forceinline__ RowWindow &row_window() {
  __shared__ RowWindow w;
  return w;
}

// The window of the rows [r0, r1) of an ELL [q][ldn] column array (all
// threads of the CTA call it; ends with a barrier).
__device__ __forceinline__ void win_init(int n, int q, int ldn, const int32_t *__restrict__ col,
                                         int r0, int r1) {
  __shared__ int s_lo, s_hi;
  const int cap = win_cap();
  const int R = r1 - r0;
  if (threadIdx.x == 0) {
    s_lo = 0x7fffffff;
    s_hi = -1;
  }
  __syncthreads();
  if (cap > 0 && R > 0) {
    int lo = 0x7fffffff, hi = -1;
    for (int e = threadIdx.x; e < R * q; e += blockDim.x) {
      const int j = e / R, i = r0 + (e - j * R);
      const int c = __ldg(col + (int64_t)j * ldn + i);
      lo = min(lo, c);
      hi = max(hi, c);
    }
    atomicMin(&s_lo, lo);
    atomicMax(&s_hi, hi);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    RowWindow &w = row_window();
    if (cap <= 0 || R <= 0 || s_hi < s_lo) {
      w.w0 = w.w1 = 0;
    } else if (s_hi - s_lo + 1 <= cap) {
      w.w0 = s_lo;
      w.w1 = s_hi + 1;
    } else {  // keep the part around the CTA's own rows
      int w0 = (r0 + r1) / 2 - cap / 2;
      w0 = max(0, min(w0, n - cap));
      w.w0 = w0;
      w.w1 = min(n, w0 + cap);
    }
  }
  __syncthreads();
}

// Stage x[w0 .. w1) into the k-th buffer (all threads of the CTA; the
// barriers keep the previous use of the buffer and this copy apart).
template <typename XT>
__device__ __forceinline__ const XT *win_stage(const XT *x, int w0, int w1, int k = 0) {
  XT *buf = reinterpret_cast<XT *>(kdev_dyn + (size_t)k * win_cap() * sizeof(double));
  __syncthreads();
  for (int t = threadIdx.x; t < w1 - w0; t += blockDim.x) buf[t] = __ldcg(x + w0 + t);
  __syncthreads();
  return buf;
}

// x(c) from the staged window when it holds c, else from L2
template <typename XT>
__device__ __forceinline__ XT win_get(const XT *buf, int w0, int wlen, const XT *x, int c) {
  const unsigned int o = (unsigned int)(c - w0);
  return o < (unsigned int)wlen ? buf[o] : __ldcg(x + c);
}

// The contiguous rows [r0, r1) of the CTA that warp `wglobal` belongs to
// (warps are numbered CTA-major: wglobal = cta * wpb + warp), n rows shared
// evenly by the nwarps / wpb CTAs.  Spreading rows evenly over the CTAs
// keeps every SM busy: dealing them from warp 0 onwards left whole SMs idle
// and doubled the FP64 work of the busy ones.
__device__ __forceinline__ void cta_rows(int n, int wglobal, int nwarps, int wpb, int &r0,
                                         int &r1, int &w) {
  const int cta = wglobal / wpb, nc = nwarps / wpb;
  const int R = (n + nc - 1) / nc;
  w = wglobal - cta * wpb;
  r0 = min(n, cta * R);
  r1 = min(n, r0 + R);
}

// y_k(i) = sum_j A(i,j) x_k(j), accumulated in AT, T threads per row
// (T = 1..8, any value; the last 32 mod T lanes of a warp idle), over each
// CTA's own rows (cta_rows).  The column indices and values of a chunk of
// CH entries are loaded first, then the CH gathers, so a row costs two
// dependent memory round trips per chunk.  f(i, y) runs on the group
// leader; all 32 lanes execute the same trip count and shuffles.  Gathered
// vectors go through __ldcg (coherent L2) because other blocks of the same
// launch write them.
template <int NR, typename AT, typename VT, typename XT, typename F>
__device__ __forceinline__ void spmv_rows(int n, int q, int ldn, int T,
                                          const int32_t *__restrict__ col,
                                          const VT *__restrict__ val, XT *const *xs, int wglobal,
                                          int nwarps, F &&f) {
  const int lane = threadIdx.x & 31;
  const int gpw = 32 / T;
  const int g = lane / T;
  const int lg = lane - g * T;
  const bool active = g < gpw;
  const int wpb = blockDim.x >> 5;
  int r0, r1, w;
  cta_rows(n, wglobal, nwarps, wpb, r0, r1, w);
  // the gathered vectors' window, staged (see win_init)
  using X = typename std::remove_const<XT>::type;
  const RowWindow rw = row_window();
  const int wlen = win_cap() > 0 ? rw.w1 - rw.w0 : 0;
  const X *wb[NR];
#pragma unroll
  for (int k = 0; k < NR; ++k)
    wb[k] = wlen > 0 ? win_stage<X>(xs[k], rw.w0, rw.w1, k) : nullptr;
  for (int base = r0 + w * gpw; base < r1; base += wpb * gpw) {
    const int i = base + g;
    const bool valid = active && i < r1;
    AT s[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) s[k] = AT(0);
    if (valid) {
      for (int j0 = lg; j0 < q; j0 += CH * T) {
        int c[CH];
        VT a[CH];
#pragma unroll
        for (int u = 0; u < CH; ++u) {
          const int j = j0 + u * T;
          const int64_t e = (int64_t)j * ldn + i;
          c[u] = j < q ? __ldg(col + e) : -1;
          a[u] = j < q ? __ldg(val + e) : VT(0);
        }
#pragma unroll
        for (int u = 0; u < CH; ++u) {
          if (c[u] >= 0) {
#pragma unroll
            for (int k = 0; k < NR; ++k)
              s[k] += AT(a[u]) * AT(win_get<X>(wb[k], rw.w0, wlen, xs[k], c[u]));
          }
        }
      }
    }
    AT tot[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) tot[k] = s[k];
    for (int u = 1; u < T; ++u) {
#pragma unroll
      for (int k = 0; k < NR; ++k) tot[k] += __shfl_sync(0xffffffffu, s[k], (lane + u) & 31);
    }
    if (valid && lg == 0) f(i, tot);
  }
}

// Block-reduce V values per thread into V partials written at outs[v][b].
// The values go through shared memory (sh holds V * NT entries) and warp v
// sums value v over the block in a fixed order: NT/32 + 5 dependent adds on
// one warp, instead of 5 butterfly levels on every warp.  On GB300 an FP64
// warp-wide add occupies the FP64 pipe for ~32 cycles, so the number of
// FP64 warp instructions, not their latency, is what a reduction costs.
template <int NT, int V, typename AT>
__device__ __forceinline__ void block_partials(AT (&val)[V], AT *sh, AT *const *outs,
                                               int lb = -1) {
  if (lb < 0) lb = blockIdx.x;
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
  for (int v = 0; v < V; ++v) sh[v * NT + threadIdx.x] = val[v];
  __syncthreads();
  for (int v = w; v < V; v += NT / 32) {  // more values than warps: warp-strided
    AT t = AT(0);
#pragma unroll 8
    for (int k = 0; k < NT / 32; ++k) t += sh[v * NT + k * 32 + l];
    t = wsum(t);
    if (l == 0 && outs[v] != nullptr) outs[v][lb] = t;
  }
}

// Grid-wide exchange: publish this block's writes (rows and partials) with
// one release add on the solve's arrival counter flags[0], wait (acquire
// loads by one thread, bounded) until the counter reaches epoch * nb --
// every block has arrived at this exchange -- then reduce the V partial
// arrays in a fixed order, one warp per array.  Every block computes
// bit-identical totals.  V = 0 is a plain barrier.
// One counter word polled by one thread per block costs ~1.8 us per
// exchange across 152 blocks on GB300; one flag per block, each polled by
// every block, cost ~4.9 us (measured with the same release/acquire pair).
// The counter is zeroed before the launch and epochs count from 1, so a
// launch may make up to 2^32 / nb exchanges.
// lb, nb: this CTA's index among, and the number of, the CTAs that share
// the solve (default: the whole grid).  A single-CTA solve needs no counter.
template <int V, typename AT>
__device__ __forceinline__ bool exchange(unsigned int *flags, int *err, unsigned int epoch,
                                         AT *const *arrs, AT *tot, AT *sh, int lb = -1,
                                         int nb = -1) {
  __shared__ int s_ok;
  if (lb < 0) lb = blockIdx.x;
  if (nb < 0) nb = gridDim.x;
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (nb == 1) {
    for (int v = w; v < V; v += blockDim.x / 32) {
      AT t = arrs[v] != nullptr ? arrs[v][0] : AT(0);
      if (l == 0) sh[v] = t;
    }
    __syncthreads();
#pragma unroll
    for (int v = 0; v < V; ++v) tot[v] = sh[v];
    __syncthreads();
    return true;
  }
  if (threadIdx.x == 0) {
    cuda::atomic_ref<unsigned int, cuda::thread_scope_device> cnt(flags[0]);
    cnt.fetch_add(1u, cuda::memory_order_release);
    const unsigned int target = epoch * (unsigned int)nb;
    long long t0 = clock64();
    bool ok = true;
    for (unsigned int spin = 1; cnt.load(cuda::memory_order_acquire) < target; ++spin) {
      // another block gave up (it will not arrive): leave without the wait
      if ((spin & 1023u) == 0 && *(volatile int *)err != 0) {
        ok = false;
        break;
      }
      if (clock64() - t0 > wait_cycles(err)) {
        ok = false;
        atomicExch(err, 1);
        break;
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  for (int v = w; v < V; v += blockDim.x / 32) {
    AT t = AT(0);
    if (arrs[v] != nullptr) {
#pragma unroll
      for (int u = 0; u < BPL; ++u) {
        const int b = l + 32 * u;
        if (b < nb) t += ld_cg(arrs[v] + b);
      }
    }
    t = wsum(t);
    if (l == 0) sh[v] = t;
  }
  __syncthreads();
#pragma unroll
  for (int v = 0; v < V; ++v) tot[v] = sh[v];
  const bool ok = s_ok != 0;
  __syncthreads();
  return ok;
}

}  // namespace kdev
}  // namespace rbffd
