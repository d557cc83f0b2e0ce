// knn.cu -- S1: cloud selection (paper Sec. 2 clouds; one-sided clouds at
// boundaries, Sec. 3.1) with a uniform cell grid.
//
// Every point gets itself plus its q-1 nearest candidates under the total
// order (d^2, index).  d^2 is formed with explicit round-to-nearest
// intrinsics (no fused multiply-add), so the selected indices are exactly
// those of a brute-force search that evaluates dx*dx + dy*dy the same way.
// The ring search stops only when the current (q-1)-th distance is strictly
// below the clearance of the searched block of cells, so no unvisited point
// can enter or tie.  A periodic axis (period L > 0) measures differences to
// the nearest image and wraps the ring around the grid, each column (row)
// visited once at its smallest offset; a cell at wrapped offset r + 1 is
// still at least r cells away, so the clearance bound holds.
#include <mutex>
#include "abi_guard.cuh"
#include "common.cuh"
#include "knn.cuh"

namespace rbffd {

__global__ void k_bbox(int n, const double *__restrict__ x, const double *__restrict__ y,
                       double *bbox) {
  __shared__ double s[4][32];
  double xmn = 1e300, xmx = -1e300, ymn = 1e300, ymx = -1e300;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double a = x[i], b = y[i];
    xmn = fmin(xmn, a); xmx = fmax(xmx, a);
    ymn = fmin(ymn, b); ymx = fmax(ymx, b);
  }
  for (int o = 16; o > 0; o >>= 1) {
    xmn = fmin(xmn, __shfl_xor_sync(0xffffffffu, xmn, o));
    xmx = fmax(xmx, __shfl_xor_sync(0xffffffffu, xmx, o));
    ymn = fmin(ymn, __shfl_xor_sync(0xffffffffu, ymn, o));
    ymx = fmax(ymx, __shfl_xor_sync(0xffffffffu, ymx, o));
  }
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { s[0][w] = xmn; s[1][w] = xmx; s[2][w] = ymn; s[3][w] = ymx; }
  __syncthreads();
  if (w == 0) {
    int nw = blockDim.x >> 5;
    xmn = l < nw ? s[0][l] : 1e300; xmx = l < nw ? s[1][l] : -1e300;
    ymn = l < nw ? s[2][l] : 1e300; ymx = l < nw ? s[3][l] : -1e300;
    for (int o = 16; o > 0; o >>= 1) {
      xmn = fmin(xmn, __shfl_xor_sync(0xffffffffu, xmn, o));
      xmx = fmax(xmx, __shfl_xor_sync(0xffffffffu, xmx, o));
      ymn = fmin(ymn, __shfl_xor_sync(0xffffffffu, ymn, o));
      ymx = fmax(ymx, __shfl_xor_sync(0xffffffffu, ymx, o));
    }
    if (l == 0) { bbox[0] = xmn; bbox[1] = xmx; bbox[2] = ymn; bbox[3] = ymx; }
  }
}

struct Grid {
  double x0, y0, cx, cy;
  int G;
};

__device__ __forceinline__ Grid load_grid(const double *bbox, int G) {
  Grid g;
  g.G = G;
  g.x0 = bbox[0];
  g.y0 = bbox[2];
  g.cx = (bbox[1] - bbox[0]) / G;
  g.cy = (bbox[3] - bbox[2]) / G;
  if (!(g.cx > 0.0)) g.cx = 1.0;
  if (!(g.cy > 0.0)) g.cy = 1.0;
  return g;
}

__device__ __forceinline__ int cell_coord(double v, double v0, double c, int G) {
  int k = (int)floor((v - v0) / c);
  return k < 0 ? 0 : (k >= G ? G - 1 : k);
}

__global__ void k_cell_count(int n, const double *__restrict__ x, const double *__restrict__ y,
                             const double *bbox, int G, int *__restrict__ cell,
                             int *__restrict__ cnt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  Grid g = load_grid(bbox, G);
  int c = cell_coord(y[i], g.y0, g.cy, G) * G + cell_coord(x[i], g.x0, g.cx, G);
  cell[i] = c;
  atomicAdd(&cnt[c], 1);
}

// Exclusive scan of m counts by one block of 1024 threads; start[m] = total.
__global__ void k_scan(const int *__restrict__ cnt, int *__restrict__ start, int m) {
  __shared__ int s[1024];
  int t = threadIdx.x;
  int chunk = (m + 1023) / 1024;
  int b = t * chunk, e = min(m, b + chunk);
  int sum = 0;
  for (int k = b; k < e; ++k) sum += cnt[k];
  s[t] = sum;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    int v = t >= o ? s[t - o] : 0;
    __syncthreads();
    s[t] += v;
    __syncthreads();
  }
  int run = s[t] - sum;
  for (int k = b; k < e; ++k) {
    start[k] = run;
    run += cnt[k];
  }
  if (t == 1023) start[m] = s[1023];
}

__global__ void k_cell_fill(int n, const int *__restrict__ cell, const int *__restrict__ start,
                            int *__restrict__ cursor, int *__restrict__ pts) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int c = cell[i];
  int pos = atomicAdd(&cursor[c], 1);
  pts[start[c] + pos] = i;
}

__device__ __forceinline__ bool key_less(double da, int ja, double db, int jb) {
  return da < db || (da == db && ja < jb);
}

// Column (row) of the ring at offset d from c, or -1 to skip it: out of a
// bounded grid, or on a periodic axis not the smallest offset of its column.
__device__ __forceinline__ int ring_index(int c, int d, int G, bool periodic) {
  if (!periodic) {
    const int k = c + d;
    return (k < 0 || k >= G) ? -1 : k;
  }
  int canon = ((d % G) + G) % G;
  if (canon > G / 2) canon -= G;
  if (canon != d) return -1;
  return ((c + d) % G + G) % G;
}

template <int KMAX>
__global__ void __launch_bounds__(128) k_knn_query(
    int n, const double *__restrict__ x, const double *__restrict__ y,
    const int8_t *__restrict__ tag, int q, const double *bbox, int G,
    const int *__restrict__ start, const int *__restrict__ pts, int32_t *__restrict__ idx,
    int *err, double Lx, double Ly) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int K = q - 1;
  int64_t o = (int64_t)i * q;
  idx[o] = i;
  if (K == 0) return;
  Grid g = load_grid(bbox, G);
  const double xi = x[i], yi = y[i];
  const bool bnd = tag != nullptr && tag[i] != 0;
  const int ci = cell_coord(xi, g.x0, g.cx, G), cj = cell_coord(yi, g.y0, g.cy, G);
  const double cmin = fmin(g.cx, g.cy);
  double bd[KMAX];
  int bj[KMAX];
  int cnt = 0;
  for (int r = 0;; ++r) {
    for (int dy = -r; dy <= r; ++dy) {
      const int yy = ring_index(cj, dy, G, Ly > 0.0);
      if (yy < 0) continue;
      const bool edge = (dy == -r || dy == r);
      const int stp = edge ? 1 : 2 * r;
      for (int dx = -r; dx <= r; dx += stp) {
        const int xx = ring_index(ci, dx, G, Lx > 0.0);
        if (xx < 0) continue;
        int c = yy * G + xx;
        for (int s = start[c], se = start[c + 1]; s < se; ++s) {
          int j = pts[s];
          if (j == i) continue;
          if (bnd && tag[j] != 0) continue;
          double ddx = pdiff(x[j], xi, Lx);
          double ddy = pdiff(y[j], yi, Ly);
          double d2 = __dadd_rn(__dmul_rn(ddx, ddx), __dmul_rn(ddy, ddy));
          int p;
          if (cnt < K) {
            p = cnt++;
          } else if (key_less(d2, j, bd[K - 1], bj[K - 1])) {
            p = K - 1;
          } else {
            continue;
          }
          while (p > 0 && key_less(d2, j, bd[p - 1], bj[p - 1])) {
            bd[p] = bd[p - 1];
            bj[p] = bj[p - 1];
            --p;
          }
          bd[p] = d2;
          bj[p] = j;
        }
      }
    }
    if (cnt == K) {
      double clear = (double)r * cmin * (1.0 - 1e-9);
      if (bd[K - 1] < clear * clear) break;
    }
    if (r > G) break;  // every cell visited
  }
  if (cnt < K) {
    atomicExch(err, 1);
    for (int s = 0; s < K; ++s) idx[o + 1 + s] = i;
    return;
  }
  for (int s = 0; s < K; ++s) idx[o + 1 + s] = bj[s];
}

int knn_workspace_bytes(int n, KnnLayout *lay) {
  int G = (int)ceil(sqrt((double)n / 2.0));
  if (G < 1) G = 1;
  int m = G * G;
  lay->G = G;
  lay->m = m;
  size_t off = 0;
  auto take = [&](size_t b) {
    size_t at = off;
    off += (b + 255) / 256 * 256;
    return at;
  };
  lay->off_bbox = take(4 * sizeof(double));
  lay->off_err = take(sizeof(int));
  lay->off_cell = take((size_t)n * sizeof(int));
  lay->off_cnt = take((size_t)(m + 1) * sizeof(int));
  lay->off_start = take((size_t)(m + 1) * sizeof(int));
  lay->off_cursor = take((size_t)m * sizeof(int));
  lay->off_pts = take((size_t)n * sizeof(int));
  lay->bytes = off;
  return RBFFD_OK;
}

int knn_run(rbffd_ctx *ctx, void *ws, const KnnLayout &lay, int n, const double *x,
            const double *y, const int8_t *tag, int q, int32_t *idx, double Lx, double Ly) {
  char *b = (char *)ws;
  double *bbox = (double *)(b + lay.off_bbox);
  int *err = (int *)(b + lay.off_err);
  int *cell = (int *)(b + lay.off_cell);
  int *cnt = (int *)(b + lay.off_cnt);
  int *start = (int *)(b + lay.off_start);
  int *cursor = (int *)(b + lay.off_cursor);
  int *pts = (int *)(b + lay.off_pts);
  cudaStream_t st = ctx->stream;
  RBFFD_CK(cudaMemsetAsync(err, 0, sizeof(int), st));
  RBFFD_CK(cudaMemsetAsync(cnt, 0, sizeof(int) * (lay.m + 1), st));
  RBFFD_CK(cudaMemsetAsync(cursor, 0, sizeof(int) * lay.m, st));
  k_bbox<<<1, 1024, 0, st>>>(n, x, y, bbox);
  RBFFD_TRY(after_launch(ctx, "k_bbox"));
  int nb = (n + 255) / 256;
  k_cell_count<<<nb, 256, 0, st>>>(n, x, y, bbox, lay.G, cell, cnt);
  RBFFD_TRY(after_launch(ctx, "k_cell_count"));
  k_scan<<<1, 1024, 0, st>>>(cnt, start, lay.m);
  RBFFD_TRY(after_launch(ctx, "k_scan"));
  k_cell_fill<<<nb, 256, 0, st>>>(n, cell, start, cursor, pts);
  RBFFD_TRY(after_launch(ctx, "k_cell_fill"));
  int qb = (n + 127) / 128;
  if (q - 1 <= 32) {
    k_knn_query<32><<<qb, 128, 0, st>>>(n, x, y, tag, q, bbox, lay.G, start, pts, idx, err, Lx,
                                                     Ly);
  } else if (q - 1 <= 64) {
    k_knn_query<64><<<qb, 128, 0, st>>>(n, x, y, tag, q, bbox, lay.G, start, pts, idx, err, Lx,
                                                     Ly);
  } else {
    k_knn_query<128><<<qb, 128, 0, st>>>(n, x, y, tag, q, bbox, lay.G, start, pts, idx, err, Lx,
                                                     Ly);
  }
  RBFFD_TRY(after_launch(ctx, "k_knn_query"));
  int herr = 0;
  RBFFD_CK(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  RBFFD_CK(cudaStreamSynchronize(st));
  if (herr) {
    set_error("a boundary point has fewer than q-1 interior candidates");
    return RBFFD_EINVAL;
  }
  return RBFFD_OK;
}

}  // namespace rbffd

using namespace rbffd;

extern "C" int rbffd_build_stencils(rbffd_ctx *ctx, int32_t n, const double *x, const double *y,
                                    const int8_t *tag, int32_t q, int32_t *idx) {
  return guarded([&]() -> int {
    if (!ctx || !x || !y || !idx || n < 1 || q < 1 || q > n || q > 129) {
      set_error("rbffd_build_stencils: bad arguments (n=%d q=%d)", n, q);
      return RBFFD_EINVAL;
    }
    RBFFD_CK(cudaSetDevice(ctx->device));
    KnnLayout lay;
    knn_workspace_bytes(n, &lay);
    void *ws = nullptr;
    RBFFD_TRY(dev_alloc(ctx, &ws, lay.bytes));
    int rc = knn_run(ctx, ws, lay, n, x, y, tag, q, idx, 0.0, 0.0);
    cudaStreamSynchronize(ctx->stream);
    dev_free(ctx, ws, lay.bytes);
    return rc;
  });
}

// ---------------------------------------------------------------------------
// Cloud building without any device allocation.
//
// rbffd_build_stencils above allocates its cell-grid workspace with
// cudaMalloc on every call and frees it afterwards.  Some callers cannot do
// that: a solver loop that must keep a fixed device-memory footprint once it
// has started, or an application whose other streams must not be stalled by
// the implicit device synchronisation of cudaMalloc / cudaFree.  For them,
// rbffd_build_stencils_static takes the same workspace from a fixed array in
// device global memory that is part of this library image.  Every GPU that
// loads the library holds the array (RBFFD_STATIC_SCRATCH_BYTES) until the
// process exits.

namespace rbffd {

static __device__ __align__(256) unsigned char g_knn_scratch[RBFFD_STATIC_SCRATCH_BYTES];

// Device address of g_knn_scratch per device.  In host code the symbol is
// only a host-side stand-in, so the address has to be asked of the runtime,
// once per device, with that device current.  The lookup runs under one
// std::once_flag per device, so host threads that make their first call on
// one device at the same time do not race on the cached pointer; the result
// (the address, or the CUDA error of the lookup) is published by call_once.
static void *g_knn_scratch_ptr[64] = {nullptr};
static cudaError_t g_knn_scratch_err[64];
static std::once_flag g_knn_scratch_once[64];

static int static_scratch(int device, void **out) {
  if (device < 0 || device >= 64) {
    set_error("rbffd_build_stencils_static: device %d not supported", device);
    return RBFFD_EINVAL;
  }
  std::call_once(g_knn_scratch_once[device], [device]() {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_knn_scratch);
    if (e == cudaSuccess && p == nullptr) e = cudaErrorInvalidSymbol;
    g_knn_scratch_err[device] = e;
    g_knn_scratch_ptr[device] = e == cudaSuccess ? p : nullptr;
  });
  if (g_knn_scratch_err[device] != cudaSuccess) {
    set_error("cudaGetSymbolAddress(static cloud scratch) failed: %s",
              cudaGetErrorString(g_knn_scratch_err[device]));
    return RBFFD_ECUDA;
  }
  *out = g_knn_scratch_ptr[device];
  return RBFFD_OK;
}

}  // namespace rbffd

extern "C" int rbffd_build_stencils_static(rbffd_ctx *ctx, int32_t n, const double *x,
                                           const double *y, const int8_t *tag, int32_t q,
                                           int32_t *idx) {
  return guarded([&]() -> int {
    if (!ctx || !x || !y || !idx || n < 1 || q < 1 || q > n || q > 129) {
      set_error("rbffd_build_stencils_static: bad arguments (n=%d q=%d)", n, q);
      return RBFFD_EINVAL;
    }
    if (n > RBFFD_STATIC_MAX_POINTS) {
      set_error("rbffd_build_stencils_static: n=%d exceeds the static limit of %d points", n,
                RBFFD_STATIC_MAX_POINTS);
      return RBFFD_EINVAL;
    }
    KnnLayout lay;
    knn_workspace_bytes(n, &lay);
    if (lay.bytes > sizeof(g_knn_scratch)) {
      set_error("rbffd_build_stencils_static: workspace of %zu bytes exceeds the %zu-byte array",
                lay.bytes, sizeof(g_knn_scratch));
      return RBFFD_EINVAL;
    }
    RBFFD_CK(cudaSetDevice(ctx->device));
    void *ws = nullptr;
    RBFFD_TRY(static_scratch(ctx->device, &ws));
    // knn_run clears the counters, cursors and error word it reads before
    // writing them, so the contents left by an earlier call do not matter.
    return knn_run(ctx, ws, lay, n, x, y, tag, q, idx, 0.0, 0.0);
  });
}
