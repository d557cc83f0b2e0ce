// weights.cu -- S2: PHS r^3 + polynomial collocation weights, one warp per
// cloud, the augmented (q+m) x (q+m+3) system in shared memory, FP64 LU with
// partial pivoting (paper Sec. 2, Eqs. RBF_interp_mat_vec ..
// RBF_interp_mat_vec_L_solve).
//
// The matrix build uses explicit round-to-nearest intrinsics (no fused
// multiply-add), as the oracle does.  On GB300 the kernel is bound by the
// FP64 pipe (about 2 FMA lanes per clock per SM), so every FP64 instruction
// counts and the kernel spends them only on the arithmetic itself:
//   - the elimination and the back substitution use one fused multiply-add
//     per update instead of a product and a difference;
//   - the trailing update of step k deals the (N-k-1) x (W-k-1) elements
//     over the 32 lanes in row-major order, so every FP64 instruction of
//     the warp carries 32 useful updates (lanes that owned whole columns
//     left 35% of them idle at N = 45);
//   - the multipliers use one reciprocal of the pivot per step, and the
//     scalings by 1/h and 1/h^2 one reciprocal each, instead of a division
//     per element (an FP64 division is a sequence of FP64 instructions);
//   - Phi is symmetric: each r^3 (and its square root) is computed once for
//     the upper triangle and stored twice.
// The weights then differ from the oracle's unfused, dividing elimination
// by rounding only (a different elimination order, LAPACK's, moves the
// 200 x 200 cavity weights by at most 4e-13 relative), well inside the
// 1e-10 the weights are held to.
#include "abi_guard.cuh"
#include "common.cuh"
#include "weights.cuh"

namespace rbffd {

// Monomial exponents in graded order, x power descending inside a degree:
// 1, x, y, x^2, xy, y^2, ...  The order for degree k is a prefix of the
// order for degree k+1, so one table serves every degree up to 8.
__constant__ int8_t c_ax[45];
__constant__ int8_t c_ay[45];

static bool g_tables_ready[64] = {false};

static int ensure_tables(int device) {
  if (device >= 0 && device < 64 && g_tables_ready[device]) return RBFFD_OK;
  int8_t ax[45], ay[45];
  int l = 0;
  for (int d = 0; d <= 8; ++d)
    for (int a = d; a >= 0; --a) {
      ax[l] = (int8_t)a;
      ay[l] = (int8_t)(d - a);
      ++l;
    }
  RBFFD_CK(cudaMemcpyToSymbol(c_ax, ax, sizeof(ax)));
  RBFFD_CK(cudaMemcpyToSymbol(c_ay, ay, sizeof(ay)));
  if (device >= 0 && device < 64) g_tables_ready[device] = true;
  return RBFFD_OK;
}

__device__ __forceinline__ double ipow_rn(double b, int e) {
  double v = 1.0;
  for (int t = 0; t < e; ++t) v = __dmul_rn(v, b);
  return v;
}

__global__ void k_weights(int n, const double *__restrict__ x, const double *__restrict__ y,
                          int q, const int32_t *__restrict__ idx, int m, int wpb,
                          double *__restrict__ wx, double *__restrict__ wy,
                          double *__restrict__ wl, int *first_singular, double Lx, double Ly) {
  extern __shared__ double smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int N = q + m, LD = (N + 3) | 1, W = N + 3;
  double *M = smem + (size_t)warp * (N * LD + 2 * q);
  double *xi = M + N * LD;
  double *eta = xi + q;
  for (int i = blockIdx.x * wpb + warp; i < n; i += gridDim.x * wpb) {
    const int32_t *cl = idx + (int64_t)i * q;
    const double xc = x[i], yc = y[i];
    // cloud radius h = max distance
    double d2m = 0.0;
    for (int a = lane; a < q; a += 32) {
      int j = cl[a];
      double dx = pdiff(x[j], xc, Lx), dy = pdiff(y[j], yc, Ly);
      double d2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
      d2m = fmax(d2m, d2);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d2m = fmax(d2m, __shfl_xor_sync(0xffffffffu, d2m, o));
    double h = __dsqrt_rn(d2m);
    if (h == 0.0) h = 1.0;
    const double hinv = __drcp_rn(h);
    for (int a = lane; a < q; a += 32) {
      int j = cl[a];
      xi[a] = __dmul_rn(pdiff(x[j], xc, Lx), hinv);
      eta[a] = __dmul_rn(pdiff(y[j], yc, Ly), hinv);
    }
    __syncwarp();
    // Phi block: r^3, symmetric with a zero diagonal; the q(q-1)/2 pairs
    // a < b of the upper triangle are dealt over the lanes in row-major
    // order (row a holds q-1-a of them)
    for (int a = lane; a < q; a += 32) M[a * LD + a] = 0.0;
    {
      // pair number e -> (a, b): past the end of row a (b >= q) it goes on
      // at b - q positions into row a + 1, whose first pair is (a+1, a+2)
      const int P = q * (q - 1) / 2;
      int a = 0, b = 1 + lane;
      while (a < q - 1 && b >= q) { b += a + 2 - q; ++a; }
      for (int e = lane; e < P; e += 32) {
        double dx = __dsub_rn(xi[a], xi[b]), dy = __dsub_rn(eta[a], eta[b]);
        double r = __dsqrt_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
        const double r3 = __dmul_rn(__dmul_rn(r, r), r);
        M[a * LD + b] = r3;
        M[b * LD + a] = r3;
        b += 32;
        while (a < q - 1 && b >= q) { b += a + 2 - q; ++a; }
      }
    }
    // P and P^T blocks
    for (int e = lane; e < q * m; e += 32) {
      int a = e / m, l = e - a * m;
      double pv = __dmul_rn(ipow_rn(xi[a], c_ax[l]), ipow_rn(eta[a], c_ay[l]));
      M[a * LD + q + l] = pv;
      M[(q + l) * LD + a] = pv;
    }
    for (int e = lane; e < m * m; e += 32) {
      int l = e / m, b = e - l * m;
      M[(q + l) * LD + q + b] = 0.0;
    }
    // right-hand sides: d/dxi, d/deta and Laplacian of r^3 about the centre,
    // then of the monomials at the centre
    for (int a = lane; a < q; a += 32) {
      double xa = xi[a], ya = eta[a];
      double rj = __dsqrt_rn(__dadd_rn(__dmul_rn(xa, xa), __dmul_rn(ya, ya)));
      double r3 = __dmul_rn(3.0, rj);
      M[a * LD + N + 0] = __dmul_rn(r3, __dsub_rn(0.0, xa));
      M[a * LD + N + 1] = __dmul_rn(r3, __dsub_rn(0.0, ya));
      M[a * LD + N + 2] = __dmul_rn(9.0, rj);
    }
    for (int l = lane; l < m; l += 32) {
      int ax = c_ax[l], ay = c_ay[l];
      M[(q + l) * LD + N + 0] = (ax == 1 && ay == 0) ? 1.0 : 0.0;
      M[(q + l) * LD + N + 1] = (ax == 0 && ay == 1) ? 1.0 : 0.0;
      M[(q + l) * LD + N + 2] = ((ax == 2 && ay == 0) || (ax == 0 && ay == 2)) ? 2.0 : 0.0;
    }
    __syncwarp();
    // LU with partial pivoting; the right-hand sides ride along
    bool singular = false;
    for (int k = 0; k < N; ++k) {
      // pivot search on the bit patterns of |a|: for finite doubles with the
      // sign bit cleared, unsigned 64-bit order is the order of the values,
      // so this picks exactly the row an FP64 comparison would (ties to the
      // lowest row) while keeping the compares off the FP64 pipe
      unsigned long long best = 0ull;
      int piv = N;
      for (int r = k + lane; r < N; r += 32) {
        const unsigned long long a =
            (unsigned long long)__double_as_longlong(M[r * LD + k]) & 0x7fffffffffffffffull;
        if (piv == N || a > best) { best = a; piv = r; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int op = __shfl_xor_sync(0xffffffffu, piv, o);
        if (op < N && (piv == N || ob > best || (ob == best && op < piv))) { best = ob; piv = op; }
      }
      if (best == 0ull) { singular = true; break; }
      if (piv != k) {
        for (int c = k + lane; c < W; c += 32) {
          double t = M[k * LD + c];
          M[k * LD + c] = M[piv * LD + c];
          M[piv * LD + c] = t;
        }
        __syncwarp();
      }
      const double kinv = __drcp_rn(M[k * LD + k]);
      for (int r = k + 1 + lane; r < N; r += 32) M[r * LD + k] = __dmul_rn(M[r * LD + k], kinv);
      __syncwarp();
      {
        // trailing update, element e = (r - k - 1) * Cc + (c - k - 1) on lane e % 32
        const int Cc = W - k - 1, E = (N - k - 1) * Cc;
        int r = k + 1 + lane / Cc, c = k + 1 + lane % Cc;
        int e = lane;
        // two elements per trip: their loads go out before either update
        for (; e + 32 < E; e += 64) {
          int r2 = r, c2 = c + 32;
          while (c2 >= W) { c2 -= Cc; ++r2; }
          const double l1 = M[r * LD + k], u1 = M[k * LD + c], a1 = M[r * LD + c];
          const double l2 = M[r2 * LD + k], u2 = M[k * LD + c2], a2 = M[r2 * LD + c2];
          M[r * LD + c] = __fma_rn(-l1, u1, a1);
          M[r2 * LD + c2] = __fma_rn(-l2, u2, a2);
          r = r2;
          c = c2 + 32;
          while (c >= W) { c -= Cc; ++r; }
        }
        if (e < E) M[r * LD + c] = __fma_rn(-M[r * LD + k], M[k * LD + c], M[r * LD + c]);
      }
      __syncwarp();
    }
    if (singular) {
      for (int a = lane; a < q; a += 32) {
        if (wx) wx[(int64_t)i * q + a] = 0.0;
        if (wy) wy[(int64_t)i * q + a] = 0.0;
        if (wl) wl[(int64_t)i * q + a] = 0.0;
      }
      if (lane == 0) atomicMin(first_singular, i);
      __syncwarp();
      continue;
    }
    // column-oriented back substitution for the three right-hand sides
    for (int j = N - 1; j >= 0; --j) {
      if (lane < 3) M[j * LD + N + lane] = __ddiv_rn(M[j * LD + N + lane], M[j * LD + j]);
      __syncwarp();
      for (int e = lane; e < 3 * j; e += 32) {
        int r = e / 3, s = e - 3 * r;
        M[r * LD + N + s] =
            __fma_rn(-M[r * LD + j], M[j * LD + N + s], M[r * LD + N + s]);
      }
      __syncwarp();
    }
    const double h2inv = __drcp_rn(__dmul_rn(h, h));
    for (int a = lane; a < q; a += 32) {
      int64_t o = (int64_t)i * q + a;
      if (wx) wx[o] = __dmul_rn(M[a * LD + N + 0], hinv);
      if (wy) wy[o] = __dmul_rn(M[a * LD + N + 1], hinv);
      if (wl) wl[o] = __dmul_rn(M[a * LD + N + 2], h2inv);
    }
    __syncwarp();
  }
}

int weights_config(int q, int degree, int *wpb, size_t *smem) {
  int m = (degree + 1) * (degree + 2) / 2;
  int N = q + m, LD = (N + 3) | 1;
  size_t per = (size_t)(N * LD + 2 * q) * sizeof(double);
  // as many warps as shared memory holds, up to 12 (N = 45: 12 x 18 KB):
  // the FP64 pipe needs several warps per scheduler to hide the shared-
  // memory latency in front of each update
  int w = (int)((224 * 1024) / per);
  if (w > 12) w = 12;
  if (w < 1) return RBFFD_EINVAL;
  *wpb = w;
  *smem = per * w;
  return RBFFD_OK;
}

int weights_run(rbffd_ctx *ctx, int n, const double *x, const double *y, int q,
                const int32_t *idx, int degree, double *wx, double *wy, double *wl,
                int *d_first_singular, double Lx, double Ly) {
  int m = (degree + 1) * (degree + 2) / 2;
  RBFFD_TRY(ensure_tables(ctx->device));
  int wpb;
  size_t smem;
  RBFFD_TRY(weights_config(q, degree, &wpb, &smem));
  RBFFD_CK(cudaFuncSetAttribute(k_weights, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem));
  int blocks = (n + wpb - 1) / wpb;
  int cap = ctx->num_sms * 16;
  if (blocks > cap) blocks = cap;
  k_weights<<<blocks, 32 * wpb, smem, ctx->stream>>>(n, x, y, q, idx, m, wpb, wx, wy, wl,
                                                     d_first_singular, Lx, Ly);
  return after_launch(ctx, "k_weights");
}

int weights_check_args(int n, int q, int degree) {
  if (n < 1 || q < 1 || q > n || degree < 0 || degree > 8) return RBFFD_EINVAL;
  int m = (degree + 1) * (degree + 2) / 2;
  if (q < m || q + m > 96) return RBFFD_EINVAL;
  return RBFFD_OK;
}

}  // namespace rbffd

using namespace rbffd;

extern "C" int rbffd_weights(rbffd_ctx *ctx, int32_t n, const double *x, const double *y,
                             int32_t q, const int32_t *idx, int32_t degree, double *wx,
                             double *wy, double *wl, int32_t *first_singular) {
  return guarded([&]() -> int {
    if (!ctx || !x || !y || !idx || weights_check_args(n, q, degree) != RBFFD_OK) {
      set_error("rbffd_weights: bad arguments (n=%d q=%d degree=%d)", n, q, degree);
      return RBFFD_EINVAL;
    }
    RBFFD_CK(cudaSetDevice(ctx->device));
    int *dfs = nullptr;
    RBFFD_TRY(dev_alloc(ctx, (void **)&dfs, sizeof(int)));
    int big = 0x7fffffff;
    int rc = RBFFD_OK;
    if (cudaMemcpyAsync(dfs, &big, sizeof(int), cudaMemcpyHostToDevice, ctx->stream) !=
        cudaSuccess) {
      rc = RBFFD_ECUDA;
    } else {
      rc = weights_run(ctx, n, x, y, q, idx, degree, wx, wy, wl, dfs, 0.0, 0.0);
    }
    int hfs = big;
    if (rc == RBFFD_OK) {
      if (cudaMemcpyAsync(&hfs, dfs, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream) !=
              cudaSuccess ||
          cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
        set_error("rbffd_weights: read-back failed");
        rc = RBFFD_ECUDA;
      }
    }
    cudaStreamSynchronize(ctx->stream);
    dev_free(ctx, dfs, sizeof(int));
    if (first_singular) *first_singular = (rc == RBFFD_OK && hfs != big) ? hfs : -1;
    if (rc == RBFFD_OK && hfs != big) {
      set_error("rbffd_weights: singular collocation matrix at point %d", hfs);
      return RBFFD_ESINGULAR;
    }
    return rc;
  });
}
