// fgmres.cu -- flexible GMRES(m) for the pressure-correction system, right-
// preconditioned by one FP32 multigrid V-cycle per Arnoldi step, as ONE
// persistent cooperative kernel per solve.
//
// The paper solves the p' equation with a preconditioned BiCGSTAB and does
// not fix the preconditioner (Sec. 3).  On GB300 the multigrid cycle is the
// cost of a preconditioned iteration, and FP64 issues at a small fraction
// of the FP32 rate; BiCGSTAB needs two cycles per iteration and cannot take
// an FP32 cycle (its short recurrences assume one fixed linear
// preconditioner).  Flexible GMRES keeps every preconditioned direction
// z_j = M_j^-1 v_j and minimises the residual over x0 + span{z_j}, so one
// FP32 cycle per step serves and rounding in the cycle only slows it
// (Saad 1993).  Everything outside the cycle is FP64: the basis V, the
// directions Z, the SpMVs, the orthogonalisation and the stopping test on
// the true residual b - A x at every restart.
//
// Per Arnoldi step: the cycle (2L - 1 grid exchanges), w = A z_j and the
// dot products of classical Gram-Schmidt with one reorthogonalisation
// (two exchanges), and the normalised v_{j+1} published (one exchange).
// The SpMV and the dot products of a step use block-contiguous row ranges,
// so they need no exchange between them.  Dot products are reduced in a
// fixed order; every block holds bit-identical scalars and runs the Givens
// rotations and the small triangular solve redundantly.
#include "amg_dev.cuh"
#include "fgmres.cuh"
#include "krylov_dev.cuh"

namespace rbffd {

namespace {

constexpr int FNT = 1024;
constexpr int FG_D = FG_MAXM + 2;  // most dot products one exchange reduces
constexpr int LDH = FG_MAXM + 1;   // leading dimension of the Hessenberg matrix
using kdev::MAXB;

// (A x)_i for the rows [r0, r1) of this block, T threads per row: f(i, Ax_i)
// on the row's first lane.  Gathers of x go through L2 (written in launch).
template <typename F>
__device__ __forceinline__ void block_spmv(int r0, int r1, int q, int ldn, int T,
                                           const int32_t *__restrict__ col,
                                           const double *__restrict__ val, const double *x,
                                           F &&f) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int gpw = 32 / T, g = lane / T, lg = lane - g * T;
  const bool active = g < gpw;
  for (int base = r0 + warp * gpw; base < r1; base += nw * gpw) {
    const int i = base + g;
    const bool valid = active && i < r1;
    double s = 0.0;
    if (valid) {
      for (int j0 = lg; j0 < q; j0 += kdev::CH * T) {
        int c[kdev::CH];
        double a[kdev::CH];
#pragma unroll
        for (int u = 0; u < kdev::CH; ++u) {
          const int j = j0 + u * T;
          const int64_t e = (int64_t)j * ldn + i;
          c[u] = j < q ? __ldg(col + e) : -1;
          a[u] = j < q ? __ldg(val + e) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < kdev::CH; ++u)
          if (c[u] >= 0) s += a[u] * __ldcg(x + c[u]);
      }
    }
    double tot = s;
    for (int u = 1; u < T; ++u) tot += __shfl_sync(0xffffffffu, s, (lane + u) & 31);
    if (valid && lg == 0) f(i, tot);
  }
}

// Block partials of the dot products (w, u_d), d < D, over rows [r0, r1):
// warp d takes product d (u_d = V_d for d < nv, u_d = w for d = nv).
// Partial d of block lb goes to part[d * MAXB + lb].
__device__ __forceinline__ void block_dots(int r0, int r1, int n, const double *w,
                                           const double *V, int nv, double *part, int lb) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int d = warp; d <= nv; d += nw) {
    const double *u = d < nv ? V + (size_t)d * n : w;
    double t = 0.0;
    for (int r = r0 + lane; r < r1; r += 32) t += __ldcg(w + r) * __ldcg(u + r);
    t = kdev::wsum(t);
    if (lane == 0) part[d * MAXB + lb] = t;
  }
}

// After every block has published its partials: barrier, then the D totals
// in a fixed order into tot[0..D).  False if a wait gave up.
__device__ __forceinline__ bool reduce_all(const amgdev::Ctx &c, const double *part, int D,
                                           double *tot, unsigned int &epoch) {
  if (!amgdev::sync(c, epoch)) return false;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int d = warp; d < D; d += nw) {
    double t = 0.0;
    for (int b = lane; b < c.nb; b += 32) t += __ldcg(part + d * MAXB + b);
    t = kdev::wsum(t);
    if (lane == 0) tot[d] = t;
  }
  __syncthreads();
  return true;
}

struct FgState {
  double bnorm, beta, relres;
  int it, restarts, state, k, stop;
};

}  // namespace

template <int NT>
__global__ void __launch_bounds__(NT) k_fgmres(FgmresArgs A) {
  __shared__ double H[LDH * FG_MAXM];
  __shared__ double cs[FG_MAXM], sn[FG_MAXM], g[FG_MAXM + 1], y[FG_MAXM];
  __shared__ double tot[FG_D];
  __shared__ double stot[16];
  __shared__ double sred[2 * NT];
  __shared__ FgState st;
  const int lb = blockIdx.x, nb = gridDim.x;
  const int tid = lb * NT + threadIdx.x, stride = nb * NT;
  const int n = A.n, m = A.m;
  const bool leader = threadIdx.x == 0;
  amgdev::Ctx c{n,  A.q, A.ldn,  A.tpr,         A.col,  A.flags, &A.bar->err,
                lb, nb,  tid,    stride,        tid >> 5, stride >> 5, stot};
  unsigned int epoch = 1;
  // this block's row range and its threads per row
  const int R = (n + nb - 1) / nb;
  const int r0 = min(n, lb * R), r1 = min(n, r0 + R);
  int Tb = 1;
  for (int t = 2; t <= 8; ++t)
    if ((32 / t) * (NT / 32) >= R) Tb = t;
  double *part0 = A.part, *part1 = A.part + FG_D * MAXB;
  double *V = A.V, *Z = A.Z;
  bool ok = true;

  if (leader) {
    st.bnorm = st.beta = 0.0;
    st.relres = 1.0;
    st.it = st.restarts = 0;
    st.state = KRY_RUNNING;
    st.stop = 0;
  }
  __syncthreads();

  // ---- r = b - A x into V_0, with (b, b) and (r, r)
  auto residual = [&](bool first) -> bool {
    double bb = 0.0, rr = 0.0;
    block_spmv(r0, r1, A.q, A.ldn, Tb, A.col, A.val, A.x, [&](int i, double ax) {
      const double bi = A.b[i], ri = bi - ax;
      V[i] = ri;
      bb += bi * bi;
      rr += ri * ri;
    });
    double v2[2] = {bb, rr};
    double *outs[2] = {part0, part0 + MAXB};
    kdev::block_partials<NT, 2>(v2, sred, outs, lb);
    if (!reduce_all(c, part0, 2, tot, epoch)) return false;
    if (leader) {
      if (first) st.bnorm = sqrt(tot[0]);
      st.beta = sqrt(tot[1]);
      st.relres = st.bnorm > 0.0 ? st.beta / st.bnorm : 0.0;
      if (st.bnorm == 0.0) st.state = KRY_OK;
      else if (!(st.relres == st.relres)) st.state = KRY_DIVERGED;
      else if (st.relres <= A.tol) st.state = KRY_OK;
      else if (st.it >= A.maxit) st.state = KRY_NOCONV;
    }
    __syncthreads();
    return true;
  };

  if (!residual(true)) ok = false;
  if (ok && st.bnorm == 0.0) {
    for (int i = tid; i < n; i += stride) A.x[i] = 0.0;
  }

  while (ok && st.state == KRY_RUNNING) {
    // ---- start of a cycle: v_0 = r / beta, published
    {
      const double inv = 1.0 / st.beta;
      for (int i = r0 + (int)threadIdx.x; i < r1; i += NT) V[i] = __ldcg(V + i) * inv;
      if (leader) {
        g[0] = st.beta;
        for (int k = 1; k <= FG_MAXM; ++k) g[k] = 0.0;
        st.k = 0;
      }
      if (!amgdev::sync(c, epoch)) { ok = false; break; }
    }
    int j = 0;
    for (; j < m; ++j) {
      double *vj = V + (size_t)j * n, *w = V + (size_t)(j + 1) * n, *zj = Z + (size_t)j * n;
      // z_j = M^-1 v_j (FP32 cycle), published by its last exchange
      if (!amgdev::vcycle(A.amg, c, vj, zj, epoch)) { ok = false; break; }
      // w = A z_j on this block's rows; dots (w, v_i), i <= j, and (w, w)
      block_spmv(r0, r1, A.q, A.ldn, Tb, A.col, A.val, zj, [&](int i, double az) { w[i] = az; });
      __syncthreads();
      block_dots(r0, r1, n, w, V, j + 1, part0, lb);
      if (!reduce_all(c, part0, j + 2, tot, epoch)) { ok = false; break; }
      if (leader)
        for (int i = 0; i <= j; ++i) H[i + LDH * j] = tot[i];
      __syncthreads();
      // w' = w - sum h_i v_i; reorthogonalisation dots (w', v_i), (w', w')
      for (int r = r0 + (int)threadIdx.x; r < r1; r += NT) {
        double t = __ldcg(w + r);
        for (int i = 0; i <= j; ++i) t -= H[i + LDH * j] * __ldcg(V + (size_t)i * n + r);
        w[r] = t;
      }
      __syncthreads();
      block_dots(r0, r1, n, w, V, j + 1, part1, lb);
      if (!reduce_all(c, part1, j + 2, tot, epoch)) { ok = false; break; }
      if (leader) {
        double s2 = 0.0;
        for (int i = 0; i <= j; ++i) {
          H[i + LDH * j] += tot[i];
          s2 += tot[i] * tot[i];
        }
        const double hn2 = tot[j + 1] - s2;
        const double hn = hn2 > 0.0 ? sqrt(hn2) : 0.0;
        H[j + 1 + LDH * j] = hn;
        // previous rotations on column j, then a new one
        for (int i = 0; i < j; ++i) {
          const double a = H[i + LDH * j], b = H[i + 1 + LDH * j];
          H[i + LDH * j] = cs[i] * a + sn[i] * b;
          H[i + 1 + LDH * j] = -sn[i] * a + cs[i] * b;
        }
        const double a = H[j + LDH * j], b = H[j + 1 + LDH * j];
        const double rr = sqrt(a * a + b * b);
        cs[j] = rr > 0.0 ? a / rr : 1.0;
        sn[j] = rr > 0.0 ? b / rr : 0.0;
        H[j + LDH * j] = rr;
        H[j + 1 + LDH * j] = 0.0;
        g[j + 1] = -sn[j] * g[j];
        g[j] = cs[j] * g[j];
        st.it++;
        st.k = j + 1;
        const double est = fabs(g[j + 1]) / st.bnorm;
        st.stop = !(est == est) ? 2 : (est <= A.tol || hn == 0.0 || st.it >= A.maxit) ? 1 : 0;
        y[0] = hn;  // the norm for the normalisation below
      }
      __syncthreads();
      if (st.stop == 2) {
        if (leader) st.state = KRY_DIVERGED;
        __syncthreads();
        break;
      }
      // v_{j+1} = (w' - sum c_i v_i) / h_{j+1,j}, published (skipped when the
      // cycle ends here: the basis vector is not used)
      if (st.stop || j + 1 == m) break;
      {
        const double hn = y[0];
        const double inv = 1.0 / hn;
        for (int r = r0 + (int)threadIdx.x; r < r1; r += NT) {
          double t = __ldcg(w + r);
          for (int i = 0; i <= j; ++i) t -= tot[i] * __ldcg(V + (size_t)i * n + r);
          w[r] = t * inv;
        }
      }
      if (!amgdev::sync(c, epoch)) { ok = false; break; }
    }
    if (!ok || st.state != KRY_RUNNING) break;
    // ---- y = H^-1 g on the k columns (upper triangular), x += Z y
    if (leader) {
      const int k = st.k;
      for (int i = k - 1; i >= 0; --i) {
        double t = g[i];
        for (int l = i + 1; l < k; ++l) t -= H[i + LDH * l] * y[l];
        y[i] = t / H[i + LDH * i];
      }
    }
    __syncthreads();
    for (int r = r0 + (int)threadIdx.x; r < r1; r += NT) {
      double t = A.x[r];
      for (int i = 0; i < st.k; ++i) t += y[i] * __ldcg(Z + (size_t)i * n + r);
      A.x[r] = t;
    }
    if (!amgdev::sync(c, epoch)) { ok = false; break; }
    if (leader) st.restarts++;
    __syncthreads();
    // ---- true residual; stop or restart from it
    if (!residual(false)) { ok = false; break; }
  }

  if (lb == 0 && leader) {
    A.out->iters = st.it;
    A.out->restarts = st.restarts;
    A.out->status = ok ? st.state : KRY_TIMEOUT;
    A.out->relres = st.relres;
  }
}

size_t fgmres_partials_doubles(int nblocks) {
  (void)nblocks;
  return (size_t)2 * FG_D * MAXB;
}

int fgmres_max_blocks(rbffd_ctx *ctx) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fgmres<FNT>, FNT, 0) !=
          cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    return 0;
  }
  int cap = per_sm * ctx->num_sms;
  if (cap > ctx->num_sms) cap = ctx->num_sms;
  if (cap > MAXB) cap = MAXB;
  return cap;
}

int fgmres_launch(rbffd_ctx *ctx, int nblocks, const FgmresArgs &args) {
  if (nblocks < 1 || nblocks > MAXB || args.m < 1 || args.m > FG_MAXM || !args.amg) {
    set_error("fgmres_launch: bad arguments (blocks %d, m %d)", nblocks, args.m);
    return RBFFD_EINVAL;
  }
  RBFFD_CK(cudaMemsetAsync(args.bar, 0, sizeof(GridBarrier), ctx->stream));
  RBFFD_CK(cudaMemsetAsync(args.flags, 0, sizeof(unsigned int) * nblocks, ctx->stream));
  void *kargs[] = {(void *)&args};
  cudaError_t e = cudaLaunchCooperativeKernel((const void *)k_fgmres<FNT>, dim3(nblocks),
                                              dim3(FNT), kargs, 0, ctx->stream);
  ctx->launches++;
  if (e != cudaSuccess) {
    set_error("cooperative launch of k_fgmres failed: %s", cudaGetErrorString(e));
    return RBFFD_ECUDA;
  }
  return RBFFD_OK;
}

}  // namespace rbffd
