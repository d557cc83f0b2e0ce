// amg_dev.cuh -- one V-cycle of the smoothed-aggregation hierarchy inside
// the persistent BiCGSTAB kernel (the preconditioner application
// z = M^-1 b), with a grid exchange between dependent steps.
//
// From a zero start: pre-smooth x_l = w D^-1 b_l (row-local; on level 0 the
// caller does it in the loop that writes b_0), residual y_l = b_l - A_l x_l,
// restriction b_{l+1} = R_l y_l, ..., coarsest x = A_L^-1 b_L (dense
// inverse), then on the way up x_l += P_l (result of level l+1) and the
// post-smoothed result y_l = x_l + w D^-1 (b_l - A_l x_l); level 0 writes
// its result to `out`.  4 (L - 1) + 1 exchanges per cycle.
//
// Level 0 uses the solve's ELL matrix (T threads per row); the CSR levels
// use one warp per row (rows of 10 to 100 entries, few rows); the
// prolongation one thread per row.  Vectors written in this launch are read
// with __ldcg (coherent L2).
#pragma once
#include "amg.cuh"
#include "krylov.cuh"
#include "krylov_dev.cuh"

namespace rbffd {
namespace amgdev {

// sum_k val[k] x[col[k]] over row i of a CSR matrix, one warp per row
__device__ __forceinline__ double csr_row(const int32_t *__restrict__ ptr,
                                          const int32_t *__restrict__ col,
                                          const double *__restrict__ val, const double *x, int i,
                                          int lane) {
  const int s = __ldg(ptr + i), e = __ldg(ptr + i + 1);
  double t = 0.0;
  for (int k = s + lane; k < e; k += 32) t += __ldg(val + k) * __ldcg(x + __ldg(col + k));
  return kdev::wsum(t);
}

struct Ctx {
  const KrylovArgs *A;
  int lb, nb, tid, stride, wglobal, nwarps;
  double *stot;
};

__device__ __forceinline__ bool sync(const Ctx &c, unsigned int &epoch) {
  return kdev::exchange<0, double>(c.A->flags, &c.A->bar->err, epoch++, nullptr, nullptr,
                                   c.stot, c.lb, c.nb);
}

// z = V-cycle(b0) into out; level 0's pre-smoothed x (= w D^-1 b0) must be
// in place and published (an exchange since it was written).
__device__ __noinline__ bool vcycle(const AmgDev *__restrict__ G, const Ctx &c,
                                    const double *b0, double *out, unsigned int &epoch) {
  const KrylovArgs &A = *c.A;
  const int L = G->nlev;
  const int lane = threadIdx.x & 31;
  // ---- down
  for (int l = 0; l + 1 < L; ++l) {
    const AmgLevel &Lv = G->lev[l];
    const double *bl = l == 0 ? b0 : Lv.b;
    double *y = Lv.y;
    const double *x = Lv.x;
    if (l == 0) {
      const double *xs[1] = {x};
      kdev::spmv_rows<1, double>(A.n, A.q, A.ldn, A.tpr, A.col, A.val, xs, c.wglobal, c.nwarps,
                                 [&](int i, const double *ax) { y[i] = __ldcg(bl + i) - ax[0]; });
    } else {
      for (int i = c.wglobal; i < Lv.n; i += c.nwarps) {
        const double ax = csr_row(Lv.a_ptr, Lv.a_col, Lv.a_val, x, i, lane);
        if (lane == 0) y[i] = __ldcg(bl + i) - ax;
      }
    }
    if (!sync(c, epoch)) return false;
    const AmgLevel &Nx = G->lev[l + 1];
    const bool last = l + 2 == L;
    for (int k = c.wglobal; k < Nx.n; k += c.nwarps) {
      const double t = csr_row(Lv.r_ptr, Lv.r_col, Lv.r_val, y, k, lane);
      if (lane == 0) {
        Nx.b[k] = t;
        if (!last) Nx.x[k] = __ldg(Nx.wdinv + k) * t;
      }
    }
    if (!sync(c, epoch)) return false;
  }
  // ---- coarsest: dense inverse
  {
    const AmgLevel &Cl = G->lev[L - 1];
    const int nc = Cl.n;
    const double *bc = L == 1 ? b0 : Cl.b;
    double *yc = L == 1 ? out : Cl.y;
    for (int i = c.wglobal; i < nc; i += c.nwarps) {
      double t = 0.0;
      for (int j = lane; j < nc; j += 32) t += __ldg(G->cinv + (size_t)i * nc + j) * __ldcg(bc + j);
      t = kdev::wsum(t);
      if (lane == 0) yc[i] = t;
    }
    if (!sync(c, epoch)) return false;
  }
  // ---- up
  for (int l = L - 2; l >= 0; --l) {
    const AmgLevel &Lv = G->lev[l];
    const double *xc = G->lev[l + 1].y;
    double *x = Lv.x;
    for (int i = c.tid; i < Lv.n; i += c.stride) {
      const int s = __ldg(Lv.p_ptr + i), e = __ldg(Lv.p_ptr + i + 1);
      double t = __ldcg(x + i);
      for (int k = s; k < e; ++k) t += __ldg(Lv.p_val + k) * __ldcg(xc + __ldg(Lv.p_col + k));
      x[i] = t;
    }
    if (!sync(c, epoch)) return false;
    const double *bl = l == 0 ? b0 : Lv.b;
    double *res = l == 0 ? out : Lv.y;
    if (l == 0) {
      const double *xs[1] = {x};
      kdev::spmv_rows<1, double>(
          A.n, A.q, A.ldn, A.tpr, A.col, A.val, xs, c.wglobal, c.nwarps, [&](int i, const double *ax) {
            res[i] = __ldcg(x + i) + __ldg(Lv.wdinv + i) * (__ldcg(bl + i) - ax[0]);
          });
    } else {
      for (int i = c.wglobal; i < Lv.n; i += c.nwarps) {
        const double ax = csr_row(Lv.a_ptr, Lv.a_col, Lv.a_val, x, i, lane);
        if (lane == 0) res[i] = __ldcg(x + i) + __ldg(Lv.wdinv + i) * (__ldcg(bl + i) - ax);
      }
    }
    if (!sync(c, epoch)) return false;
  }
  return true;
}

}  // namespace amgdev
}  // namespace rbffd
