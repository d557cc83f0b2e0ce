// amg_dev.cuh -- one V-cycle of the smoothed-aggregation hierarchy inside
// the persistent BiCGSTAB kernel (the preconditioner application
// z = M^-1 b), with the smoothing folded into the transfer operators (see
// amg.cuh): on the way down z_l = S_l b_l and b_{l+1} = R~_l b_l in one
// phase, at the bottom y = A_L^-1 b_L (dense inverse), on the way up
// y_l = z_l + P~_l y_{l+1}; one grid exchange after each phase, 2 L - 1 per
// cycle for L levels.  b_0 (the BiCGSTAB vector p or s) must be published
// (an exchange since it was written) before the call.
//
// With the composed operators (AmgCompT) and room for the coarse vector in
// the launch's shared memory, the same cycle runs in four phases.
//
// Level 0's S uses the solve's ELL columns (T threads per row); the CSR
// operators use grp lanes per row.  The cycle computes in the hierarchy's
// value type T (FP64 or FP32, see amg.cuh); it reads b_0 and writes its
// result in the solve's vector types XT and OT (FP64 inside BiCGSTAB, FP32
// inside flexible GMRES).  Vectors written in this launch are read with __ldcg
// (coherent L2).  Ctx carries the grid-exchange state; it is independent of
// the Krylov method around the cycle.
#pragma once
#include "amg.cuh"
#include "krylov.cuh"
#include "krylov_dev.cuh"

namespace rbffd {
namespace amgdev {

// f(i, sum_k M(i,k) x(k)) for the rows of a CSR matrix, M.grp lanes per
// row (a power of two); all 32 lanes of a warp run the same trip count.
// Each lane loads CC column indices and values of its strided share first,
// then the CC gathers, so a long row costs two dependent L2 round trips per
// CC entries a lane, not per entry.
constexpr int CC = AMG_CSR_CHUNK;

// zadd (may be null): z(i) is added to the row's sum, loaded with the row
// pointers instead of after the sum.
// xs (may be null): x[0 .. xlen) staged in shared memory, gathered from there.
template <typename T, typename XT, typename F>
__device__ __forceinline__ void csr_rows(const AmgCsrT<T> &M, int nrows, const XT *x, int wglobal,
                                         int nwarps, F &&f, const T *zadd = nullptr,
                                         const XT *xs = nullptr, int xlen = 0) {
  const int lane = threadIdx.x & 31;
  const int G = M.grp, rpw = 32 / G, g = lane / G, lg = lane - g * G;
  for (int base = wglobal * rpw; base < nrows; base += nwarps * rpw) {
    const int i = base + g;
    T t = 0;
    const T zi = (zadd != nullptr && i < nrows && lg == 0) ? __ldcg(zadd + i) : T(0);
    if (i < nrows) {
      const int s = __ldg(M.ptr + i), e = __ldg(M.ptr + i + 1);
      for (int k0 = s + lg; k0 < e; k0 += CC * G) {
        int c[CC];
        T a[CC];
#pragma unroll
        for (int u = 0; u < CC; ++u) {
          const int k = k0 + u * G;
          c[u] = k < e ? __ldg(M.col + k) : -1;
          a[u] = k < e ? __ldg(M.val + k) : T(0);
        }
#pragma unroll
        for (int u = 0; u < CC; ++u)
          if (c[u] >= 0) t += a[u] * T(kdev::win_get<XT>(xs, 0, xlen, x, c[u]));
      }
    }
    for (int o = G >> 1; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (i < nrows && lg == 0) f(i, t + zi);
  }
}

// What a cycle needs from the solve around it: level 0's ELL structure,
// the grid-exchange flags and this thread's place in the grid.
struct Ctx {
  int n, q, ldn, tpr;
  const int32_t *col;
  unsigned int *flags;
  int *err;
  int lb, nb, tid, stride, wglobal, nwarps;
  double *stot;
};

__device__ __forceinline__ bool sync(const Ctx &c, unsigned int &epoch) {
  return kdev::exchange<0, double>(c.flags, c.err, epoch++, nullptr, nullptr, c.stot, c.lb,
                                   c.nb);
}

// y = A_L^-1 b on the coarsest level, one warp per row
template <typename T, typename XT, typename YT>
__device__ __forceinline__ void coarse_solve(const AmgDevT<T> *__restrict__ G, int nc,
                                             const XT *b, YT *y, const Ctx &c) {
  const int lane = threadIdx.x & 31;
  for (int i = c.wglobal; i < nc; i += c.nwarps) {
    T t = 0;
    for (int j = lane; j < nc; j += 32)
      t += __ldg(G->cinv + (size_t)i * nc + j) * T(__ldcg(b + j));
    t = kdev::wsum(t);
    if (lane == 0) y[i] = YT(t);
  }
}

// ---- the composed cycle (amg.cuh: AmgCompT)

// Chunk sums of the stacked restriction applied to b_1: warp w of the
// launch (in the order given) takes chunks w, w + nwarps, ...; a chunk
// holds at most AMG_RCHUNK = 32 x CC entries, one load of CC per lane.
template <typename T, typename XT>
__device__ __forceinline__ void comp_chunks(const AmgCompT<T> &C, const XT *b1, int wglobal,
                                            int nwarps) {
  const int lane = threadIdx.x & 31;
  for (int ch = wglobal; ch < C.nchunk; ch += nwarps) {
    const int s = __ldg(C.cs + ch), e = __ldg(C.cs + ch + 1);
    int cc[CC];
    T a[CC];
#pragma unroll
    for (int u = 0; u < CC; ++u) {
      const int k = s + lane + 32 * u;
      cc[u] = k < e ? __ldg(C.rcol + k) : -1;
      a[u] = k < e ? __ldg(C.rval + k) : T(0);
    }
    T t = 0;
#pragma unroll
    for (int u = 0; u < CC; ++u)
      if (cc[u] >= 0) t += a[u] * T(__ldcg(b1 + cc[u]));
    t = kdev::wsum(t);
    if (lane == 0) C.part[ch] = t;
  }
}

// The coarse vector: every CTA sums the chunks of all nc entries, in order,
// into its dynamic shared memory (all threads of the CTA; ends with a
// barrier).  Level s + 2's entries take seg_grp[s] lanes each.
template <typename T>
__device__ __forceinline__ const T *comp_gather(const AmgCompT<T> &C) {
  T *cv = reinterpret_cast<T *>(kdev::kdev_dyn);
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  __syncthreads();  // the buffer's previous use
  for (int s = 0; s < C.nseg; ++s) {
    const int G = C.seg_grp[s], rpw = 32 / G, g = lane / G, lg = lane - g * G;
    const int k1 = C.seg_off[s + 1];
    for (int base = C.seg_off[s] + wl * rpw; base < k1; base += wpb * rpw) {
      const int k = base + g;
      T t = 0;
      if (k < k1) {
        const int c1 = __ldg(C.kc + k + 1);
#pragma unroll 4
        for (int ch = __ldg(C.kc + k) + lg; ch < c1; ch += G) t += __ldcg(C.part + ch);
      }
      for (int o = G >> 1; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (k < k1 && lg == 0) cv[k] = t;
    }
  }
  __syncthreads();
  return cv;
}

// the launch runs the composed cycle: built, and its shared memory holds c
template <typename T>
__device__ __forceinline__ bool comp_fits(const AmgDevT<T> *__restrict__ G) {
  const int nc = G->comp.nc;
  return nc > 0 && kdev::dyn_smem_bytes() >= (unsigned int)nc * (unsigned int)sizeof(T);
}

// out = V-cycle(b0)
template <typename T, typename XT, typename OT>
__device__ __forceinline__ bool vcycle(const AmgDevT<T> *__restrict__ G, const Ctx &c,
                                       const XT *b0, OT *out, unsigned int &epoch) {
  const int L = G->nlev;
  if (L == 1) {
    coarse_solve(G, G->lev[0].n, b0, out, c);
    return sync(c, epoch);
  }
  // warp orders of the CSR phases: row groups go to warp 0 of every CTA,
  // then warp 1, ... (wfw: S_l, P~_l, the coarsest rows), or to the last
  // warp of every CTA first (wbw: R~_l), so the two products of a down
  // phase run side by side on disjoint warps of every CTA when they fit
  // (level 0's S runs on each CTA's own rows from warp 0, kdev::cta_rows),
  // and every phase spreads over all SMs
  const int wpb = blockDim.x >> 5, nbk = c.nwarps / wpb;
  const int cta = c.wglobal / wpb, wl = c.wglobal - cta * wpb;
  const int wfw = wl * nbk + cta, wbw = (wpb - 1 - wl) * nbk + cta;
  if (comp_fits(G)) {
    const AmgCompT<T> &C = G->comp;
    const AmgLevelT<T> &L0 = G->lev[0];
    const AmgLevelT<T> &L1 = G->lev[1];
    T *z0 = L0.z;
    T *b1 = L1.b;
    T *z1 = L1.z;
    T *y1 = L1.y;
    const int n1 = L1.n;
    // (A) z_0 = S_0 b_0 on this CTA's rows, b_1 = R~_0 b_0
    {
      const XT *xs[1] = {b0};
      kdev::spmv_rows<1, T>(c.n, c.q, c.ldn, G->ts0, c.col, G->s0, xs, c.wglobal, c.nwarps,
                            [&](int i, const T *sb) { z0[i] = sb[0]; });
      csr_rows(L0.R, n1, b0, wbw, c.nwarps, [&](int k, T t) { b1[k] = t; });
    }
    if (!sync(c, epoch)) return false;
    // (B1) z_1 = S_1 b_1; every deeper right-hand side as chunk sums
    csr_rows(L1.S, n1, (const T *)b1, wfw, c.nwarps, [&](int i, T t) { z1[i] = t; });
    comp_chunks(C, (const T *)b1, wbw, c.nwarps);
    if (!sync(c, epoch)) return false;
    // (B2) the coarse vector in shared memory, y_1 = z_1 + Q c
    {
      const T *cv = comp_gather(C);
      csr_rows(
          C.Q, n1, cv, wfw, c.nwarps, [&](int i, T t) { y1[i] = t; }, (const T *)z1, cv, C.nc);
    }
    if (!sync(c, epoch)) return false;
    // (C) out = z_0 + P~_0 y_1
    {
      const T *ys = kdev::win_cap() >= n1 ? kdev::win_stage<T>(y1, 0, n1) : nullptr;
      csr_rows(
          L0.P, L0.n, (const T *)y1, wfw, c.nwarps, [&](int i, T t) { out[i] = OT(t); },
          (const T *)z0, ys, ys ? n1 : 0);
    }
    return sync(c, epoch);
  }
  for (int l = 0; l + 1 < L; ++l) {
    const AmgLevelT<T> &Lv = G->lev[l];
    const AmgLevelT<T> &Nx = G->lev[l + 1];
    T *z = Lv.z;
    T *bn = Nx.b;
    if (l == 0) {
      const XT *xs[1] = {b0};
      kdev::spmv_rows<1, T>(c.n, c.q, c.ldn, G->ts0, c.col, G->s0, xs, c.wglobal, c.nwarps,
                            [&](int i, const T *sb) { z[i] = sb[0]; });
      csr_rows(Lv.R, Nx.n, b0, wbw, c.nwarps, [&](int k, T t) { bn[k] = t; });
    } else {
      const T *bl = Lv.b;
      csr_rows(Lv.S, Lv.n, bl, wfw, c.nwarps, [&](int i, T t) { z[i] = t; });
      csr_rows(Lv.R, Nx.n, bl, wbw, c.nwarps, [&](int k, T t) { bn[k] = t; });
    }
    if (!sync(c, epoch)) return false;
  }
  // ---- coarsest
  {
    const AmgLevelT<T> &Cl = G->lev[L - 1];
    coarse_solve(G, Cl.n, Cl.b, Cl.y, c);
    if (!sync(c, epoch)) return false;
  }
  // ---- up
  for (int l = L - 2; l >= 0; --l) {
    const AmgLevelT<T> &Lv = G->lev[l];
    const T *z = Lv.z;
    if (l == 0) {
      // level 1's y is gathered by every row of level 0: staged whole in
      // shared memory when it fits (kdev::win_stage)
      const int n1 = G->lev[1].n;
      const T *ys = kdev::win_cap() >= n1 ? kdev::win_stage<T>(G->lev[1].y, 0, n1) : nullptr;
      csr_rows(
          Lv.P, Lv.n, G->lev[1].y, wfw, c.nwarps, [&](int i, T t) { out[i] = OT(t); }, z, ys,
          ys ? n1 : 0);
    } else {
      T *res = Lv.y;
      csr_rows(
          Lv.P, Lv.n, G->lev[l + 1].y, wfw, c.nwarps, [&](int i, T t) { res[i] = t; }, z);
    }
    if (!sync(c, epoch)) return false;
  }
  return true;
}

}  // namespace amgdev
}  // namespace rbffd
