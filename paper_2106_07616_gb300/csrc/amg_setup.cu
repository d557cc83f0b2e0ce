// amg_setup.cu -- level 0 of the smoothed-aggregation hierarchy (amg.cu)
// built on the device, so that the host part of a build is only the small
// coarse levels.  The same steps and formulas as the host build:
//
//   diagonal, D^-1 and the strength flags of every row (one thread a row);
//   the transposes the later steps walk (strong edges, A^T);
//   rho(D^-1 A) by 12 power steps from the same start;
//   the MIS(2) aggregation with the same priorities and rules
//     (amg.cu: aggregate_mis2), so the aggregates are the host's;
//   P = T - w_P D^-1 A T, A P, A^T P and A_1 = R (A P) by Gustavson rows,
//     one thread a row (a coarse row of A_1: one a segment, then merged):
//     the row's distinct columns in order of first emission in a table of
//     AMG_SETUP_DMAX entries (more: the device build gives up and the host
//     build runs instead);
//   P~ = P - W (A P) and R~ = (P - W A^T P)^T;
//   level 0's S and A in the cycle's type, straight into the operators'
//   allocation.
//
// Every row's sums run in the host's order (A_1's per segment, then over
// the segments in order); products and sums are rounded one by one (no
// fused multiply-add), like the scalar definitions.  The partial sums of
// the power iteration's norms and of A_1's segments run in a fixed order of
// their own, so rho and A_1 may differ from the host's in the last bits.
#include <algorithm>
#include <mutex>
#include <vector>

#include "amg.cuh"
#include "amg_setup.cuh"

namespace rbffd {

namespace {

constexpr int SNT = 256;  // threads per CTA of the row kernels
constexpr int SCAN_NT = 1024;
constexpr int MIS_MAX_ROUNDS = 64;
enum : unsigned char { M_UND = 0, M_ROOT = 1, M_OUT = 2, M_ISO = 3 };

inline int nblk(long long n) { return (int)std::max<long long>(1, (n + SNT - 1) / SNT); }

// ---- stream-ordered scratch, counted against the context's budget
struct Scratch {
  rbffd_ctx *ctx;
  cudaStream_t st;
  std::vector<std::pair<void *, size_t>> held;
  Scratch(rbffd_ctx *c, cudaStream_t s) : ctx(c), st(s) {}
  template <typename T>
  int take(T **p, size_t n) {
    *p = nullptr;
    const size_t bytes = std::max<size_t>(1, n) * sizeof(T);
    if (!dev_reserve(ctx, bytes)) return RBFFD_ENOMEM;
    void *v = nullptr;
    if (cudaMallocAsync(&v, bytes, st) != cudaSuccess) {
      cudaGetLastError();
      dev_release(ctx, bytes);
      set_error("multigrid setup: cudaMallocAsync(%zu) failed", bytes);
      return RBFFD_ENOMEM;
    }
    held.emplace_back(v, bytes);
    *p = (T *)v;
    return RBFFD_OK;
  }
  ~Scratch() {
    for (auto &h : held) {
      cudaFreeAsync(h.first, st);
      dev_release(ctx, h.second);
    }
  }
};

// exclusive scan of in[0 .. m) into out[0 .. m], out[m] = the total (one CTA)
__global__ void k_scan(const int *__restrict__ in, int *__restrict__ out, int m) {
  __shared__ int part[SCAN_NT];
  const int t = threadIdx.x;
  const int per = (m + SCAN_NT - 1) / SCAN_NT;
  const int a = min(m, t * per), b = min(m, a + per);
  int s = 0;
  for (int i = a; i < b; ++i) s += in[i];
  part[t] = s;
  __syncthreads();
  for (int o = 1; o < SCAN_NT; o <<= 1) {
    const int v = t >= o ? part[t - o] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  int run = t > 0 ? part[t - 1] : 0;
  for (int i = a; i < b; ++i) {
    const int v = in[i];
    out[i] = run;
    run += v;
  }
  if (t == SCAN_NT - 1) out[m] = part[SCAN_NT - 1];
}

__device__ __forceinline__ bool kept(double a, int c, int i) { return a != 0.0 || c == i; }

// diagonal, D^-1, strength flags (bit j: slot j of the ELL row), kept
// entries per row, and the column counts of A and of the strong edges
__global__ void k_rows(int n, int q, int ldn, const int32_t *__restrict__ col,
                       const double *__restrict__ val, double theta, double *__restrict__ dinv,
                       unsigned long long *__restrict__ smask, int *__restrict__ kcnt,
                       int *__restrict__ atcnt, int *__restrict__ stcnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double d = 0.0, mx = 0.0;
  int cnt = 0;
  for (int j = 0; j < q; ++j) {
    const size_t e = (size_t)j * ldn + i;
    const int c = col[e];
    const double a = val[e];
    if (!kept(a, c, i)) continue;
    ++cnt;
    atomicAdd(atcnt + c, 1);
    if (c == i)
      d += a;
    else
      mx = fmax(mx, fabs(a));
  }
  unsigned long long m = 0;
  for (int j = 0; j < q; ++j) {
    const size_t e = (size_t)j * ldn + i;
    const int c = col[e];
    const double a = val[e];
    if (kept(a, c, i) && c != i && mx > 0.0 && fabs(a) >= theta * mx) {
      m |= 1ull << j;
      atomicAdd(stcnt + c, 1);
    }
  }
  dinv[i] = d != 0.0 ? 1.0 / d : 0.0;
  smask[i] = m;
  kcnt[i] = cnt;
}

// the kept entries as CSR rows; A^T and the transposed strong edges
// (unordered within a row: k_sort_rows orders them)
__global__ void k_fill_rows(int n, int q, int ldn, const int32_t *__restrict__ col,
                            const double *__restrict__ val,
                            const unsigned long long *__restrict__ smask,
                            const int *__restrict__ kptr, int *__restrict__ kcol,
                            double *__restrict__ kval, const int *__restrict__ atptr,
                            int *__restrict__ atfill, int *__restrict__ atcol,
                            double *__restrict__ atval, const int *__restrict__ stptr,
                            int *__restrict__ stfill, int *__restrict__ stcol) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int k = kptr[i];
  const unsigned long long m = smask[i];
  for (int j = 0; j < q; ++j) {
    const size_t e = (size_t)j * ldn + i;
    const int c = col[e];
    const double a = val[e];
    if (!kept(a, c, i)) continue;
    kcol[k] = c;
    kval[k++] = a;
    const int p = atptr[c] + atomicAdd(atfill + c, 1);
    atcol[p] = i;
    atval[p] = a;
    if ((m >> j) & 1ull) stcol[stptr[c] + atomicAdd(stfill + c, 1)] = i;
  }
}

// every row's entries in increasing column order (insertion sort; rows of
// a transpose hold a few dozen to a few hundred entries)
__global__ void k_sort_rows(int nrows, const int *__restrict__ ptr, int *__restrict__ c,
                            double *__restrict__ v) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrows) return;
  const int a = ptr[r], b = ptr[r + 1];
  for (int k = a + 1; k < b; ++k) {
    const int ck = c[k];
    const double vk = v ? v[k] : 0.0;
    int t = k - 1;
    while (t >= a && c[t] > ck) {
      c[t + 1] = c[t];
      if (v) v[t + 1] = v[t];
      --t;
    }
    c[t + 1] = ck;
    if (v) v[t + 1] = vk;
  }
}

// the same for long rows (the transposes onto the aggregates: hundreds of
// entries), one CTA a row: a bitonic sort in shared memory (keys are the
// distinct source rows); a row beyond its capacity is sorted by one thread
constexpr int SORT_CAP = 2048;
__global__ void k_sort_rows_cta(int nrows, const int *__restrict__ ptr, int *__restrict__ c,
                                double *__restrict__ v) {
  __shared__ int sk[SORT_CAP];
  __shared__ double sv[SORT_CAP];
  const int r = blockIdx.x;
  if (r >= nrows) return;
  const int a = ptr[r], len = ptr[r + 1] - a;
  if (len <= 1) return;
  if (len > SORT_CAP) {
    if (threadIdx.x != 0) return;
    for (int k = a + 1; k < a + len; ++k) {
      const int ck = c[k];
      const double vk = v[k];
      int t = k - 1;
      while (t >= a && c[t] > ck) {
        c[t + 1] = c[t];
        v[t + 1] = v[t];
        --t;
      }
      c[t + 1] = ck;
      v[t + 1] = vk;
    }
    return;
  }
  int p2 = 1;
  while (p2 < len) p2 <<= 1;
  for (int t = threadIdx.x; t < p2; t += blockDim.x) {
    sk[t] = t < len ? c[a + t] : 0x7fffffff;
    sv[t] = t < len ? v[a + t] : 0.0;
  }
  __syncthreads();
  for (int k = 2; k <= p2; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < p2; t += blockDim.x) {
        const int u = t ^ j;
        if (u > t) {
          const bool up = (t & k) == 0;
          if ((sk[t] > sk[u]) == up) {
            const int tk = sk[t];
            sk[t] = sk[u];
            sk[u] = tk;
            const double tv = sv[t];
            sv[t] = sv[u];
            sv[u] = tv;
          }
        }
      }
      __syncthreads();
    }
  for (int t = threadIdx.x; t < len; t += blockDim.x) {
    c[a + t] = sk[t];
    v[a + t] = sv[t];
  }
}

// ---- the strength graph: row i's strong slots and the rows holding i as
// strong (duplicates are harmless to every rule below: maxima and "any")
struct Strong {
  int q, ldn;
  const int32_t *col;
  const unsigned long long *mask;
  const int *tp, *tc;
  template <typename F>
  __device__ __forceinline__ void each(int i, F &&f) const {
    const unsigned long long m = mask[i];
    for (int j = 0; j < q; ++j)
      if ((m >> j) & 1ull) f(col[(size_t)j * ldn + i]);
    for (int k = tp[i]; k < tp[i + 1]; ++k) f(tc[k]);
  }
};

__global__ void k_mis_init(int n, Strong S, unsigned char *__restrict__ st, int *__restrict__ und) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const bool iso = S.mask[i] == 0ull && S.tp[i] == S.tp[i + 1];
  st[i] = iso ? M_ISO : M_UND;
  if (!iso) atomicAdd(und, 1);
}

__global__ void k_mis_m1(int n, Strong S, const unsigned char *__restrict__ st,
                         unsigned long long *__restrict__ m1) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  unsigned long long m = st[i] == M_UND ? mis_key(i) : 0ull;
  S.each(i, [&](int j) {
    if (st[j] == M_UND) m = max(m, (unsigned long long)mis_key(j));
  });
  m1[i] = m;
}

__global__ void k_mis_m2(int n, Strong S, const unsigned char *__restrict__ st,
                         const unsigned long long *__restrict__ m1,
                         unsigned char *__restrict__ nr) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  unsigned long long m = m1[i];
  S.each(i, [&](int j) { m = max(m, m1[j]); });
  nr[i] = st[i] == M_UND && m == mis_key(i);
}

__global__ void k_mis_d1(int n, Strong S, const unsigned char *__restrict__ nr,
                         unsigned char *__restrict__ d1) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  bool d = nr[i];
  S.each(i, [&](int j) { d = d || nr[j]; });
  d1[i] = d;
}

__global__ void k_mis_d2(int n, Strong S, const unsigned char *__restrict__ nr,
                         const unsigned char *__restrict__ d1, unsigned char *__restrict__ st,
                         int *__restrict__ und) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (nr[i]) {
    st[i] = M_ROOT;
  } else if (st[i] == M_UND) {
    bool d = d1[i];
    S.each(i, [&](int j) { d = d || d1[j]; });
    if (d)
      st[i] = M_OUT;
    else
      atomicAdd(und, 1);
  }
}

__global__ void k_flag(int n, const unsigned char *__restrict__ st, unsigned char what,
                       int *__restrict__ flag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) flag[i] = st[i] == what;
}

// the first pass: roots number their aggregates, a point next to roots
// joins the one of largest key
__global__ void k_join1(int n, Strong S, const unsigned char *__restrict__ st,
                        const int *__restrict__ rank, int *__restrict__ a1) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (st[i] == M_ROOT) {
    a1[i] = rank[i];
    return;
  }
  int best = -1;
  if (st[i] == M_OUT)
    S.each(i, [&](int j) {
      if (st[j] == M_ROOT && (best < 0 || mis_key(j) > mis_key(best))) best = j;
    });
  a1[i] = best >= 0 ? rank[best] : -1;
}

// the second pass: a point still without one joins the neighbour of the
// first pass of largest key; left: 1 where nothing was found
__global__ void k_join2(int n, Strong S, const unsigned char *__restrict__ st,
                        const int *__restrict__ a1, int *__restrict__ agg,
                        int *__restrict__ left) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int a = a1[i];
  if (a < 0 && st[i] != M_ISO) {
    int best = -1;
    S.each(i, [&](int j) {
      if (a1[j] >= 0 && (best < 0 || mis_key(j) > mis_key(best))) best = j;
    });
    a = best >= 0 ? a1[best] : -1;
  }
  agg[i] = a;
  left[i] = a < 0;
}

// singletons after the roots, in index order
__global__ void k_join3(int n, int nroots, const int *__restrict__ lrank, int *__restrict__ agg) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && agg[i] < 0) agg[i] = nroots + lrank[i];
}

// ---- rho(D^-1 A): one power step y = D^-1 A x, with block partial sums of
// x^2 and y^2 (a fixed tree per block)
__global__ void k_rho_step(int n, const int *__restrict__ kp, const int *__restrict__ kc,
                           const double *__restrict__ kv, const double *__restrict__ dinv,
                           const double *__restrict__ x, double *__restrict__ y,
                           double *__restrict__ part) {
  __shared__ double sx[SNT], sy[SNT];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double xx = 0.0, yy = 0.0;
  if (i < n) {
    double s = 0.0;
    for (int k = kp[i]; k < kp[i + 1]; ++k) s = __dadd_rn(s, __dmul_rn(kv[k], x[kc[k]]));
    const double yi = __dmul_rn(dinv[i], s);
    y[i] = yi;
    xx = __dmul_rn(x[i], x[i]);
    yy = __dmul_rn(yi, yi);
  }
  sx[threadIdx.x] = xx;
  sy[threadIdx.x] = yy;
  __syncthreads();
  for (int o = SNT / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      sx[threadIdx.x] += sx[threadIdx.x + o];
      sy[threadIdx.x] += sy[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = sx[0];
    part[2 * blockIdx.x + 1] = sy[0];
  }
}

// the norms in block order; sc[0] = lam, sc[1] = 1 / |y|, sc[2] = stopped
__global__ void k_rho_fin(int nb, const double *__restrict__ part, double *__restrict__ sc) {
  if (threadIdx.x != 0 || sc[2] != 0.0) return;
  double nx = 0.0, ny = 0.0;
  for (int b = 0; b < nb; ++b) {
    nx += part[2 * b];
    ny += part[2 * b + 1];
  }
  if (!(ny > 0.0)) {
    sc[2] = 1.0;
  } else {
    sc[0] = sqrt(ny / nx);
    sc[1] = 1.0 / sqrt(ny);
  }
}

__global__ void k_rho_next(int n, const double *__restrict__ y, const double *__restrict__ sc,
                           double *__restrict__ x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && sc[2] == 0.0) x[i] = __dmul_rn(y[i], sc[1]);
}

__global__ void k_rho_start(int n, double *__restrict__ x, double *__restrict__ sc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = rho_start(i);
  if (i == 0) {
    sc[0] = 1.0;
    sc[1] = 1.0;
    sc[2] = 0.0;
  }
}

// w = min(2/3, 4 / (3 lam)) D^-1 (the smoother's) and w_P = 4 / (3 lam)
__global__ void k_weights_w(int n, const double *__restrict__ sc, const double *__restrict__ dinv,
                            double *__restrict__ w, double *__restrict__ om) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const double lam = sc[0];
  const double wp = 4.0 / (3.0 * lam);
  const double os = fmin(AMG_OMEGA, wp);
  if (i < n) w[i] = __dmul_rn(os, dinv[i]);
  if (i == 0) {
    om[0] = os;
    om[1] = wp;
  }
}

// ---- a row's distinct columns in order of first emission, found through
// an open-addressed hash of the column (Fibonacci hashing, linear probing)
constexpr int RT_HBITS = 7;
constexpr int RT_HSZ = 1 << RT_HBITS;  // > AMG_SETUP_DMAX: probes stay short
struct RowTable {
  int c[AMG_SETUP_DMAX];
  double v[AMG_SETUP_DMAX];
  short h[RT_HSZ];
  int m = 0;
  __device__ __forceinline__ RowTable() {
    for (int k = 0; k < RT_HSZ; ++k) h[k] = -1;
  }
  __device__ __forceinline__ bool add(int col, double val) {
    unsigned x = ((unsigned)col * 2654435761u) >> (32 - RT_HBITS);
    for (;;) {
      const int t = h[x];
      if (t < 0) break;
      if (c[t] == col) {
        v[t] = __dadd_rn(v[t], val);
        return true;
      }
      x = (x + 1) & (RT_HSZ - 1);
    }
    if (m == AMG_SETUP_DMAX) return false;
    h[x] = (short)m;
    c[m] = col;
    v[m++] = val;
    return true;
  }
};

// P = T - w_P D^-1 A T: row i emits (agg_i, 1), then (agg_c, -w_P d_i a_ic)
// per entry; exact zeros dropped, order kept.  Count (FILL false) or fill.
template <bool FILL>
__global__ void k_prolong(int n, const int *__restrict__ kp, const int *__restrict__ kc,
                          const double *__restrict__ kv, const int *__restrict__ agg,
                          const double *__restrict__ dinv, const double *__restrict__ om,
                          int *__restrict__ cnt, const int *__restrict__ pp,
                          int *__restrict__ pc, double *__restrict__ pv, int *__restrict__ err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  RowTable t;
  bool ok = t.add(agg[i], 1.0);
  const double f = __dmul_rn(-om[1], dinv[i]);
  for (int k = kp[i]; k < kp[i + 1] && ok; ++k) ok = t.add(agg[kc[k]], __dmul_rn(f, kv[k]));
  if (!ok) {
    atomicOr(err, 1);
    return;
  }
  int o = FILL ? pp[i] : 0, m = 0;
  for (int s = 0; s < t.m; ++s)
    if (t.v[s] != 0.0) {
      if (FILL) {
        pc[o + m] = t.c[s];
        pv[o + m] = t.v[s];
      }
      ++m;
    }
  if (!FILL) cnt[i] = m;
}

// C = L B by rows (Gustavson): row i emits b_rt * l_ir over its entries
template <bool FILL>
__global__ void k_rowprod(int nrows, const int *__restrict__ lp, const int *__restrict__ lc,
                          const double *__restrict__ lv, const int *__restrict__ bp,
                          const int *__restrict__ bc, const double *__restrict__ bv,
                          int *__restrict__ cnt, const int *__restrict__ op, int *__restrict__ oc,
                          double *__restrict__ ov, int *__restrict__ err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nrows) return;
  RowTable t;
  for (int k = lp[i]; k < lp[i + 1]; ++k) {
    const int r = lc[k];
    const double a = lv[k];
    for (int s = bp[r]; s < bp[r + 1]; ++s)
      if (!t.add(bc[s], __dmul_rn(a, bv[s]))) {
        atomicOr(err, 1);
        return;
      }
  }
  if (FILL) {
    const int o = op[i];
    for (int s = 0; s < t.m; ++s) {
      oc[o + s] = t.c[s];
      ov[o + s] = t.v[s];
    }
  } else {
    cnt[i] = t.m;
  }
}

// C = L B for few long rows of L (A_1 = R (A P): a coarse row holds the
// hundreds of fine rows of its aggregate's reach): row i's entries are cut
// into SEG consecutive segments, each gathered into a table of its own
// (k_rowprod_seg), then the tables are merged in segment order
// (k_rowmerge), which keeps the first-emission order of the columns.
constexpr int SEG = 8;
__global__ void k_rowprod_seg(int nrows, const int *__restrict__ lp, const int *__restrict__ lc,
                              const double *__restrict__ lv, const int *__restrict__ bp,
                              const int *__restrict__ bc, const double *__restrict__ bv,
                              int *__restrict__ sm, int *__restrict__ sc, double *__restrict__ sv,
                              int *__restrict__ err) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nrows * SEG) return;
  const int i = g / SEG, sg = g - i * SEG;
  const int a = lp[i], len = lp[i + 1] - a;
  const int k0 = a + (int)((long long)len * sg / SEG), k1 = a + (int)((long long)len * (sg + 1) / SEG);
  RowTable t;
  for (int k = k0; k < k1; ++k) {
    const int r = lc[k];
    const double x = lv[k];
    for (int s2 = bp[r]; s2 < bp[r + 1]; ++s2)
      if (!t.add(bc[s2], __dmul_rn(x, bv[s2]))) {
        atomicOr(err, 1);
        sm[g] = 0;
        return;
      }
  }
  sm[g] = t.m;
  for (int s2 = 0; s2 < t.m; ++s2) {
    sc[(size_t)g * AMG_SETUP_DMAX + s2] = t.c[s2];
    sv[(size_t)g * AMG_SETUP_DMAX + s2] = t.v[s2];
  }
}
template <bool FILL>
__global__ void k_rowmerge(int nrows, const int *__restrict__ sm, const int *__restrict__ sc,
                           const double *__restrict__ sv, int *__restrict__ cnt,
                           const int *__restrict__ op, int *__restrict__ oc,
                           double *__restrict__ ov, int *__restrict__ err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nrows) return;
  RowTable t;
  for (int sg = 0; sg < SEG; ++sg) {
    const size_t g = (size_t)i * SEG + sg;
    for (int s2 = 0; s2 < sm[g]; ++s2)
      if (!t.add(sc[g * AMG_SETUP_DMAX + s2], sv[g * AMG_SETUP_DMAX + s2])) {
        atomicOr(err, 1);
        if (!FILL) cnt[i] = 0;
        return;
      }
  }
  if (FILL) {
    const int o = op[i];
    for (int s2 = 0; s2 < t.m; ++s2) {
      oc[o + s2] = t.c[s2];
      ov[o + s2] = t.v[s2];
    }
  } else {
    cnt[i] = t.m;
  }
}

// out = X - W Y on Y's pattern (rows scaled by w): every entry of X must
// sit in Y's pattern (the diagonal of A is kept), else the device build
// gives up
__global__ void k_minus_scaled(int n, const int *__restrict__ yp, const int *__restrict__ yc,
                               const double *__restrict__ yv, const int *__restrict__ xp,
                               const int *__restrict__ xc, const double *__restrict__ xv,
                               const double *__restrict__ w, double *__restrict__ out,
                               int *__restrict__ err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double wi = w[i];
  for (int k = yp[i]; k < yp[i + 1]; ++k) out[k] = __dmul_rn(-wi, yv[k]);
  for (int k = xp[i]; k < xp[i + 1]; ++k) {
    int p = -1;
    for (int s = yp[i]; s < yp[i + 1] && p < 0; ++s)
      if (yc[s] == xc[k]) p = s;
    if (p < 0) {
      atomicOr(err, 2);
      return;
    }
    out[p] = __dadd_rn(out[p], xv[k]);
  }
}

// transpose: column counts, then unordered fill (k_sort_rows orders)
__global__ void k_tcount(int nrows, const int *__restrict__ p, const int *__restrict__ c,
                         int *__restrict__ cnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nrows) return;
  for (int k = p[i]; k < p[i + 1]; ++k) atomicAdd(cnt + c[k], 1);
}
__global__ void k_tfill(int nrows, const int *__restrict__ p, const int *__restrict__ c,
                        const double *__restrict__ v, const int *__restrict__ tp,
                        int *__restrict__ tfill, int *__restrict__ tc, double *__restrict__ tv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nrows) return;
  for (int k = p[i]; k < p[i + 1]; ++k) {
    const int at = tp[c[k]] + atomicAdd(tfill + c[k], 1);
    tc[at] = i;
    tv[at] = v[k];
  }
}

// level 0's S = 2 W - W A W in the ELL layout (every slot, the first
// diagonal slot adds 2 w_i) and A in the cycle's FP32, if asked
template <typename T>
__global__ void k_level0_ell(int n, int q, int ldn, const int32_t *__restrict__ col,
                             const double *__restrict__ val, const double *__restrict__ w,
                             T *__restrict__ s0, float *__restrict__ a0) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double wi = w[i];
  bool diag = false;
  for (int j = 0; j < q; ++j) {
    const size_t e = (size_t)j * ldn + i;
    const int c = col[e];
    double v = __dmul_rn(__dmul_rn(-wi, val[e]), w[c]);
    if (c == i && !diag) {
      v = __dadd_rn(v, __dmul_rn(2.0, wi));
      diag = true;
    }
    s0[e] = (T)v;
    if (a0) a0[e] = (float)val[e];
  }
}

template <typename T>
__global__ void k_to_type(long long m, const double *__restrict__ in, T *__restrict__ out) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < m) out[k] = (T)in[k];
}

__global__ void k_maxlen(int nrows, const int *__restrict__ p, int *__restrict__ mx) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nrows) atomicMax(mx, p[i + 1] - p[i]);
}

#define SETUP_LAUNCH(what)                                                   \
  do {                                                                       \
    const cudaError_t e_ = cudaGetLastError();                               \
    if (e_ != cudaSuccess) {                                                 \
      set_error("multigrid setup: %s: %s", what, cudaGetErrorString(e_));    \
      return RBFFD_ECUDA;                                                    \
    }                                                                        \
  } while (0)

}  // namespace

// The scratch of a build comes from the device's stream-ordered pool; the
// pool keeps up to 4 GB it gets back instead of returning it at every
// synchronisation, so a rebuild reuses the previous build's memory (a
// setting of this process only).
void keep_pool(int device) {
  static std::once_flag once[64];
  if (device < 0 || device >= 64) return;
  std::call_once(once[device], [device] {
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
      uint64_t thr = 4ull << 30;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
  });
}

template <typename T>
int amg_level0_device(rbffd_ctx *ctx, cudaStream_t st, int n, int q, int ldn,
                      const int32_t *col, const double *val, bool low, AmgL0 *out) {
  if (q > 64 || n < 1) return RBFFD_ENOTIMPL;
  keep_pool(ctx->device);
  Scratch S(ctx, st);
  const long long nq = (long long)n * q;
  // ---- rows, strength, transposes
  double *dinv, *w, *x, *y, *part, *sc, *om;
  unsigned long long *smask, *m1;
  int *kcnt, *kptr, *kcol, *atcnt, *atptr, *atfill, *atcol, *stcnt, *stptr, *stfill, *stcol;
  double *kval, *atval;
  int *misc;  // [0] error bits, [1..MIS_MAX_ROUNDS] undecided counts, maxima
  const int nb = nblk(n);
  RBFFD_TRY(S.take(&dinv, n));
  RBFFD_TRY(S.take(&w, n));
  RBFFD_TRY(S.take(&x, n));
  RBFFD_TRY(S.take(&y, n));
  RBFFD_TRY(S.take(&part, 2 * nb));
  RBFFD_TRY(S.take(&sc, 3));
  RBFFD_TRY(S.take(&om, 2));
  RBFFD_TRY(S.take(&smask, n));
  RBFFD_TRY(S.take(&m1, n));
  RBFFD_TRY(S.take(&kcnt, n + 1));
  RBFFD_TRY(S.take(&kptr, n + 1));
  RBFFD_TRY(S.take(&kcol, nq));
  RBFFD_TRY(S.take(&kval, nq));
  RBFFD_TRY(S.take(&atcnt, n + 1));
  RBFFD_TRY(S.take(&atptr, n + 1));
  RBFFD_TRY(S.take(&atfill, n));
  RBFFD_TRY(S.take(&atcol, nq));
  RBFFD_TRY(S.take(&atval, nq));
  RBFFD_TRY(S.take(&stcnt, n + 1));
  RBFFD_TRY(S.take(&stptr, n + 1));
  RBFFD_TRY(S.take(&stfill, n));
  RBFFD_TRY(S.take(&stcol, nq));
  constexpr int MISC = 8 + MIS_MAX_ROUNDS;
  RBFFD_TRY(S.take(&misc, MISC));
  int *err = misc, *undc = misc + 8;
  RBFFD_CK(cudaMemsetAsync(misc, 0, sizeof(int) * MISC, st));
  RBFFD_CK(cudaMemsetAsync(atcnt, 0, sizeof(int) * (n + 1), st));
  RBFFD_CK(cudaMemsetAsync(stcnt, 0, sizeof(int) * (n + 1), st));
  RBFFD_CK(cudaMemsetAsync(atfill, 0, sizeof(int) * n, st));
  RBFFD_CK(cudaMemsetAsync(stfill, 0, sizeof(int) * n, st));
  k_rows<<<nb, SNT, 0, st>>>(n, q, ldn, col, val, AMG_THETA, dinv, smask, kcnt, atcnt, stcnt);
  SETUP_LAUNCH("k_rows");
  k_scan<<<1, SCAN_NT, 0, st>>>(kcnt, kptr, n);
  k_scan<<<1, SCAN_NT, 0, st>>>(atcnt, atptr, n);
  k_scan<<<1, SCAN_NT, 0, st>>>(stcnt, stptr, n);
  SETUP_LAUNCH("k_scan");
  k_fill_rows<<<nb, SNT, 0, st>>>(n, q, ldn, col, val, smask, kptr, kcol, kval, atptr, atfill,
                                   atcol, atval, stptr, stfill, stcol);
  k_sort_rows<<<nb, SNT, 0, st>>>(n, atptr, atcol, atval);
  k_sort_rows<<<nb, SNT, 0, st>>>(n, stptr, stcol, nullptr);
  SETUP_LAUNCH("k_fill_rows");
  // ---- rho and the weights
  k_rho_start<<<nb, SNT, 0, st>>>(n, x, sc);
  for (int it = 0; it < 12; ++it) {
    k_rho_step<<<nb, SNT, 0, st>>>(n, kptr, kcol, kval, dinv, x, y, part);
    k_rho_fin<<<1, 32, 0, st>>>(nb, part, sc);
    k_rho_next<<<nb, SNT, 0, st>>>(n, y, sc, x);
  }
  k_weights_w<<<nb, SNT, 0, st>>>(n, sc, dinv, w, om);
  SETUP_LAUNCH("rho");
  // ---- MIS(2) aggregation
  const Strong G{q, ldn, col, smask, stptr, stcol};
  unsigned char *mst, *nr, *d1;
  int *flag, *rank, *a1, *agg;
  RBFFD_TRY(S.take(&mst, n));
  RBFFD_TRY(S.take(&nr, n));
  RBFFD_TRY(S.take(&d1, n));
  RBFFD_TRY(S.take(&flag, n + 1));
  RBFFD_TRY(S.take(&rank, n + 1));
  RBFFD_TRY(S.take(&a1, n));
  RBFFD_TRY(S.take(&agg, n));
  k_mis_init<<<nb, SNT, 0, st>>>(n, G, mst, undc);
  SETUP_LAUNCH("k_mis_init");
  int und = 0;
  RBFFD_CK(cudaMemcpyAsync(&und, undc, sizeof(int), cudaMemcpyDeviceToHost, st));
  RBFFD_CK(cudaStreamSynchronize(st));
  for (int r = 1; und > 0; ++r) {
    if (r >= MIS_MAX_ROUNDS) return RBFFD_ENOTIMPL;
    k_mis_m1<<<nb, SNT, 0, st>>>(n, G, mst, m1);
    k_mis_m2<<<nb, SNT, 0, st>>>(n, G, mst, m1, nr);
    k_mis_d1<<<nb, SNT, 0, st>>>(n, G, nr, d1);
    k_mis_d2<<<nb, SNT, 0, st>>>(n, G, nr, d1, mst, undc + r);
    SETUP_LAUNCH("MIS(2) round");
    RBFFD_CK(cudaMemcpyAsync(&und, undc + r, sizeof(int), cudaMemcpyDeviceToHost, st));
    RBFFD_CK(cudaStreamSynchronize(st));
  }
  k_flag<<<nb, SNT, 0, st>>>(n, mst, M_ROOT, flag);
  k_scan<<<1, SCAN_NT, 0, st>>>(flag, rank, n);
  k_join1<<<nb, SNT, 0, st>>>(n, G, mst, rank, a1);
  k_join2<<<nb, SNT, 0, st>>>(n, G, mst, a1, agg, flag);
  SETUP_LAUNCH("aggregation");
  int nroots = 0;
  RBFFD_CK(cudaMemcpyAsync(&nroots, rank + n, sizeof(int), cudaMemcpyDeviceToHost, st));
  int *lrank = kcnt;  // free again (kptr holds the scan)
  k_scan<<<1, SCAN_NT, 0, st>>>(flag, lrank, n);
  int nleft = 0;
  RBFFD_CK(cudaMemcpyAsync(&nleft, lrank + n, sizeof(int), cudaMemcpyDeviceToHost, st));
  RBFFD_CK(cudaStreamSynchronize(st));
  k_join3<<<nb, SNT, 0, st>>>(n, nroots, lrank, agg);
  SETUP_LAUNCH("k_join3");
  const int n1 = nroots + nleft;
  if (n1 == 0 || n1 > 0.8 * n) return RBFFD_ENOTIMPL;  // coarsening stalled: the host decides
  // ---- P, A P, A^T P (count, scan, fill)
  const long long pmax = (long long)n * (q + 1);
  int *pcnt, *pptr, *pc, *apcnt, *apptr, *atpcnt, *atpptr;
  double *pv;
  RBFFD_TRY(S.take(&pcnt, n + 1));
  RBFFD_TRY(S.take(&pptr, n + 1));
  RBFFD_TRY(S.take(&pc, pmax));
  RBFFD_TRY(S.take(&pv, pmax));
  RBFFD_TRY(S.take(&apcnt, n + 1));
  RBFFD_TRY(S.take(&apptr, n + 1));
  RBFFD_TRY(S.take(&atpcnt, n + 1));
  RBFFD_TRY(S.take(&atpptr, n + 1));
  k_prolong<false><<<nb, SNT, 0, st>>>(n, kptr, kcol, kval, agg, dinv, om, pcnt, nullptr,
                                        nullptr, nullptr, err);
  k_scan<<<1, SCAN_NT, 0, st>>>(pcnt, pptr, n);
  k_prolong<true><<<nb, SNT, 0, st>>>(n, kptr, kcol, kval, agg, dinv, om, nullptr, pptr, pc,
                                       pv, err);
  k_rowprod<false><<<nb, SNT, 0, st>>>(n, kptr, kcol, kval, pptr, pc, pv, apcnt, nullptr,
                                        nullptr, nullptr, err);
  k_rowprod<false><<<nb, SNT, 0, st>>>(n, atptr, atcol, atval, pptr, pc, pv, atpcnt, nullptr,
                                        nullptr, nullptr, err);
  k_scan<<<1, SCAN_NT, 0, st>>>(apcnt, apptr, n);
  k_scan<<<1, SCAN_NT, 0, st>>>(atpcnt, atpptr, n);
  SETUP_LAUNCH("P and the product counts");
  int tot[3] = {0, 0, 0}, e0 = 0;
  RBFFD_CK(cudaMemcpyAsync(&tot[0], apptr + n, sizeof(int), cudaMemcpyDeviceToHost, st));
  RBFFD_CK(cudaMemcpyAsync(&tot[1], atpptr + n, sizeof(int), cudaMemcpyDeviceToHost, st));
  RBFFD_CK(cudaMemcpyAsync(&tot[2], pptr + n, sizeof(int), cudaMemcpyDeviceToHost, st));
  RBFFD_CK(cudaMemcpyAsync(&e0, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  RBFFD_CK(cudaStreamSynchronize(st));
  if (e0) return RBFFD_ENOTIMPL;
  const int nap = tot[0], natp = tot[1], np = tot[2];
  int *apc, *atpc, *rtp, *rtfill, *rtc, *rp, *rfill, *rc;
  double *apv, *ptv, *atpv, *rttv, *rtv, *rv;
  RBFFD_TRY(S.take(&apc, nap));
  RBFFD_TRY(S.take(&apv, nap));
  RBFFD_TRY(S.take(&ptv, nap));
  RBFFD_TRY(S.take(&atpc, natp));
  RBFFD_TRY(S.take(&atpv, natp));
  RBFFD_TRY(S.take(&rttv, natp));
  RBFFD_TRY(S.take(&rtp, n1 + 1));
  RBFFD_TRY(S.take(&rtfill, n1));
  RBFFD_TRY(S.take(&rtc, natp));
  RBFFD_TRY(S.take(&rtv, natp));
  RBFFD_TRY(S.take(&rp, n1 + 1));
  RBFFD_TRY(S.take(&rfill, n1));
  RBFFD_TRY(S.take(&rc, np));
  RBFFD_TRY(S.take(&rv, np));
  k_rowprod<true><<<nb, SNT, 0, st>>>(n, kptr, kcol, kval, pptr, pc, pv, nullptr, apptr, apc,
                                       apv, err);
  k_rowprod<true><<<nb, SNT, 0, st>>>(n, atptr, atcol, atval, pptr, pc, pv, nullptr, atpptr,
                                       atpc, atpv, err);
  // P~ = P - W (A P) and R~^T = P - W (A^T P) on their products' patterns
  k_minus_scaled<<<nb, SNT, 0, st>>>(n, apptr, apc, apv, pptr, pc, pv, w, ptv, err);
  k_minus_scaled<<<nb, SNT, 0, st>>>(n, atpptr, atpc, atpv, pptr, pc, pv, w, rttv, err);
  SETUP_LAUNCH("products");
  // R~ = (R~^T)^T and R = P^T, rows in increasing fine index
  const int nb1 = nblk(n1);
  int *cnt1 = rtfill;  // counts, then reused as fill cursors
  RBFFD_CK(cudaMemsetAsync(cnt1, 0, sizeof(int) * n1, st));
  k_tcount<<<nb, SNT, 0, st>>>(n, atpptr, atpc, cnt1);
  k_scan<<<1, SCAN_NT, 0, st>>>(cnt1, rtp, n1);
  RBFFD_CK(cudaMemsetAsync(rtfill, 0, sizeof(int) * n1, st));
  k_tfill<<<nb, SNT, 0, st>>>(n, atpptr, atpc, rttv, rtp, rtfill, rtc, rtv);
  k_sort_rows_cta<<<n1, SNT, 0, st>>>(n1, rtp, rtc, rtv);
  RBFFD_CK(cudaMemsetAsync(rfill, 0, sizeof(int) * n1, st));
  k_tcount<<<nb, SNT, 0, st>>>(n, pptr, pc, rfill);
  k_scan<<<1, SCAN_NT, 0, st>>>(rfill, rp, n1);
  RBFFD_CK(cudaMemsetAsync(rfill, 0, sizeof(int) * n1, st));
  k_tfill<<<nb, SNT, 0, st>>>(n, pptr, pc, pv, rp, rfill, rc, rv);
  k_sort_rows_cta<<<n1, SNT, 0, st>>>(n1, rp, rc, rv);
  SETUP_LAUNCH("transposes");
  // A_1 = R (A P), each coarse row in SEG segments
  int *accnt, *acptr, *segm, *segc;
  double *segv;
  RBFFD_TRY(S.take(&accnt, n1 + 1));
  RBFFD_TRY(S.take(&acptr, n1 + 1));
  RBFFD_TRY(S.take(&segm, (size_t)n1 * SEG));
  RBFFD_TRY(S.take(&segc, (size_t)n1 * SEG * AMG_SETUP_DMAX));
  RBFFD_TRY(S.take(&segv, (size_t)n1 * SEG * AMG_SETUP_DMAX));
  k_rowprod_seg<<<nblk((long long)n1 * SEG), SNT, 0, st>>>(n1, rp, rc, rv, apptr, apc, apv, segm,
                                                           segc, segv, err);
  k_rowmerge<false><<<nb1, SNT, 0, st>>>(n1, segm, segc, segv, accnt, nullptr, nullptr, nullptr,
                                          err);
  k_scan<<<1, SCAN_NT, 0, st>>>(accnt, acptr, n1);
  SETUP_LAUNCH("A_1 count");
  int nac = 0;
  RBFFD_CK(cudaMemcpyAsync(&nac, acptr + n1, sizeof(int), cudaMemcpyDeviceToHost, st));
  RBFFD_CK(cudaMemcpyAsync(&e0, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  RBFFD_CK(cudaStreamSynchronize(st));
  if (e0) return RBFFD_ENOTIMPL;
  int *acc;
  double *acv;
  RBFFD_TRY(S.take(&acc, nac));
  RBFFD_TRY(S.take(&acv, nac));
  k_rowmerge<true><<<nb1, SNT, 0, st>>>(n1, segm, segc, segv, nullptr, acptr, acc, acv, err);
  SETUP_LAUNCH("A_1");

  // ---- level 0's operators in the cycle's type, one allocation
  AmgL0 &o = *out;
  o.n1 = n1;
  o.nnz_a = 0;
  o.nnz_r = natp;
  o.nnz_p = nap;
  size_t at = 0;
  auto place = [&](size_t bytes) {
    const size_t p = at;
    at += (bytes + 255) / 256 * 256;
    return p;
  };
  o.o_s0 = place(sizeof(T) * (size_t)q * ldn);
  o.o_a0 = low ? place(sizeof(float) * (size_t)q * ldn) : 0;
  o.o_rp = place(sizeof(int) * (n1 + 1));
  o.o_rc = place(sizeof(int) * (size_t)natp);
  o.o_rv = place(sizeof(T) * (size_t)natp);
  o.o_pp = place(sizeof(int) * (n + 1));
  o.o_pc = place(sizeof(int) * (size_t)nap);
  o.o_pv = place(sizeof(T) * (size_t)nap);
  o.o_z = place(sizeof(T) * n);
  o.o_y = place(sizeof(T) * n);
  o.bytes = at;
  RBFFD_TRY(dev_alloc(ctx, &o.mem, o.bytes));
  char *b = (char *)o.mem;
  RBFFD_CK(cudaMemsetAsync(b + o.o_s0, 0, sizeof(T) * (size_t)q * ldn, st));
  if (low) RBFFD_CK(cudaMemsetAsync(b + o.o_a0, 0, sizeof(float) * (size_t)q * ldn, st));
  k_level0_ell<T><<<nb, SNT, 0, st>>>(n, q, ldn, col, val, w, (T *)(b + o.o_s0),
                                      low ? (float *)(b + o.o_a0) : nullptr);
  RBFFD_CK(cudaMemcpyAsync(b + o.o_rp, rtp, sizeof(int) * (n1 + 1), cudaMemcpyDeviceToDevice, st));
  RBFFD_CK(cudaMemcpyAsync(b + o.o_rc, rtc, sizeof(int) * (size_t)natp, cudaMemcpyDeviceToDevice,
                           st));
  k_to_type<T><<<nblk(natp), SNT, 0, st>>>(natp, rtv, (T *)(b + o.o_rv));
  RBFFD_CK(cudaMemcpyAsync(b + o.o_pp, apptr, sizeof(int) * (n + 1), cudaMemcpyDeviceToDevice, st));
  RBFFD_CK(cudaMemcpyAsync(b + o.o_pc, apc, sizeof(int) * (size_t)nap, cudaMemcpyDeviceToDevice,
                           st));
  k_to_type<T><<<nblk(nap), SNT, 0, st>>>(nap, ptv, (T *)(b + o.o_pv));
  int *mx = misc + 2;
  k_maxlen<<<nb1, SNT, 0, st>>>(n1, rtp, mx);
  k_maxlen<<<nb, SNT, 0, st>>>(n, apptr, mx + 1);
  SETUP_LAUNCH("level 0 operators");
  // ---- A_1 and the scalars to the host
  o.a1ptr.resize(n1 + 1);
  o.a1col.resize(nac);
  o.a1val.resize(nac);
  double hs[3], hom[2];
  int hm[2], hk = 0;
  RBFFD_CK(cudaMemcpyAsync(o.a1ptr.data(), acptr, sizeof(int) * (n1 + 1), cudaMemcpyDeviceToHost,
                           st));
  RBFFD_CK(cudaMemcpyAsync(o.a1col.data(), acc, sizeof(int) * (size_t)nac, cudaMemcpyDeviceToHost,
                           st));
  RBFFD_CK(cudaMemcpyAsync(o.a1val.data(), acv, sizeof(double) * (size_t)nac,
                           cudaMemcpyDeviceToHost, st));
  RBFFD_CK(cudaMemcpyAsync(hs, sc, sizeof(hs), cudaMemcpyDeviceToHost, st));
  RBFFD_CK(cudaMemcpyAsync(hom, om, sizeof(hom), cudaMemcpyDeviceToHost, st));
  RBFFD_CK(cudaMemcpyAsync(hm, mx, sizeof(hm), cudaMemcpyDeviceToHost, st));
  RBFFD_CK(cudaMemcpyAsync(&e0, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  RBFFD_CK(cudaMemcpyAsync(&hk, kptr + n, sizeof(int), cudaMemcpyDeviceToHost, st));
  RBFFD_CK(cudaStreamSynchronize(st));
  if (e0) {
    dev_free(ctx, o.mem, o.bytes);
    o.mem = nullptr;
    return RBFFD_ENOTIMPL;
  }
  o.lam = hs[0];
  o.omega = hom[0];
  o.maxlen_r = hm[0];
  o.maxlen_p = hm[1];
  o.nnz_a = hk;
  return RBFFD_OK;
}

template int amg_level0_device<double>(rbffd_ctx *, cudaStream_t, int, int, int,
                                       const int32_t *, const double *, bool, AmgL0 *);
template int amg_level0_device<float>(rbffd_ctx *, cudaStream_t, int, int, int,
                                      const int32_t *, const double *, bool, AmgL0 *);

}  // namespace rbffd
