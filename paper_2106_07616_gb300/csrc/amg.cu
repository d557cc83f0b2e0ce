// amg.cu -- host construction of the smoothed-aggregation hierarchy of the
// pressure-correction matrix (see amg.cuh), then one upload.
//
// Per level l (A_0 = the p' matrix):
//   strength  i ~ j  if |a_ij| >= theta * max_{k != i} |a_ik|, symmetrised;
//   aggregates: on level 0 a distance-2 maximal independent set of roots
//     (aggregate_mis2); on the coarser levels greedy in index order -- a
//     point whose strong neighbours are all free roots a new aggregate with
//     them; leftovers join the aggregate of a strong neighbour; what is
//     still free becomes a singleton;
//   tentative prolongation T (one 1 per row, in the point's aggregate);
//   smoothed prolongation P = (I - w_P D^-1 A) T, w_P = 4 / (3 rho(D^-1 A))
//     (rho by power iteration);
//   R = P^T, A_{l+1} = R (A P) (Gustavson sparse products);
//   the fused V-cycle operators S, R~, P~ of amg.cuh;
// until at most AMG_NCOARSE rows remain, whose matrix is inverted densely.
// Everything is deterministic: fixed start vectors, index-ordered loops;
// the sparse products run over rows in parallel (OpenMP) with per-thread
// accumulators, each row's result independent of the thread count.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <cstdio>
#include <memory>
#include <thread>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "abi_guard.cuh"
#include "amg.cuh"
#include "amg_job.cuh"
#include "amg_setup.cuh"
#include "krylov_dev.cuh"

namespace rbffd {

namespace {

constexpr int AMG_NCOARSE = 64;     // coarsest level solved by a dense inverse
constexpr int AMG_NCOARSE_MAX = 600;

// Work (entries a loop touches) below which it runs on the calling thread
// alone: an OpenMP fork and join costs tens of microseconds on a 16-core
// host, more than a coarse level's whole loop.
constexpr long long AMG_PAR_WORK = 1 << 17;
inline bool par(long long work) { return work >= AMG_PAR_WORK; }

struct Csr {
  int n = 0, m = 0;  // rows, columns
  std::vector<int32_t> ptr, col;
  std::vector<double> val;
  long long nnz() const { return (long long)col.size(); }
};

Csr from_ell(int n, int q, int ldn, const std::vector<int32_t> &col,
             const std::vector<double> &val) {
  Csr A;
  A.n = A.m = n;
  A.ptr.assign(n + 1, 0);
  auto kept = [&](int i, int j) {  // identity rows store zero weights
    const size_t e = (size_t)j * ldn + i;
    return val[e] != 0.0 || col[e] == i;
  };
  const bool pa = par((long long)n * q);
#pragma omp parallel for schedule(static) if (pa)
  for (int i = 0; i < n; ++i) {
    int c = 0;
    for (int j = 0; j < q; ++j) c += kept(i, j);
    A.ptr[i + 1] = c;
  }
  for (int i = 0; i < n; ++i) A.ptr[i + 1] += A.ptr[i];
  A.col.resize(A.ptr[n]);
  A.val.resize(A.ptr[n]);
#pragma omp parallel for schedule(static) if (pa)
  for (int i = 0; i < n; ++i) {
    int k = A.ptr[i];
    for (int j = 0; j < q; ++j)
      if (kept(i, j)) {
        const size_t e = (size_t)j * ldn + i;
        A.col[k] = col[e];
        A.val[k++] = val[e];
      }
  }
  return A;
}

std::vector<double> diagonal(const Csr &A) {
  std::vector<double> d(A.n, 0.0);
#pragma omp parallel for schedule(static) if (par(A.nnz()))
  for (int i = 0; i < A.n; ++i)
    for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k)
      if (A.col[k] == i) d[i] += A.val[k];
  return d;
}

// Rows per dynamically scheduled chunk: about 16 chunks a thread, at most
// 256 rows (the coarse-row products R A and R A P have a few thousand heavy
// rows, which fixed large chunks leave to a few threads).
int row_chunk(int n) {
  const int c = n / (16 * std::max(1, omp_get_max_threads()));
  return std::max(1, std::min(256, c));
}

// A CSR matrix whose row i is produced by row(i, mark, emit): `mark` is a
// per-thread int array of m entries (the row index marks a column as seen),
// emit(c, v) adds v at column c.  Two parallel passes -- sizes, then values
// into place -- so no per-row allocation; column order = first emission.
// `work`: about how many emissions the rows make (threads or not).
template <typename RowFn>
Csr build_rows(int n, int m, long long work, RowFn &&row) {
  Csr C;
  C.n = n;
  C.m = m;
  C.ptr.assign(n + 1, 0);
  const int chunk = row_chunk(n);
  const bool pa = par(work);
#pragma omp parallel if (pa)
  {
    std::vector<int32_t> mark(m, -1);
#pragma omp for schedule(dynamic, chunk)
    for (int i = 0; i < n; ++i) {
      int cnt = 0;
      row(i, mark, [&](int c, double) {
        if (mark[c] != i) {
          mark[c] = i;
          ++cnt;
        }
      });
      C.ptr[i + 1] = cnt;
    }
  }
  for (int i = 0; i < n; ++i) C.ptr[i + 1] += C.ptr[i];
  C.col.resize(C.ptr[n]);
  C.val.resize(C.ptr[n]);
#pragma omp parallel if (pa)
  {
    std::vector<int32_t> mark(m, -1), where(m, 0);
#pragma omp for schedule(dynamic, chunk)
    for (int i = 0; i < n; ++i) {
      int o = C.ptr[i];
      row(i, mark, [&](int c, double v) {
        if (mark[c] != i) {
          mark[c] = i;
          where[c] = o;
          C.col[o] = c;
          C.val[o++] = v;
        } else {
          C.val[where[c]] += v;
        }
      });
    }
  }
  return C;
}

// A^T with the rows of each column in increasing order.  Threads take
// contiguous row ranges in order, count their columns, and place their
// entries after those of the ranges before them: the same result as one
// pass over the rows.
Csr transpose(const Csr &A) {
  Csr T;
  T.n = A.m;
  T.m = A.n;
  T.ptr.assign(A.m + 1, 0);
  T.col.resize(A.col.size());
  T.val.resize(A.val.size());
  const int nt = par(A.nnz()) ? std::max(1, omp_get_max_threads()) : 1;
  const size_t m1 = (size_t)A.m + 1;
  std::vector<int32_t> at((size_t)nt * m1, 0);  // per range: count, then start, per column
  auto range = [&](int t, int &lo, int &hi) {
    lo = (int)((long long)A.n * t / nt);
    hi = (int)((long long)A.n * (t + 1) / nt);
  };
#pragma omp parallel for num_threads(nt) schedule(static, 1)
  for (int t = 0; t < nt; ++t) {
    int lo, hi;
    range(t, lo, hi);
    int32_t *cnt = at.data() + (size_t)t * m1;
    for (int k = A.ptr[lo]; k < A.ptr[hi]; ++k) cnt[A.col[k]]++;
  }
  for (int c = 0; c < A.m; ++c) {
    int32_t s = T.ptr[c];
    for (int t = 0; t < nt; ++t) {
      int32_t &x = at[(size_t)t * m1 + c];
      const int32_t k = x;
      x = s;
      s += k;
    }
    T.ptr[c + 1] = s;
  }
#pragma omp parallel for num_threads(nt) schedule(static, 1)
  for (int t = 0; t < nt; ++t) {
    int lo, hi;
    range(t, lo, hi);
    int32_t *fill = at.data() + (size_t)t * m1;
    for (int i = lo; i < hi; ++i)
      for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k) {
        const int f = fill[A.col[k]]++;
        T.col[f] = i;
        T.val[f] = A.val[k];
      }
  }
  return T;
}

// |lambda|max of D^-1 A by 12 power steps from a fixed non-constant start.
// Norms are summed per fixed chunk of rows, then over the chunks in order,
// so the estimate does not depend on the thread count.
double rho_estimate(const Csr &A, const std::vector<double> &dinv) {
  constexpr int CHUNK = 4096;
  const int nch = (A.n + CHUNK - 1) / CHUNK;
  std::vector<double> x(A.n), y(A.n), px(nch), py(nch);
  for (int i = 0; i < A.n; ++i) x[i] = rho_start(i);
  double lam = 1.0, sc = 1.0;
  bool stop = false;
  // one parallel region for all the steps (a fork per step costs more
  // than a coarse level's product); the norms are summed by one thread
#pragma omp parallel if (par(A.nnz()))
  for (int it = 0; it < 12; ++it) {
#pragma omp for schedule(static)
    for (int c = 0; c < nch; ++c) {
      double sx = 0.0, sy = 0.0;
      const int e = std::min(A.n, (c + 1) * CHUNK);
      for (int i = c * CHUNK; i < e; ++i) {
        double s = 0.0;
        for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k) s += A.val[k] * x[A.col[k]];
        y[i] = dinv[i] * s;
        sx += x[i] * x[i];
        sy += y[i] * y[i];
      }
      px[c] = sx;
      py[c] = sy;
    }
#pragma omp single
    {
      double nx = 0.0, ny = 0.0;
      for (int c = 0; c < nch; ++c) {
        nx += px[c];
        ny += py[c];
      }
      if (!(ny > 0.0)) {
        stop = true;
      } else {
        lam = std::sqrt(ny / nx);
        sc = 1.0 / std::sqrt(ny);
      }
    }
    if (stop) break;
#pragma omp for schedule(static)
    for (int i = 0; i < A.n; ++i) x[i] = y[i] * sc;
  }
  return lam;
}

// symmetric strength graph as adjacency lists: row i's strong columns in
// stored order, then the rows that hold i as strong and are not yet listed
void strength(const Csr &A, double theta, std::vector<int32_t> &sp, std::vector<int32_t> &sc) {
  const int n = A.n;
  std::vector<char> st(A.nnz(), 0);
  std::vector<int32_t> cnt(n + 1, 0);
  const bool pa = par(A.nnz());
#pragma omp parallel for schedule(static) if (pa)
  for (int i = 0; i < n; ++i) {
    double mx = 0.0;
    for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k)
      if (A.col[k] != i) mx = std::max(mx, std::fabs(A.val[k]));
    int c = 0;
    for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k) {
      st[k] = A.col[k] != i && mx > 0.0 && std::fabs(A.val[k]) >= theta * mx;
      c += st[k];
    }
    cnt[i + 1] = c;
  }
  // strong matrix S1 and its transpose
  Csr S1;
  S1.n = S1.m = n;
  S1.ptr = cnt;
  for (int i = 0; i < n; ++i) S1.ptr[i + 1] += S1.ptr[i];
  S1.col.resize(S1.ptr[n]);
  S1.val.assign(S1.ptr[n], 1.0);
#pragma omp parallel for schedule(static) if (pa)
  for (int i = 0; i < n; ++i) {
    int w = S1.ptr[i];
    for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k)
      if (st[k]) S1.col[w++] = A.col[k];
  }
  const Csr S1T = transpose(S1);
  Csr U = build_rows(n, n, 2 * S1.nnz(), [&](int i, std::vector<int32_t> &, auto &&emit) {
    for (int k = S1.ptr[i]; k < S1.ptr[i + 1]; ++k) emit(S1.col[k], 1.0);
    for (int k = S1T.ptr[i]; k < S1T.ptr[i + 1]; ++k) emit(S1T.col[k], 1.0);
  });
  sp = std::move(U.ptr);
  sc = std::move(U.col);
}

// ---- level 0's aggregation: a distance-2 maximal independent set of the
// strength graph as aggregate roots (the MIS(2) aggregation of Bell, Dalton
// and Olson 2012), with fixed pseudo-random priorities so that the rounds
// run in parallel and give the same aggregates on the host and the device.
// key(i) = (h(i) << 32 | i) + 1, h the 32-bit finaliser of MurmurHash3
// (Appleby); 0 means "none".  Per round: every undecided point whose key is
// the largest among the undecided points within distance 2 becomes a root;
// the undecided points within distance 2 of a new root are out.  Then the
// roots number their aggregates in index order; a point next to roots joins
// the one of largest key; a point still without an aggregate joins the
// neighbour (of the first pass) of largest key; isolated points become
// singletons, numbered after the roots in index order.
int aggregate_mis2(int n, const std::vector<int32_t> &sp, const std::vector<int32_t> &sc,
                   std::vector<int32_t> &agg) {
  enum : char { UND = 0, ROOT = 1, OUT = 2, ISO = 3 };
  std::vector<char> st(n), nr(n), d1(n);
  std::vector<uint64_t> m1(n);
  for (int i = 0; i < n; ++i) st[i] = sp[i] == sp[i + 1] ? ISO : UND;
  const bool pa = par((long long)sp[n]);
  for (int round = 0;; ++round) {
    long long und = 0;
#pragma omp parallel for schedule(static) reduction(+ : und) if (pa)
    for (int i = 0; i < n; ++i) und += st[i] == UND;
    if (und == 0) break;
#pragma omp parallel for schedule(static) if (pa)
    for (int i = 0; i < n; ++i) {
      uint64_t m = st[i] == UND ? mis_key(i) : 0;
      for (int k = sp[i]; k < sp[i + 1]; ++k)
        if (st[sc[k]] == UND) m = std::max(m, mis_key(sc[k]));
      m1[i] = m;
    }
#pragma omp parallel for schedule(static) if (pa)
    for (int i = 0; i < n; ++i) {
      uint64_t m = m1[i];
      for (int k = sp[i]; k < sp[i + 1]; ++k) m = std::max(m, m1[sc[k]]);
      nr[i] = st[i] == UND && m == mis_key(i);
    }
#pragma omp parallel for schedule(static) if (pa)
    for (int i = 0; i < n; ++i) {
      bool d = nr[i];
      for (int k = sp[i]; k < sp[i + 1] && !d; ++k) d = nr[sc[k]];
      d1[i] = d;
    }
#pragma omp parallel for schedule(static) if (pa)
    for (int i = 0; i < n; ++i) {
      if (nr[i]) {
        st[i] = ROOT;
      } else if (st[i] == UND) {
        bool d = d1[i];
        for (int k = sp[i]; k < sp[i + 1] && !d; ++k) d = d1[sc[k]];
        if (d) st[i] = OUT;
      }
    }
  }
  agg.assign(n, -1);
  int na = 0;
  for (int i = 0; i < n; ++i)
    if (st[i] == ROOT) agg[i] = na++;
  // the first pass: next to a root
  std::vector<int32_t> a1(agg);
#pragma omp parallel for schedule(static) if (pa)
  for (int i = 0; i < n; ++i) {
    if (st[i] != OUT) continue;
    int best = -1;
    for (int k = sp[i]; k < sp[i + 1]; ++k) {
      const int j = sc[k];
      if (st[j] == ROOT && (best < 0 || mis_key(j) > mis_key(best))) best = j;
    }
    if (best >= 0) a1[i] = agg[best];
  }
  // the second pass: next to a point of the first
#pragma omp parallel for schedule(static) if (pa)
  for (int i = 0; i < n; ++i) {
    if (a1[i] >= 0 || st[i] == ISO) {
      agg[i] = a1[i];
      continue;
    }
    int best = -1;
    for (int k = sp[i]; k < sp[i + 1]; ++k) {
      const int j = sc[k];
      if (a1[j] >= 0 && (best < 0 || mis_key(j) > mis_key(best))) best = j;
    }
    agg[i] = best >= 0 ? a1[best] : -1;
  }
  for (int i = 0; i < n; ++i)
    if (agg[i] < 0) agg[i] = na++;
  return na;
}

// greedy aggregation (the coarse levels); returns the number of aggregates
int aggregate(int n, const std::vector<int32_t> &sp, const std::vector<int32_t> &sc,
              std::vector<int32_t> &agg) {
  agg.assign(n, -1);
  int na = 0;
  for (int i = 0; i < n; ++i) {  // roots with a free neighbourhood
    if (agg[i] >= 0 || sp[i] == sp[i + 1]) continue;
    bool free_nb = true;
    for (int k = sp[i]; k < sp[i + 1] && free_nb; ++k) free_nb = agg[sc[k]] < 0;
    if (!free_nb) continue;
    agg[i] = na;
    for (int k = sp[i]; k < sp[i + 1]; ++k) agg[sc[k]] = na;
    na++;
  }
  std::vector<int32_t> join(n, -1);
  for (int i = 0; i < n; ++i) {  // leftovers join a neighbouring aggregate
    if (agg[i] >= 0) continue;
    for (int k = sp[i]; k < sp[i + 1]; ++k)
      if (agg[sc[k]] >= 0) {
        join[i] = agg[sc[k]];
        break;
      }
  }
  for (int i = 0; i < n; ++i)
    if (agg[i] < 0 && join[i] >= 0) agg[i] = join[i];
  for (int i = 0; i < n; ++i)  // isolated points: singletons
    if (agg[i] < 0) agg[i] = na++;
  return na;
}

// P = T - w D^-1 A T, T[i, agg[i]] = 1
Csr smoothed_prolongator(const Csr &A, const std::vector<double> &dinv,
                         const std::vector<int32_t> &agg, int na, double w) {
  Csr P = build_rows(A.n, na, A.nnz(), [&](int i, std::vector<int32_t> &, auto &&emit) {
    emit(agg[i], 1.0);
    for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k) emit(agg[A.col[k]], -w * dinv[i] * A.val[k]);
  });
  // drop exact zeros (a row whose terms cancel), keeping the order
  Csr Q;
  Q.n = P.n;
  Q.m = P.m;
  Q.ptr.assign(P.n + 1, 0);
  for (int i = 0; i < P.n; ++i) {
    for (int k = P.ptr[i]; k < P.ptr[i + 1]; ++k)
      if (P.val[k] != 0.0) {
        Q.col.push_back(P.col[k]);
        Q.val.push_back(P.val[k]);
      }
    Q.ptr[i + 1] = (int32_t)Q.col.size();
  }
  return Q;
}

// C = A B (Gustavson: row i of C accumulates the rows of B picked by row i
// of A, columns in order of first appearance)
Csr spgemm(const Csr &A, const Csr &B) {
  const long long per = B.n > 0 ? std::max(1LL, B.nnz() / B.n) : 1;
  return build_rows(A.n, B.m, A.nnz() * per, [&](int i, std::vector<int32_t> &, auto &&emit) {
    for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k) {
      const int r = A.col[k];
      const double a = A.val[k];
      for (int t = B.ptr[r]; t < B.ptr[r + 1]; ++t) emit(B.col[t], a * B.val[t]);
    }
  });
}

// X - s(Y), s scaling Y's columns (cols = true) or rows by w.  Y's pattern
// must hold X's (true here: Y = R A or A P with A's diagonal nonzero), so
// the result has Y's pattern.
Csr minus_scaled(const Csr &X, const Csr &Y, const std::vector<double> &w, bool cols) {
  Csr C;
  C.n = Y.n;
  C.m = Y.m;
  C.ptr = Y.ptr;
  C.col = Y.col;
  C.val.resize(Y.val.size());
  int bad = 0;
  const int chunk = row_chunk(Y.n);
#pragma omp parallel if (par(Y.nnz()))
  {
    std::vector<int32_t> pos(Y.m, -1);
#pragma omp for schedule(dynamic, chunk)
    for (int i = 0; i < Y.n; ++i) {
      for (int k = Y.ptr[i]; k < Y.ptr[i + 1]; ++k) {
        C.val[k] = -(cols ? w[Y.col[k]] : w[i]) * Y.val[k];
        pos[Y.col[k]] = k;
      }
      for (int k = X.ptr[i]; k < X.ptr[i + 1]; ++k) {
        const int p = pos[X.col[k]];
        if (p >= Y.ptr[i] && p < Y.ptr[i + 1] && Y.col[p] == X.col[k])
          C.val[p] += X.val[k];
        else {
#pragma omp atomic write
          bad = 1;
        }
      }
    }
  }
  if (bad) {  // a pattern not covered (not expected): build the union serially
    C = Csr();
    C.n = X.n;
    C.m = X.m;
    C.ptr.assign(X.n + 1, 0);
    std::vector<int32_t> mark(X.m, -1), list;
    std::vector<double> acc(X.m, 0.0);
    for (int i = 0; i < X.n; ++i) {
      list.clear();
      auto add = [&](int c, double v) {
        if (mark[c] != i) {
          mark[c] = i;
          acc[c] = 0.0;
          list.push_back(c);
        }
        acc[c] += v;
      };
      for (int k = X.ptr[i]; k < X.ptr[i + 1]; ++k) add(X.col[k], X.val[k]);
      for (int k = Y.ptr[i]; k < Y.ptr[i + 1]; ++k)
        add(Y.col[k], -(cols ? w[Y.col[k]] : w[i]) * Y.val[k]);
      for (int c : list) {
        C.col.push_back(c);
        C.val.push_back(acc[c]);
      }
      C.ptr[i + 1] = (int32_t)C.col.size();
    }
  }
  return C;
}

// S = 2 W - W A W on A's pattern (every row of these matrices holds its
// diagonal; a row without one gets it appended)
Csr smoother_matrix(const Csr &A, const std::vector<double> &w) {
  Csr S;
  S.n = S.m = A.n;
  S.ptr.assign(A.n + 1, 0);
  std::vector<char> has(A.n, 0);
  const bool pa = par(A.nnz());
#pragma omp parallel for schedule(static) if (pa)
  for (int i = 0; i < A.n; ++i) {
    for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k) has[i] |= A.col[k] == i;
    S.ptr[i + 1] = A.ptr[i + 1] - A.ptr[i] + !has[i];
  }
  for (int i = 0; i < A.n; ++i) S.ptr[i + 1] += S.ptr[i];
  S.col.resize(S.ptr[A.n]);
  S.val.resize(S.ptr[A.n]);
#pragma omp parallel for schedule(static) if (pa)
  for (int i = 0; i < A.n; ++i) {
    int o = S.ptr[i];
    bool diag = false;
    for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k) {
      const int j = A.col[k];
      double v = -w[i] * A.val[k] * w[j];
      if (j == i && !diag) {
        v += 2.0 * w[i];
        diag = true;
      }
      S.col[o] = j;
      S.val[o++] = v;
    }
    if (!diag) {
      S.col[o] = i;
      S.val[o] = 2.0 * w[i];
    }
  }
  return S;
}

// ---- how the cycle spreads an operator's rows over the launch's warps
// A phase of the cycle costs the dependent L2 round trips of its slowest
// warp.  A CSR row with g lanes costs one trip for its row pointers and two
// (indices and values, then the gathers) per AMG_CSR_CHUNK entries a lane;
// an ELL row with T threads two per kdev::CH entries a thread; a warp that
// takes more than one pass over its rows pays each pass.  CSR row groups
// are spread over the CTAs (warp w of every CTA before warp w + 1), level
// 0's S runs on each CTA's own ceil(n / nb) rows; the down phase runs S_l
// and R~_l side by side (R~_l from the last warp of every CTA), so their
// lanes per row are chosen together: side by side when their warps per CTA
// fit in one CTA, one after the other otherwise.
struct Grid {
  long long nb, wpb;  // CTAs, warps per CTA
};
struct Shape {
  int rows = 0, maxlen = 0;
};
Shape shape(const Csr &M) {
  Shape s;
  s.rows = M.n;
  for (int i = 0; i < M.n; ++i) s.maxlen = std::max(s.maxlen, M.ptr[i + 1] - M.ptr[i]);
  return s;
}
long long ceil_div(long long a, long long b) { return (a + b - 1) / b; }
// warps per CTA a CSR operator keeps busy (spread over the CTAs)
long long csr_warps(const Shape &s, int g, const Grid &G) {
  return std::min(G.wpb, ceil_div(ceil_div(s.rows, 32 / g), G.nb));
}
int csr_trips(const Shape &s, int g, const Grid &G) {
  const int passes = (int)ceil_div(s.rows, G.nb * G.wpb * (32 / g));
  const int chunks = std::max(1, (s.maxlen + g * AMG_CSR_CHUNK - 1) / (g * AMG_CSR_CHUNK));
  return passes * (1 + 2 * chunks);
}
long long ell_warps(int n, int T, const Grid &G) {
  return std::min(G.wpb, ceil_div(ceil_div(n, G.nb), 32 / T));
}
int ell_trips(int n, int q, int T, const Grid &G) {
  const int passes = (int)ceil_div(ceil_div(n, G.nb), G.wpb * (32 / T));
  const int chunks = std::max(1, (q + T * kdev::CH - 1) / (T * kdev::CH));
  return passes * 2 * chunks;
}
int pair_trips(int ta, long long wa, int tb, long long wb, const Grid &G) {
  return wa + wb <= G.wpb ? std::max(ta, tb) : ta + tb;
}
// lanes per row of one CSR operator run alone
int lanes_alone(const Shape &s, const Grid &G) {
  int best = 1, bt = 1 << 30;
  for (int g = 1; g <= 32; g *= 2) {
    const int t = csr_trips(s, g, G);
    if (t < bt) bt = t, best = g;
  }
  return best;
}
// lanes per row of S_l and R~_l run side by side
void lanes_pair(const Shape &a, const Shape &b, const Grid &G, int &ga, int &gb) {
  int bt = 1 << 30;
  long long bw = 0;
  for (int x = 1; x <= 32; x *= 2)
    for (int y = 1; y <= 32; y *= 2) {
      const long long wa = csr_warps(a, x, G), wb = csr_warps(b, y, G);
      const int t = pair_trips(csr_trips(a, x, G), wa, csr_trips(b, y, G), wb, G);
      if (t < bt || (t == bt && wa + wb < bw)) bt = t, bw = wa + wb, ga = x, gb = y;
    }
}
// threads per row of level 0's S (ELL, q wide) and lanes of R~_0
void lanes_level0(int n, int q, const Shape &r, const Grid &G, int &ts, int &gr) {
  int bt = 1 << 30;
  long long bw = 0;
  for (int T = 1; T <= 8; ++T)
    for (int y = 1; y <= 32; y *= 2) {
      const long long wa = ell_warps(n, T, G), wb = csr_warps(r, y, G);
      const int t = pair_trips(ell_trips(n, q, T, G), wa, csr_trips(r, y, G), wb, G);
      if (t < bt || (t == bt && wa + wb < bw)) bt = t, bw = wa + wb, ts = T, gr = y;
    }
}

// inverse of a small CSR matrix by Gauss-Jordan with partial pivoting
bool dense_inverse(const Csr &A, std::vector<double> &inv) {
  const int n = A.n, w = 2 * n;
  std::vector<double> M((size_t)n * w, 0.0);
  for (int i = 0; i < n; ++i) {
    for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k) M[(size_t)i * w + A.col[k]] += A.val[k];
    M[(size_t)i * w + n + i] = 1.0;
  }
  for (int k = 0; k < n; ++k) {
    int piv = k;
    double best = std::fabs(M[(size_t)k * w + k]);
    for (int i = k + 1; i < n; ++i) {
      const double a = std::fabs(M[(size_t)i * w + k]);
      if (a > best) {
        best = a;
        piv = i;
      }
    }
    if (best == 0.0) return false;
    if (piv != k)
      for (int j = 0; j < w; ++j) std::swap(M[(size_t)k * w + j], M[(size_t)piv * w + j]);
    const double r = 1.0 / M[(size_t)k * w + k];
    for (int j = 0; j < w; ++j) M[(size_t)k * w + j] *= r;
    for (int i = 0; i < n; ++i) {
      if (i == k) continue;
      const double f = M[(size_t)i * w + k];
      if (f == 0.0) continue;
      for (int j = 0; j < w; ++j) M[(size_t)i * w + j] -= f * M[(size_t)k * w + j];
    }
  }
  inv.resize((size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) inv[(size_t)i * n + j] = M[(size_t)i * w + n + j];
  return true;
}

struct Hierarchy {
  std::vector<Csr> A, S, R, P;         // A_l; S_l (l >= 1); R~_l, P~_l (l < L-1)
  std::vector<std::vector<double>> W;  // w_l D_l^-1
  std::vector<double> omega, cinv;
};

// The levels of A0 (see the top of the file).  RBFFD_OK, or an error with
// its text set.
int build_levels(Hierarchy &H);

int build_hierarchy(Csr A0, Hierarchy &H) {
  H.A.push_back(std::move(A0));
  return build_levels(H);
}

// The levels from H.A.back() on (H holds the finer levels already).
int build_levels(Hierarchy &H) {
  for (;;) {
    const Csr &A = H.A.back();
    std::vector<double> d = diagonal(A), dinv(A.n);
    for (int i = 0; i < A.n; ++i) dinv[i] = d[i] != 0.0 ? 1.0 / d[i] : 0.0;
    const double lam = rho_estimate(A, dinv);
    const double om = std::min(AMG_OMEGA, 4.0 / (3.0 * lam));
    std::vector<double> wd(A.n);
    for (int i = 0; i < A.n; ++i) wd[i] = om * dinv[i];
    H.omega.push_back(om);
    H.S.push_back(H.A.size() > 1 ? smoother_matrix(A, wd) : Csr());  // level 0: ELL copy
    H.W.push_back(std::move(wd));
    if (A.n <= AMG_NCOARSE || (int)H.A.size() == AMG_MAXLEV) break;
    std::vector<int32_t> sp, sc, agg;
    strength(A, AMG_THETA, sp, sc);
    const int na = H.A.size() == 1 ? aggregate_mis2(A.n, sp, sc, agg)
                                   : aggregate(A.n, sp, sc, agg);
    if (na > 0.8 * A.n || na == 0) break;  // coarsening stalled
    Csr P = smoothed_prolongator(A, dinv, agg, na, 4.0 / (3.0 * lam));
    Csr R = transpose(P);
    Csr AP = spgemm(A, P);
    Csr Ac = spgemm(R, AP);  // R (A P)
    // R~ = R (I - A W) = ((I - W A^T) P)^T, built row by row over the fine
    // level like P~ (the device's level-0 build takes the same route)
    Csr AtP = spgemm(transpose(A), P);
    const std::vector<double> &w = H.W.back();
    H.R.push_back(transpose(minus_scaled(P, AtP, w, false)));
    H.P.push_back(minus_scaled(P, AP, w, false));  // (I - W A) P
    H.A.push_back(std::move(Ac));
  }
  if (H.A.back().n > AMG_NCOARSE_MAX) {
    set_error("amg: coarsening stalled at %d rows", H.A.back().n);
    return RBFFD_ENOTIMPL;
  }
  if (!dense_inverse(H.A.back(), H.cinv)) {
    set_error("amg: the coarsest matrix (%d rows) is singular", H.A.back().n);
    return RBFFD_ESINGULAR;
  }
  return RBFFD_OK;
}

// ---- the composed cycle (amg.cuh): the folded V-cycle is one linear map;
// below level 1 it regroups as
//   y_1 = S_1 b_1 + sum_{l >= 2} Q_l b_l,   b_l = Rh_l b_1,
// with Rh_2 = R~_1, Rh_l = R~_{l-1} Rh_{l-1} (restriction straight from
// level 1), Q_l = P~_1 ... P~_{l-1} S_l and, on the coarsest level,
// P~_1 ... P~_{L-2} A_{L-1}^-1 (the corrections prolonged to level 1): the
// same sums as the level-by-level cycle, so that its 2 L - 1 dependent
// phases become four.  The rows of the stacked Rh are cut into chunks of at
// most AMG_RCHUNK entries, each summed by one warp; coarse entry k is the
// sum of its chunks in order.
struct Composed {
  Csr R;                               // Nc x n1: Rh_2; Rh_3; ... stacked
  Csr Q;                               // n1 x Nc: [Q_2 | Q_3 | ...]
  std::vector<int32_t> cs, kc;         // chunk c: entries [cs[c], cs[c+1]); entry k: chunks [kc[k], kc[k+1])
  std::vector<int> seg_off, seg_grp;   // level s + 2: entries [seg_off[s], seg_off[s+1]); lanes per entry
};

// M * D with D dense row-major (m x m), every product kept
Csr times_dense(const Csr &M, const std::vector<double> &D, int m) {
  Csr C;
  C.n = M.n;
  C.m = m;
  C.ptr.resize(M.n + 1);
  for (int i = 0; i <= M.n; ++i) C.ptr[i] = i * m;
  C.col.resize((size_t)M.n * m);
  C.val.assign((size_t)M.n * m, 0.0);
#pragma omp parallel for schedule(static) if (par(M.nnz() * m))
  for (int i = 0; i < M.n; ++i) {
    double *o = C.val.data() + (size_t)i * m;
    for (int j = 0; j < m; ++j) C.col[(size_t)i * m + j] = j;
    for (int k = M.ptr[i]; k < M.ptr[i + 1]; ++k) {
      const double a = M.val[k];
      const double *d = D.data() + (size_t)M.col[k] * m;
      for (int j = 0; j < m; ++j) o[j] += a * d[j];
    }
  }
  return C;
}

// Rows of A (n x ma), then of B (n x mb) as columns ma.. : [A | B]
Csr hcat(const Csr &A, const Csr &B) {
  Csr C;
  C.n = A.n;
  C.m = A.m + B.m;
  C.ptr.assign(A.n + 1, 0);
  for (int i = 0; i < A.n; ++i)
    C.ptr[i + 1] = C.ptr[i] + (A.ptr[i + 1] - A.ptr[i]) + (B.ptr[i + 1] - B.ptr[i]);
  C.col.resize(C.ptr[A.n]);
  C.val.resize(C.ptr[A.n]);
  for (int i = 0; i < A.n; ++i) {
    int o = C.ptr[i];
    for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k) C.col[o] = A.col[k], C.val[o++] = A.val[k];
    for (int k = B.ptr[i]; k < B.ptr[i + 1]; ++k) C.col[o] = A.m + B.col[k], C.val[o++] = B.val[k];
  }
  return C;
}

// The composed operators, for hierarchies of three or more levels (with two
// the cycle already has four phases or fewer); false: the level-by-level
// cycle only.  The products are level-1-sized: small next to the build.
bool compose(const Hierarchy &H, Composed &C) {
  const int L = (int)H.A.size();
  if (L < 3) return false;
  // stacked Rh_2 .. Rh_{L-1}, each n_l x n_1
  C = Composed();
  C.R.m = H.A[1].n;
  C.R.ptr.assign(1, 0);
  C.seg_off.assign(1, 0);
  Csr Rh;
  for (int l = 2; l < L; ++l) {
    Rh = l == 2 ? H.R[1] : spgemm(H.R[l - 1], Rh);
    for (int i = 0; i < Rh.n; ++i) C.R.ptr.push_back(C.R.ptr.back() + Rh.ptr[i + 1] - Rh.ptr[i]);
    C.R.col.insert(C.R.col.end(), Rh.col.begin(), Rh.col.end());
    C.R.val.insert(C.R.val.end(), Rh.val.begin(), Rh.val.end());
    C.R.n += Rh.n;
    C.seg_off.push_back(C.R.n);
  }
  // Q = [Q_2 | ... | Q_{L-1}] on level 1's rows; M = P~_1 ... P~_{l-1}
  Csr M = H.P[1], Q;
  for (int l = 2; l < L; ++l) {
    const Csr Ql = l + 1 < L ? spgemm(M, H.S[l]) : times_dense(M, H.cinv, H.A[l].n);
    Q = l == 2 ? Ql : hcat(Q, Ql);
    if (l + 1 < L) M = spgemm(M, H.P[l]);
  }
  C.Q = std::move(Q);
  // chunks: a row of length len in ceil(len / AMG_RCHUNK) near-equal pieces
  C.cs.assign(1, 0);
  C.kc.assign(1, 0);
  std::vector<int> maxch(L, 1);
  for (int k = 0, s = 0; k < C.R.n; ++k) {
    while (k >= C.seg_off[s + 1]) ++s;
    const int a = C.R.ptr[k], len = C.R.ptr[k + 1] - a;
    const int nch = std::max(1, (len + AMG_RCHUNK - 1) / AMG_RCHUNK);
    for (int j = 1; j <= nch; ++j) C.cs.push_back(a + (int)((long long)len * j / nch));
    C.kc.push_back(C.kc.back() + nch);
    maxch[s] = std::max(maxch[s], nch);
  }
  // lanes per coarse entry summing its chunks: at most 4 loads a lane
  C.seg_grp.assign(L - 2, 1);
  for (int s = 0; s + 2 < L; ++s) {
    int g = 1;
    while (g < 32 && (maxch[s] + g - 1) / g > 4) g *= 2;
    C.seg_grp[s] = g;
  }
  return true;
}

// The per-level V-cycle and the composed one applied on the host in FP64
// (a check of the composition: the two agree to rounding).  The composed
// form sums in the device's order: chunk by chunk, then the chunks of an
// entry in order.
void cycle_levels(const Hierarchy &H, const std::vector<double> &b0, std::vector<double> &out) {
  const int L = (int)H.A.size();
  auto mv = [](const Csr &M, const std::vector<double> &x) {
    std::vector<double> y(M.n, 0.0);
    for (int i = 0; i < M.n; ++i)
      for (int k = M.ptr[i]; k < M.ptr[i + 1]; ++k) y[i] += M.val[k] * x[M.col[k]];
    return y;
  };
  auto smooth0 = [&](const std::vector<double> &b) {  // S_0 = 2 W - W A W
    const std::vector<double> &w = H.W[0];
    const Csr &A = H.A[0];
    std::vector<double> y(A.n, 0.0);
    for (int i = 0; i < A.n; ++i) {
      double t = 2.0 * w[i] * b[i];
      for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k) t -= w[i] * A.val[k] * w[A.col[k]] * b[A.col[k]];
      y[i] = t;
    }
    return y;
  };
  auto dense = [&](const std::vector<double> &b) {
    const int m = (int)b.size();
    std::vector<double> y(m, 0.0);
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) y[i] += H.cinv[(size_t)i * m + j] * b[j];
    return y;
  };
  if (L == 1) {
    out = dense(b0);
    return;
  }
  std::vector<std::vector<double>> z(L), b(L);
  b[0] = b0;
  for (int l = 0; l + 1 < L; ++l) {
    z[l] = l == 0 ? smooth0(b[0]) : mv(H.S[l], b[l]);
    b[l + 1] = mv(H.R[l], b[l]);
  }
  std::vector<double> y = dense(b[L - 1]);
  for (int l = L - 2; l >= 0; --l) {
    std::vector<double> t = mv(H.P[l], y);
    for (size_t i = 0; i < t.size(); ++i) t[i] += z[l][i];
    y = std::move(t);
  }
  out = std::move(y);
}

void cycle_composed(const Hierarchy &H, const Composed &C, const std::vector<double> &b0,
                    std::vector<double> &out) {
  auto mv = [](const Csr &M, const std::vector<double> &x) {
    std::vector<double> y(M.n, 0.0);
    for (int i = 0; i < M.n; ++i)
      for (int k = M.ptr[i]; k < M.ptr[i + 1]; ++k) y[i] += M.val[k] * x[M.col[k]];
    return y;
  };
  const std::vector<double> b1 = mv(H.R[0], b0);
  const int nch = (int)C.cs.size() - 1;
  std::vector<double> part(nch, 0.0), cv(C.R.n, 0.0);
  for (int c = 0; c < nch; ++c)
    for (int k = C.cs[c]; k < C.cs[c + 1]; ++k) part[c] += C.R.val[k] * b1[C.R.col[k]];
  for (int k = 0; k < C.R.n; ++k)
    for (int c = C.kc[k]; c < C.kc[k + 1]; ++c) cv[k] += part[c];
  std::vector<double> y1 = mv(H.S[1], b1);
  const std::vector<double> q = mv(C.Q, cv);
  for (size_t i = 0; i < y1.size(); ++i) y1[i] += q[i];
  const std::vector<double> &w = H.W[0];
  const Csr &A = H.A[0];
  out.assign(A.n, 0.0);
  for (int i = 0; i < A.n; ++i) {
    double t = 2.0 * w[i] * b0[i];
    for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k) t -= w[i] * A.val[k] * w[A.col[k]] * b0[A.col[k]];
    for (int k = H.P[0].ptr[i]; k < H.P[0].ptr[i + 1]; ++k) t += H.P[0].val[k] * y1[H.P[0].col[k]];
    out[i] = t;
  }
}

void fill_info(const Hierarchy &H, double ms, AmgInfo *info, const Composed *C = nullptr,
               const AmgL0 *l0 = nullptr) {
  if (!info) return;
  memset(info, 0, sizeof(*info));
  info->device_l0 = l0 != nullptr;
  if (C) {
    info->comp_nc = C->R.n;
    info->comp_chunks = (int)C->cs.size() - 1;
    info->comp_nnz_r = C->R.nnz();
    info->comp_nnz_q = C->Q.nnz();
  }
  const int L = (int)H.A.size();
  info->nlev = L;
  info->setup_ms = ms;
  for (int l = 0; l < L; ++l) {
    info->n[l] = H.A[l].n;
    info->nnz[l] = H.A[l].nnz();
    info->nnz_r[l] = l + 1 < L ? H.R[l].nnz() : 0;
    info->nnz_p[l] = l + 1 < L ? H.P[l].nnz() : 0;
    info->omega[l] = H.omega[l];
  }
  if (l0) {  // level 0 was built on the device: its sizes come from there
    info->nnz[0] = l0->nnz_a;
    info->nnz_r[0] = l0->nnz_r;
    info->nnz_p[0] = l0->nnz_p;
  }
}

double ms_since(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

// One host buffer for the whole upload, packed in two passes over the same
// sequence of take / put calls: the first (buf null) only measures, the
// second fills one allocation of that size.  Regions that are only taken
// (level vectors, alignment gaps) are left as they are: the cycle writes
// its vectors before it reads them.
struct Staging {
  size_t size = 0;
  char *buf = nullptr;
  std::unique_ptr<char[]> own;
  void fill_pass() {
    own.reset(new char[size]);
    buf = own.get();
    size = 0;
  }
  size_t take(size_t bytes) {
    const size_t at = size;
    size += (bytes + 255) / 256 * 256;
    return at;
  }
  template <typename T>
  size_t put(const std::vector<T> &v) {
    const size_t at = take(v.size() * sizeof(T));
    if (buf && !v.empty()) memcpy(buf + at, v.data(), v.size() * sizeof(T));
    return at;
  }
  // FP64 values stored in the cycle's arithmetic T (round to nearest)
  template <typename T>
  size_t put_as(const std::vector<double> &v) {
    const size_t at = take(v.size() * sizeof(T));
    if (buf) {
      T *d = reinterpret_cast<T *>(buf + at);
      const long long m = (long long)v.size();
#pragma omp parallel for schedule(static) if (par(m))
      for (long long k = 0; k < m; ++k) d[k] = (T)v[k];
    }
    return at;
  }
};

}  // namespace

int amg_analyze(int n, const int32_t *rowptr, const int32_t *col, const double *val,
                AmgInfo *info) {
  const auto t0 = std::chrono::steady_clock::now();
  Csr A;
  A.n = A.m = n;
  A.ptr.assign(rowptr, rowptr + n + 1);
  A.col.assign(col, col + rowptr[n]);
  A.val.assign(val, val + rowptr[n]);
  Hierarchy H;
  RBFFD_TRY(build_hierarchy(std::move(A), H));
  Composed C;
  const bool comp = compose(H, C);
  fill_info(H, ms_since(t0), info, comp ? &C : nullptr);
  return RBFFD_OK;
}

int amg_aggregates_host(int n, const int32_t *rowptr, const int32_t *col, const double *val,
                        int32_t *agg, int32_t *naggs) {
  Csr A;
  A.n = A.m = n;
  A.ptr.assign(rowptr, rowptr + n + 1);
  A.col.assign(col, col + rowptr[n]);
  A.val.assign(val, val + rowptr[n]);
  std::vector<int32_t> sp, sc, a;
  strength(A, AMG_THETA, sp, sc);
  *naggs = aggregate_mis2(n, sp, sc, a);
  std::copy(a.begin(), a.end(), agg);
  return RBFFD_OK;
}

int amg_cycle_host(int n, const int32_t *rowptr, const int32_t *col, const double *val,
                   const double *b, double *out_levels, double *out_composed, AmgInfo *info) {
  Csr A;
  A.n = A.m = n;
  A.ptr.assign(rowptr, rowptr + n + 1);
  A.col.assign(col, col + rowptr[n]);
  A.val.assign(val, val + rowptr[n]);
  Hierarchy H;
  RBFFD_TRY(build_hierarchy(std::move(A), H));
  Composed C;
  const bool comp = compose(H, C);
  fill_info(H, 0.0, info, comp ? &C : nullptr);
  const std::vector<double> b0(b, b + n);
  std::vector<double> y;
  cycle_levels(H, b0, y);
  std::copy(y.begin(), y.end(), out_levels);
  if (comp) {
    cycle_composed(H, C, b0, y);
    std::copy(y.begin(), y.end(), out_composed);
  } else {
    std::fill(out_composed, out_composed + n, 0.0);
  }
  return RBFFD_OK;
}

// ---- the build as a job: the host part (copy of the packed matrix, the
// hierarchy, its staging) runs on a host thread of its own, the device part
// (allocation, upload) on the caller's thread, so the host part overlaps
// the device work the caller issues meanwhile.
struct CsrOff {
  size_t ptr = 0, col = 0, val = 0;
  int grp = 1;
};
struct LevelOff {
  CsrOff S, R, P;
  size_t b = 0, z = 0, y = 0;
};
struct CompOff {
  size_t rcol = 0, rval = 0, cs = 0, kc = 0, part = 0;
  CsrOff Q;
};

struct AmgJob {
  int device = 0, n = 0, q = 0, ldn = 0, nblocks = 0, wpb = 0;
  const int32_t *dcol = nullptr;
  const double *dval = nullptr;
  cudaEvent_t ready = nullptr;  // the packed matrix is written (caller's stream)
  std::thread th;
  int rc = RBFFD_OK;
  char err[256] = "";
  double host_ms = 0;  // copy, hierarchy and staging, from the matrix being ready
  Hierarchy H;
  Staging S;
  std::vector<LevelOff> off;
  size_t o_dev = 0, o_s0 = 0, o_a0 = 0, o_cinv = 0;
  int ts0 = 1;
  bool low = false;  // the cycle's type is FP32
  bool compose = true;  // build the composed cycle when it pays
  bool comp = false;    // built
  Composed C;
  CompOff coff;
  rbffd_ctx *ctx = nullptr;
  bool l0dev = false;  // level 0 built on the device (amg_setup.cu)
  AmgL0 L0;
  int gR0 = 1, gP0 = 1;  // lanes per row of level 0's R~ and P~ (device-built)
};

namespace {

// The coarse levels after a device-built level 0: level 0 stands in the
// hierarchy by its size only, A_1 comes from the device.
template <typename T>
int host_part_coarse(AmgJob &J) {
  const auto t0 = std::chrono::steady_clock::now();
  const int n = J.n, q = J.q;
  const AmgL0 &L0 = J.L0;
  const int n1 = L0.n1;
  Hierarchy &H = J.H;
  Csr A0, R0, P0, A1;
  A0.n = A0.m = n;
  A0.ptr.assign(n + 1, 0);
  R0.n = n1;
  R0.m = n;
  R0.ptr.assign(n1 + 1, 0);
  P0.n = n;
  P0.m = n1;
  P0.ptr.assign(n + 1, 0);
  A1.n = A1.m = n1;
  A1.ptr = L0.a1ptr;
  A1.col = L0.a1col;
  A1.val = L0.a1val;
  H.A.push_back(std::move(A0));
  H.omega.push_back(L0.omega);
  H.S.push_back(Csr());
  H.W.push_back(std::vector<double>());
  H.R.push_back(std::move(R0));
  H.P.push_back(std::move(P0));
  H.A.push_back(std::move(A1));
  RBFFD_TRY(build_levels(H));
  const int L = (int)H.A.size();
  J.comp = J.compose && compose(H, J.C);
  Staging &S = J.S;
  auto put_csr = [&](const Csr &M, int grp) {
    CsrOff o;
    o.ptr = S.put(M.ptr);
    o.col = S.put(M.col);
    o.val = S.put_as<T>(M.val);
    o.grp = grp;
    return o;
  };
  const Grid W{J.nblocks > 0 ? J.nblocks : 128, J.wpb > 0 ? J.wpb : 32};
  std::vector<int> gS(L, 1), gR(L, 1), gP(L, 1);
  {
    Shape r0, p0;
    r0.rows = n1;
    r0.maxlen = L0.maxlen_r;
    p0.rows = n;
    p0.maxlen = L0.maxlen_p;
    lanes_level0(n, q, r0, W, J.ts0, J.gR0);
    J.gP0 = lanes_alone(p0, W);
  }
  for (int l = 1; l + 1 < L; ++l) {
    lanes_pair(shape(H.S[l]), shape(H.R[l]), W, gS[l], gR[l]);
    gP[l] = lanes_alone(shape(H.P[l]), W);
  }
  std::vector<LevelOff> &off = J.off;
  off.assign(L, LevelOff());
  J.low = sizeof(T) < sizeof(double);
  for (int pass = 0; pass < 2; ++pass) {
    if (pass == 1) S.fill_pass();
    J.o_dev = S.take(sizeof(AmgDevT<T>));
    for (int l = 1; l < L; ++l) {
      off[l].S = put_csr(H.S[l], l + 1 < L ? gS[l] : 1);
      if (l + 1 < L) {
        off[l].R = put_csr(H.R[l], gR[l]);
        off[l].P = put_csr(H.P[l], gP[l]);
      }
      off[l].b = S.take(sizeof(T) * H.A[l].n);
      off[l].z = S.take(sizeof(T) * H.A[l].n);
      off[l].y = S.take(sizeof(T) * H.A[l].n);
    }
    J.o_cinv = S.put_as<T>(H.cinv);
    if (J.comp) {
      CompOff &co = J.coff;
      co.rcol = S.put(J.C.R.col);
      co.rval = S.put_as<T>(J.C.R.val);
      co.cs = S.put(J.C.cs);
      co.kc = S.put(J.C.kc);
      co.Q = put_csr(J.C.Q, lanes_alone(shape(J.C.Q), W));
      co.part = S.take(sizeof(T) * (J.C.cs.size() - 1));
    }
  }
  J.host_ms = ms_since(t0);
  return RBFFD_OK;
}

template <typename T>
int host_part(AmgJob &J) {
  if (J.l0dev) return host_part_coarse<T>(J);
  const int n = J.n, q = J.q, ldn = J.ldn;
  std::vector<int32_t> hcol((size_t)q * ldn);
  std::vector<double> hval((size_t)q * ldn);
  if (cudaEventSynchronize(J.ready) != cudaSuccess) {
    set_error("amg: wait for the p' matrix failed");
    return RBFFD_ECUDA;
  }
  const auto t0 = std::chrono::steady_clock::now();
  {
    // the copies run on a stream of their own (the caller's may hold more work)
    cudaStream_t cs = nullptr;
    RBFFD_CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    const bool okc =
        cudaMemcpyAsync(hcol.data(), J.dcol, hcol.size() * 4, cudaMemcpyDeviceToHost, cs) ==
            cudaSuccess &&
        cudaMemcpyAsync(hval.data(), J.dval, hval.size() * 8, cudaMemcpyDeviceToHost, cs) ==
            cudaSuccess &&
        cudaStreamSynchronize(cs) == cudaSuccess;
    cudaStreamDestroy(cs);
    if (!okc) {
      set_error("amg: copy of the p' matrix failed");
      return RBFFD_ECUDA;
    }
  }
  Hierarchy &H = J.H;
  RBFFD_TRY(build_hierarchy(from_ell(n, q, ldn, hcol, hval), H));
  const int L = (int)H.A.size();
  J.comp = J.compose && compose(H, J.C);
  // level 0's S in the solve's ELL layout: s_e = -w_i a_e w_c (+ 2 w_i on the diagonal)
  std::vector<double> s0((size_t)q * ldn, 0.0);
  {
    const std::vector<double> &w = H.W[0];
#pragma omp parallel for schedule(static) if (par((long long)n * q))
    for (int i = 0; i < n; ++i) {
      bool diag = false;
      for (int j = 0; j < q; ++j) {
        const size_t e = (size_t)j * ldn + i;
        const int c = hcol[e];
        double v = -w[i] * hval[e] * w[c];
        if (c == i && !diag) {
          v += 2.0 * w[i];
          diag = true;
        }
        s0[e] = v;
      }
    }
  }

  // ---- pack everything into one staging buffer, then one upload
  Staging &S = J.S;
  auto put_csr = [&](const Csr &M, int grp) {
    CsrOff o;
    o.ptr = S.put(M.ptr);
    o.col = S.put(M.col);
    o.val = S.put_as<T>(M.val);
    o.grp = grp;
    return o;
  };
  // lanes per row for the launch's CTAs (see Shape)
  const Grid W{J.nblocks > 0 ? J.nblocks : 128, J.wpb > 0 ? J.wpb : 32};
  std::vector<int> gS(L, 1), gR(L, 1), gP(L, 1);
  for (int l = 0; l + 1 < L; ++l) {
    const Shape r = shape(H.R[l]);
    if (l == 0)
      lanes_level0(n, q, r, W, J.ts0, gR[0]);
    else
      lanes_pair(shape(H.S[l]), r, W, gS[l], gR[l]);
    gP[l] = lanes_alone(shape(H.P[l]), W);
  }
  std::vector<LevelOff> &off = J.off;
  off.assign(L, LevelOff());
  // an FP32 cycle's solve (flexible GMRES) runs its inner SpMVs on level
  // 0's matrix in FP32 too: a rounded copy of the ELL values
  J.low = sizeof(T) < sizeof(double);
  for (int pass = 0; pass < 2; ++pass) {
    if (pass == 1) S.fill_pass();
    J.o_dev = S.take(sizeof(AmgDevT<T>));
    J.o_s0 = S.put_as<T>(s0);
    J.o_a0 = J.low ? S.put_as<T>(hval) : 0;
    for (int l = 0; l < L; ++l) {
      if (l > 0) off[l].S = put_csr(H.S[l], l + 1 < L ? gS[l] : 1);
      if (l + 1 < L) {
        off[l].R = put_csr(H.R[l], gR[l]);
        off[l].P = put_csr(H.P[l], gP[l]);
      }
      if (l > 0) off[l].b = S.take(sizeof(T) * H.A[l].n);
      off[l].z = S.take(sizeof(T) * H.A[l].n);
      off[l].y = S.take(sizeof(T) * H.A[l].n);
    }
    J.o_cinv = S.put_as<T>(H.cinv);
    if (J.comp) {
      CompOff &co = J.coff;
      co.rcol = S.put(J.C.R.col);
      co.rval = S.put_as<T>(J.C.R.val);
      co.cs = S.put(J.C.cs);
      co.kc = S.put(J.C.kc);
      co.Q = put_csr(J.C.Q, lanes_alone(shape(J.C.Q), W));
      co.part = S.take(sizeof(T) * (J.C.cs.size() - 1));
    }
  }
  J.host_ms = ms_since(t0);
  return RBFFD_OK;
}

void join(AmgJob *J) {
  if (J->th.joinable()) J->th.join();
  if (J->ready) cudaEventDestroy(J->ready);
  J->ready = nullptr;
}

// a job given up: its device-built level 0 goes with it
void drop(AmgJob *J) {
  join(J);
  if (J->L0.mem) dev_free(J->ctx, J->L0.mem, J->L0.bytes);
  J->L0.mem = nullptr;
  delete J;
}

}  // namespace

template <typename T>
int amg_build_begin(rbffd_ctx *ctx, int n, int q, int ldn, const int32_t *col,
                    const double *val, int nblocks, int wpb, AmgJob **job) {
  *job = nullptr;
  AmgJob *J = new AmgJob();
  J->device = ctx->device;
  J->n = n;
  J->q = q;
  J->ldn = ldn;
  J->nblocks = nblocks;
  J->wpb = wpb;
  J->dcol = col;
  J->dval = val;
  J->compose = ctx->amg_compose;
  J->ctx = ctx;
  // level 0 on the device when it applies (amg_setup.cu), on the caller's
  // stream before it goes on (issued from the job's thread beside a running
  // persistent solve, the setup's short kernels and readbacks took 16 ms
  // instead of 3.6); else, or when the device build gives up, the whole
  // hierarchy on the host
  if (ctx->amg_device_setup && n >= AMG_SETUP_MIN_ROWS) {
    const int rc = amg_level0_device<T>(ctx, ctx->stream, n, q, ldn, col, val,
                                        sizeof(T) < sizeof(double), &J->L0);
    if (rc == RBFFD_OK) {
      J->l0dev = true;
    } else if (rc != RBFFD_ENOTIMPL) {
      drop(J);
      return rc;
    }
    cudaGetLastError();
  }
  if (cudaEventCreateWithFlags(&J->ready, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventRecord(J->ready, ctx->stream) != cudaSuccess) {
    cudaGetLastError();
    drop(J);
    set_error("amg: event for the hierarchy build failed");
    return RBFFD_ECUDA;
  }
  const int rc = guarded([&] {
    J->th = std::thread([J] {
      cudaSetDevice(J->device);
      J->rc = guarded([J] { return host_part<T>(*J); });
      if (J->rc != RBFFD_OK) snprintf(J->err, sizeof(J->err), "%s", rbffd_last_error());
    });
    return RBFFD_OK;
  });
  if (rc != RBFFD_OK) {
    drop(J);
    return rc;
  }
  *job = J;
  return RBFFD_OK;
}

template <typename T>
int amg_build_end(rbffd_ctx *ctx, AmgJob **job, void **mem, size_t *bytes, void **mem0,
                  size_t *bytes0, const AmgDevT<T> **dev, AmgDevT<T> *host_view,
                  AmgInfo *info) {
  *mem = nullptr;
  *bytes = 0;
  *mem0 = nullptr;
  *bytes0 = 0;
  *dev = nullptr;
  AmgJob *J = *job;
  join(J);
  if (J->rc != RBFFD_OK) {
    *job = nullptr;
    set_error("%s", J->err);
    const int rc = J->rc;
    drop(J);
    return rc;
  }
  const Hierarchy &H = J->H;
  Staging &S = J->S;
  const int L = (int)H.A.size();
  void *dmem = nullptr;
  // no device memory for the upload: the finished host part stays with the
  // caller (*job unchanged), which may retry once memory has been freed
  const int arc = dev_alloc(ctx, &dmem, S.size);
  if (arc != RBFFD_OK) return arc;
  *job = nullptr;
  // the device-built level 0 passes to the caller with the rest
  void *l0mem = J->L0.mem;
  const size_t l0bytes = J->L0.bytes;
  J->L0.mem = nullptr;
  std::unique_ptr<AmgJob> own(J);
  char *base = (char *)dmem;
  char *base0 = (char *)l0mem;
  auto csr_at = [&](const CsrOff &o, bool have) {
    AmgCsrT<T> c;
    c.ptr = have ? (const int32_t *)(base + o.ptr) : nullptr;
    c.col = have ? (const int32_t *)(base + o.col) : nullptr;
    c.val = have ? (const T *)(base + o.val) : nullptr;
    c.grp = o.grp;
    return c;
  };
  AmgDevT<T> h;
  memset(&h, 0, sizeof(h));
  h.nlev = L;
  h.cinv = (const T *)(base + J->o_cinv);
  h.ts0 = J->ts0;
  for (int l = 0; l < L; ++l) {
    AmgLevelT<T> &v = h.lev[l];
    const LevelOff &o = J->off[l];
    v.n = H.A[l].n;
    v.S = csr_at(o.S, l > 0);
    v.R = csr_at(o.R, l + 1 < L);
    v.P = csr_at(o.P, l + 1 < L);
    v.b = l > 0 ? (T *)(base + o.b) : nullptr;
    v.z = (T *)(base + o.z);
    v.y = (T *)(base + o.y);
  }
  if (J->l0dev) {
    const AmgL0 &d = J->L0;
    h.s0 = (const T *)(base0 + d.o_s0);
    h.a0 = J->low ? (const T *)(base0 + d.o_a0) : nullptr;
    AmgLevelT<T> &v = h.lev[0];
    v.R.ptr = (const int32_t *)(base0 + d.o_rp);
    v.R.col = (const int32_t *)(base0 + d.o_rc);
    v.R.val = (const T *)(base0 + d.o_rv);
    v.R.grp = J->gR0;
    v.P.ptr = (const int32_t *)(base0 + d.o_pp);
    v.P.col = (const int32_t *)(base0 + d.o_pc);
    v.P.val = (const T *)(base0 + d.o_pv);
    v.P.grp = J->gP0;
    v.z = (T *)(base0 + d.o_z);
    v.y = (T *)(base0 + d.o_y);
  } else {
    h.s0 = (const T *)(base + J->o_s0);
    h.a0 = J->low ? (const T *)(base + J->o_a0) : nullptr;
  }
  if (J->comp) {
    const Composed &C = J->C;
    const CompOff &co = J->coff;
    AmgCompT<T> &m = h.comp;
    m.nc = C.R.n;
    m.nchunk = (int)C.cs.size() - 1;
    m.nseg = (int)C.seg_grp.size();
    for (int s = 0; s <= m.nseg; ++s) m.seg_off[s] = C.seg_off[s];
    for (int s = 0; s < m.nseg; ++s) m.seg_grp[s] = C.seg_grp[s];
    m.rcol = (const int32_t *)(base + co.rcol);
    m.rval = (const T *)(base + co.rval);
    m.cs = (const int32_t *)(base + co.cs);
    m.kc = (const int32_t *)(base + co.kc);
    m.Q = csr_at(co.Q, true);
    m.part = (T *)(base + co.part);
  }
  memcpy(S.buf + J->o_dev, &h, sizeof(h));
  if (cudaMemcpyAsync(dmem, S.buf, S.size, cudaMemcpyHostToDevice, ctx->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
    dev_free(ctx, dmem, S.size);
    if (l0mem) dev_free(ctx, l0mem, l0bytes);
    set_error("amg: upload failed");
    return RBFFD_ECUDA;
  }
  *mem = dmem;
  *bytes = S.size;
  *mem0 = l0mem;
  *bytes0 = l0mem ? l0bytes : 0;
  *dev = (const AmgDevT<T> *)(base + J->o_dev);
  if (host_view) *host_view = h;
  fill_info(H, J->host_ms, info, J->comp ? &J->C : nullptr, J->l0dev ? &J->L0 : nullptr);
  return RBFFD_OK;
}

void amg_build_abandon(AmgJob *J) {
  if (!J) return;
  drop(J);
}

template <typename T>
int amg_build(rbffd_ctx *ctx, int n, int q, int ldn, const int32_t *col, const double *val,
              int nblocks, int wpb, void **mem, size_t *bytes, void **mem0, size_t *bytes0,
              const AmgDevT<T> **dev, AmgDevT<T> *host_view, AmgInfo *info) {
  AmgJob *J = nullptr;
  RBFFD_TRY(amg_build_begin<T>(ctx, n, q, ldn, col, val, nblocks, wpb, &J));
  const int rc = amg_build_end<T>(ctx, &J, mem, bytes, mem0, bytes0, dev, host_view, info);
  amg_build_abandon(J);  // still set only when the upload found no memory
  return rc;
}

#define RBFFD_AMG_INSTANCES(T)                                                                  \
  template int amg_build<T>(rbffd_ctx *, int, int, int, const int32_t *, const double *, int,  \
                            int, void **, size_t *, void **, size_t *, const AmgDevT<T> **,     \
                            AmgDevT<T> *, AmgInfo *);                                          \
  template int amg_build_begin<T>(rbffd_ctx *, int, int, int, const int32_t *, const double *, \
                                  int, int, AmgJob **);                                        \
  template int amg_build_end<T>(rbffd_ctx *, AmgJob **, void **, size_t *, void **, size_t *,  \
                                const AmgDevT<T> **, AmgDevT<T> *, AmgInfo *);
RBFFD_AMG_INSTANCES(double)
RBFFD_AMG_INSTANCES(float)

}  // namespace rbffd
