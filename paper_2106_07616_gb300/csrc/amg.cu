// amg.cu -- host construction of the smoothed-aggregation hierarchy of the
// pressure-correction matrix (see amg.cuh), then one upload.
//
// Per level l (A_0 = the p' matrix):
//   strength  i ~ j  if |a_ij| >= theta * max_{k != i} |a_ik|, symmetrised;
//   aggregates: greedy in index order -- a point whose strong neighbours are
//     all free roots a new aggregate with them; leftovers join the aggregate
//     of a strong neighbour; what is still free becomes a singleton;
//   tentative prolongation T (one 1 per row, in the point's aggregate);
//   smoothed prolongation P = (I - w_P D^-1 A) T, w_P = 4 / (3 rho(D^-1 A))
//     (rho by power iteration);
//   R = P^T, A_{l+1} = R A P (Gustavson sparse products);
// until at most AMG_NCOARSE rows remain, whose matrix is inverted densely.
// Everything is deterministic: fixed start vectors, index-ordered loops.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "amg.cuh"

namespace rbffd {

namespace {

constexpr int AMG_NCOARSE = 200;    // coarsest level solved by a dense inverse
constexpr int AMG_NCOARSE_MAX = 600;
constexpr double AMG_THETA = 0.08;  // strength threshold
constexpr double AMG_OMEGA = 2.0 / 3.0;

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
  A.col.reserve((size_t)n * q);
  A.val.reserve((size_t)n * q);
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j < q; ++j) {
      const size_t e = (size_t)j * ldn + i;
      const int c = col[e];
      const double v = val[e];
      if (v == 0.0 && c != i) continue;  // identity rows store zero weights
      A.col.push_back(c);
      A.val.push_back(v);
    }
    A.ptr[i + 1] = (int32_t)A.col.size();
  }
  return A;
}

std::vector<double> diagonal(const Csr &A) {
  std::vector<double> d(A.n, 0.0);
  for (int i = 0; i < A.n; ++i)
    for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k)
      if (A.col[k] == i) d[i] += A.val[k];
  return d;
}

// |lambda|max of D^-1 A by 15 power steps from a fixed non-constant start
double rho_estimate(const Csr &A, const std::vector<double> &dinv) {
  std::vector<double> x(A.n), y(A.n);
  for (int i = 0; i < A.n; ++i) x[i] = 1.0 + 0.5 * (double)((i * 7919) % 13) / 13.0;
  double lam = 1.0;
  for (int it = 0; it < 15; ++it) {
    double nx = 0.0, ny = 0.0;
    for (int i = 0; i < A.n; ++i) {
      double s = 0.0;
      for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k) s += A.val[k] * x[A.col[k]];
      y[i] = dinv[i] * s;
      nx += x[i] * x[i];
      ny += y[i] * y[i];
    }
    if (!(ny > 0.0)) break;
    lam = std::sqrt(ny / nx);
    const double sc = 1.0 / std::sqrt(ny);
    for (int i = 0; i < A.n; ++i) x[i] = y[i] * sc;
  }
  return lam;
}

// symmetric strength graph as adjacency lists (sorted, unique)
void strength(const Csr &A, double theta, std::vector<int32_t> &sp, std::vector<int32_t> &sc) {
  const int n = A.n;
  std::vector<double> mx(n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k)
      if (A.col[k] != i) mx[i] = std::max(mx[i], std::fabs(A.val[k]));
  auto strong = [&](int i, int k) {
    const int j = A.col[k];
    return j != i && mx[i] > 0.0 && std::fabs(A.val[k]) >= theta * mx[i];
  };
  std::vector<int32_t> cnt(n + 1, 0);
  for (int i = 0; i < n; ++i)
    for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k)
      if (strong(i, k)) {
        cnt[i]++;
        cnt[A.col[k]]++;
      }
  sp.assign(n + 1, 0);
  for (int i = 0; i < n; ++i) sp[i + 1] = sp[i] + cnt[i];
  sc.assign(sp[n], 0);
  std::vector<int32_t> fill(sp.begin(), sp.end() - 1);
  for (int i = 0; i < n; ++i)
    for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k)
      if (strong(i, k)) {
        const int j = A.col[k];
        sc[fill[i]++] = j;
        sc[fill[j]++] = i;
      }
  // sort and deduplicate each list, then compact
  int w = 0;
  std::vector<int32_t> np(n + 1, 0);
  for (int i = 0; i < n; ++i) {
    auto b = sc.begin() + sp[i], e = sc.begin() + sp[i + 1];
    std::sort(b, e);
    auto u = std::unique(b, e);
    for (auto it = b; it != u; ++it) sc[w++] = *it;
    np[i + 1] = w;
  }
  sc.resize(w);
  sp.swap(np);
}

// greedy aggregation; returns the number of aggregates
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
  Csr P;
  P.n = A.n;
  P.m = na;
  P.ptr.assign(A.n + 1, 0);
  std::vector<int32_t> mark(na, -1), cols;
  std::vector<double> acc(na, 0.0);
  for (int i = 0; i < A.n; ++i) {
    cols.clear();
    auto add = [&](int c, double v) {
      if (mark[c] != i) {
        mark[c] = i;
        acc[c] = 0.0;
        cols.push_back(c);
      }
      acc[c] += v;
    };
    add(agg[i], 1.0);
    for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k) add(agg[A.col[k]], -w * dinv[i] * A.val[k]);
    for (int c : cols)
      if (acc[c] != 0.0) {
        P.col.push_back(c);
        P.val.push_back(acc[c]);
      }
    P.ptr[i + 1] = (int32_t)P.col.size();
  }
  return P;
}

Csr transpose(const Csr &A) {
  Csr T;
  T.n = A.m;
  T.m = A.n;
  T.ptr.assign(A.m + 1, 0);
  for (int32_t c : A.col) T.ptr[c + 1]++;
  for (int i = 0; i < A.m; ++i) T.ptr[i + 1] += T.ptr[i];
  T.col.resize(A.col.size());
  T.val.resize(A.val.size());
  std::vector<int32_t> fill(T.ptr.begin(), T.ptr.end() - 1);
  for (int i = 0; i < A.n; ++i)
    for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k) {
      const int f = fill[A.col[k]]++;
      T.col[f] = i;
      T.val[f] = A.val[k];
    }
  return T;
}

// C = A B (Gustavson, dense accumulator over B's columns)
Csr spgemm(const Csr &A, const Csr &B) {
  Csr C;
  C.n = A.n;
  C.m = B.m;
  C.ptr.assign(A.n + 1, 0);
  std::vector<int32_t> mark(B.m, -1), cols;
  std::vector<double> acc(B.m, 0.0);
  for (int i = 0; i < A.n; ++i) {
    cols.clear();
    for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k) {
      const int r = A.col[k];
      const double a = A.val[k];
      for (int t = B.ptr[r]; t < B.ptr[r + 1]; ++t) {
        const int c = B.col[t];
        if (mark[c] != i) {
          mark[c] = i;
          acc[c] = 0.0;
          cols.push_back(c);
        }
        acc[c] += a * B.val[t];
      }
    }
    for (int c : cols) {
      C.col.push_back(c);
      C.val.push_back(acc[c]);
    }
    C.ptr[i + 1] = (int32_t)C.col.size();
  }
  return C;
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

struct Staging {
  std::vector<char> buf;
  size_t take(size_t bytes) {
    size_t at = buf.size();
    buf.resize(at + (bytes + 255) / 256 * 256, 0);
    return at;
  }
  template <typename T>
  size_t put(const std::vector<T> &v) {
    size_t at = take(v.size() * sizeof(T));
    if (!v.empty()) memcpy(buf.data() + at, v.data(), v.size() * sizeof(T));
    return at;
  }
};

}  // namespace

int amg_build(rbffd_ctx *ctx, int n, int q, int ldn, const int32_t *col, const double *val,
              void **mem, size_t *bytes, const AmgDev **dev, AmgDev *host_view, AmgInfo *info) {
  *mem = nullptr;
  *bytes = 0;
  *dev = nullptr;
  std::vector<int32_t> hcol((size_t)q * ldn);
  std::vector<double> hval((size_t)q * ldn);
  RBFFD_CK(cudaMemcpyAsync(hcol.data(), col, hcol.size() * 4, cudaMemcpyDeviceToHost,
                           ctx->stream));
  RBFFD_CK(cudaMemcpyAsync(hval.data(), val, hval.size() * 8, cudaMemcpyDeviceToHost,
                           ctx->stream));
  RBFFD_CK(cudaStreamSynchronize(ctx->stream));

  std::vector<Csr> As, Ps, Rs;
  std::vector<std::vector<double>> W;  // smoother weight / diagonal per level
  std::vector<double> omegas;
  As.push_back(from_ell(n, q, ldn, hcol, hval));
  for (;;) {
    const Csr &A = As.back();
    std::vector<double> d = diagonal(A), dinv(A.n);
    for (int i = 0; i < A.n; ++i) dinv[i] = d[i] != 0.0 ? 1.0 / d[i] : 0.0;
    const double lam = rho_estimate(A, dinv);
    const double om = std::min(AMG_OMEGA, 4.0 / (3.0 * lam));
    std::vector<double> wd(A.n);
    for (int i = 0; i < A.n; ++i) wd[i] = om * dinv[i];
    W.push_back(wd);
    omegas.push_back(om);
    if (A.n <= AMG_NCOARSE || (int)As.size() == AMG_MAXLEV) break;
    std::vector<int32_t> sp, sc, agg;
    strength(A, AMG_THETA, sp, sc);
    const int na = aggregate(A.n, sp, sc, agg);
    if (na > 0.8 * A.n || na == 0) break;  // coarsening stalled
    Csr P = smoothed_prolongator(A, dinv, agg, na, 4.0 / (3.0 * lam));
    Csr R = transpose(P);
    Csr AP = spgemm(A, P);
    Csr Ac = spgemm(R, AP);
    Ps.push_back(std::move(P));
    Rs.push_back(std::move(R));
    As.push_back(std::move(Ac));
  }
  const int L = (int)As.size();
  if (As.back().n > AMG_NCOARSE_MAX) {
    set_error("amg: coarsening stalled at %d rows", As.back().n);
    return RBFFD_ENOTIMPL;
  }
  std::vector<double> cinv;
  if (!dense_inverse(As.back(), cinv)) {
    set_error("amg: the coarsest matrix (%d rows) is singular", As.back().n);
    return RBFFD_ESINGULAR;
  }

  // ---- pack everything into one staging buffer, then one upload
  Staging S;
  const size_t o_dev = S.take(sizeof(AmgDev));
  struct Off {
    size_t a_ptr = 0, a_col = 0, a_val = 0, wd = 0, p_ptr = 0, p_col = 0, p_val = 0, r_ptr = 0,
           r_col = 0, r_val = 0, x = 0, b = 0, y = 0;
  };
  std::vector<Off> off(L);
  for (int l = 0; l < L; ++l) {
    if (l > 0) {
      off[l].a_ptr = S.put(As[l].ptr);
      off[l].a_col = S.put(As[l].col);
      off[l].a_val = S.put(As[l].val);
    }
    off[l].wd = S.put(W[l]);
    if (l + 1 < L) {
      off[l].p_ptr = S.put(Ps[l].ptr);
      off[l].p_col = S.put(Ps[l].col);
      off[l].p_val = S.put(Ps[l].val);
      off[l].r_ptr = S.put(Rs[l].ptr);
      off[l].r_col = S.put(Rs[l].col);
      off[l].r_val = S.put(Rs[l].val);
    }
    off[l].x = S.take(sizeof(double) * As[l].n);
    if (l > 0) off[l].b = S.take(sizeof(double) * As[l].n);
    off[l].y = S.take(sizeof(double) * As[l].n);
  }
  const size_t o_cinv = S.put(cinv);
  void *dmem = nullptr;
  RBFFD_TRY(dev_alloc(ctx, &dmem, S.buf.size()));
  char *base = (char *)dmem;
  AmgDev h;
  memset(&h, 0, sizeof(h));
  h.nlev = L;
  h.cinv = (const double *)(base + o_cinv);
  for (int l = 0; l < L; ++l) {
    AmgLevel &v = h.lev[l];
    v.n = As[l].n;
    if (l > 0) {
      v.a_ptr = (const int32_t *)(base + off[l].a_ptr);
      v.a_col = (const int32_t *)(base + off[l].a_col);
      v.a_val = (const double *)(base + off[l].a_val);
      v.b = (double *)(base + off[l].b);
    }
    v.wdinv = (const double *)(base + off[l].wd);
    if (l + 1 < L) {
      v.p_ptr = (const int32_t *)(base + off[l].p_ptr);
      v.p_col = (const int32_t *)(base + off[l].p_col);
      v.p_val = (const double *)(base + off[l].p_val);
      v.r_ptr = (const int32_t *)(base + off[l].r_ptr);
      v.r_col = (const int32_t *)(base + off[l].r_col);
      v.r_val = (const double *)(base + off[l].r_val);
    }
    v.x = (double *)(base + off[l].x);
    v.y = (double *)(base + off[l].y);
  }
  memcpy(S.buf.data() + o_dev, &h, sizeof(h));
  if (cudaMemcpyAsync(dmem, S.buf.data(), S.buf.size(), cudaMemcpyHostToDevice, ctx->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
    dev_free(ctx, dmem, S.buf.size());
    set_error("amg: upload failed");
    return RBFFD_ECUDA;
  }
  *mem = dmem;
  *bytes = S.buf.size();
  *dev = (const AmgDev *)(base + o_dev);
  if (host_view) *host_view = h;
  if (info) {
    memset(info, 0, sizeof(*info));
    info->nlev = L;
    for (int l = 0; l < L; ++l) {
      info->n[l] = As[l].n;
      info->nnz[l] = As[l].nnz();
      info->nnz_p[l] = l + 1 < L ? Ps[l].nnz() : 0;
      info->omega[l] = omegas[l];
    }
  }
  return RBFFD_OK;
}

}  // namespace rbffd
