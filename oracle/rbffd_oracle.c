/*
 * rbffd_oracle.c -- plain, slow, FP64 CPU oracle for the semi-implicit
 * PHS-RBF-FD Navier-Stokes method of Shahane & Vanka (arXiv 2106.07616).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness reference that the
 * CUDA path is compared against.  Only the test suite, the smoke check and
 * the benchmark's CPU-baseline leg may load it; the product library never
 * links, includes or calls it, and shares no code with it.
 *
 * Written for a reader who checks it against the paper by eye:
 *   - no blocking, fusion or reordering beyond what the paper states;
 *   - every dot product is a serial loop in index order;
 *   - compiled with -ffp-contract=off so a*b+c is two roundings, exactly
 *     as written.
 *
 * Sections of the paper followed (each function names its own):
 *   Sec. 2, Eq. (RBF_interp)..(RBF_interp_mat_vec_L_solve): PHS r^3 +
 *       polynomial collocation and the operator weights B1.
 *   Sec. 3, Eqs. (u:tilde), (v:tilde), (pressure poisson), (u:correction),
 *       (v:correction), (p:correction): one outer iteration.
 *   Sec. 3.1, Eq. (normal momentum): boundary pressure and p' Neumann rows.
 *   Sec. 3.2 "Summary of Solution Steps": step order of the outer loop and
 *       the adaptive outer tolerance min(1e-4, dt*eps_s).
 *
 * Readings where the paper is silent:
 *   - cloud = the q nearest points, self first, others by (d^2, index);
 *   - local coordinates shifted to the centre and scaled by the stencil
 *     radius h = max |x_j - x_c| (weights are invariant in exact arithmetic);
 *   - "direct linear solver" = LU with partial pivoting, lowest row wins a
 *     pivot tie, column-oriented back substitution;
 *   - "preconditioned BiCGSTAB" = right-Jacobi BiCGSTAB (van der Vorst 1992);
 *   - Delta = mean|u^{r+1}-u^r| + mean|v^{r+1}-v^r|;
 *   - the cloud of a boundary point = itself + its nearest interior points;
 *   - p' pinned (identity row, zero RHS) at one boundary point, in place of
 *     its Neumann row;
 *   - boundary pressure: one Jacobi sweep of the normal-momentum equation,
 *     convection/diffusion on (u~, v~), BDF2 time derivative of the boundary
 *     value.
 *
 * Parity pins for every function here live in tests/test_oracle_*.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL -1
#define ORC_ENOMEM -2
#define ORC_ESINGULAR -3
#define ORC_ENOCONV -4
#define ORC_EDIVERGED -5

#define TAG_INTERIOR 0
#define TAG_DIRICHLET 1 /* wall / inlet: u, v prescribed */
#define TAG_OUTFLOW 2   /* fixed-pressure outlet: p held, p' = 0, du/dn = dv/dn = 0 */
#define TAG_SYMMETRY 3  /* symmetry line: normal velocity prescribed, tangential d/dn = 0 */

/* ------------------------------------------------------------------------ */
/* Sec. 2, below Eq. (RBF_interp_poly): m = C(k+d, k) monomials for d = 2.   */
int orc_num_monomials(int degree) { return (degree + 1) * (degree + 2) / 2; }

/* Graded monomial order of Eq. (RBF_interp_poly): total degree 0..k, and
 * inside one degree the x power descends: 1, x, y, x^2, xy, y^2, x^3, ...   */
void orc_monomial_exponents(int degree, int32_t *ax, int32_t *ay) {
  int l = 0;
  for (int d = 0; d <= degree; ++d)
    for (int a = d; a >= 0; --a) {
      ax[l] = a;
      ay[l] = d - a;
      ++l;
    }
}

static double ipow_seq(double base, int e) {
  double v = 1.0;
  for (int t = 0; t < e; ++t) v = v * base;
  return v;
}

/* ------------------------------------------------------------------------ */
/* Cloud selection (Sec. 2: "a cloud of neighboring points"; Sec. 3.1: only */
/* one-sided clouds are used at boundaries).  Brute force over all points.  */
/* The point itself comes first; the other q-1 members are the nearest      */
/* candidates in the order (d^2, index), d^2 = dx*dx + dy*dy without fusion. */
/* Candidates of an interior point: every other point.  Candidates of a     */
/* boundary point (tag != 0): the interior points only, which makes its     */
/* cloud one-sided.  tag == NULL treats every point as interior.            */
static int key_less(double d2a, int ja, double d2b, int jb) {
  return d2a < d2b || (d2a == d2b && ja < jb);
}

/* a - b along an axis that is periodic with length L (L = 0: not          */
/* periodic): the difference moved by one period when it exceeds half of   */
/* one, i.e. the nearest image (Sec. 3.1: clouds wrap around a periodic    */
/* boundary).                                                              */
static double pdiff(double a, double b, double L) {
  double d = a - b;
  if (L > 0.0) {
    if (d > 0.5 * L) d = d - L;
    else if (d < -0.5 * L) d = d + L;
  }
  return d;
}

/* The cloud of point i into out[0..q-1]; bd, bj: work arrays of q-1.     */
static void knn_one(int n, const double *x, const double *y, const int8_t *tag, int q, int i,
                    const double *per, double *bd, int *bj, int32_t *out) {
  int boundary = tag && tag[i] != TAG_INTERIOR;
  int cnt = 0;
  for (int j = 0; j < n; ++j) {
    if (j == i) continue;
    if (boundary && tag[j] != TAG_INTERIOR) continue;
    double dx = pdiff(x[j], x[i], per ? per[0] : 0.0);
    double dy = pdiff(y[j], y[i], per ? per[1] : 0.0);
    double d2 = dx * dx + dy * dy;
    /* keep the q-1 best in a sorted list (insertion) */
    if (cnt < q - 1) {
      int s = cnt++;
      while (s > 0 && key_less(d2, j, bd[s - 1], bj[s - 1])) {
        bd[s] = bd[s - 1]; bj[s] = bj[s - 1]; --s;
      }
      bd[s] = d2; bj[s] = j;
    } else if (q > 1 && key_less(d2, j, bd[q - 2], bj[q - 2])) {
      int s = q - 2;
      while (s > 0 && key_less(d2, j, bd[s - 1], bj[s - 1])) {
        bd[s] = bd[s - 1]; bj[s] = bj[s - 1]; --s;
      }
      bd[s] = d2; bj[s] = j;
    }
  }
  out[0] = i;
  for (int s = 0; s < q - 1; ++s) out[1 + s] = bj[s];
}

/* Clouds of the points rows[0..nrows-1] (all points when rows == NULL,     */
/* nrows = n), written row by row to idx (nrows x q).                       */
static int knn_rows(int n, const double *x, const double *y, const int8_t *tag, int q,
                    int nrows, const int32_t *rows, const double *per, int32_t *idx) {
  if (n <= 0 || q <= 0 || q > n || nrows < 0) return ORC_EINVAL;
  int n_int = 0;
  for (int j = 0; j < n; ++j) n_int += (!tag || tag[j] == TAG_INTERIOR);
  int any_bnd = n_int < n;
  if (any_bnd && q - 1 > n_int) return ORC_EINVAL;
  if (rows)
    for (int k = 0; k < nrows; ++k)
      if (rows[k] < 0 || rows[k] >= n) return ORC_EINVAL;
  int status = ORC_OK;
#pragma omp parallel
  {
  double *bd = (double *)malloc(sizeof(double) * q);
  int *bj = (int *)malloc(sizeof(int) * q);
  if (!bd || !bj) {
#pragma omp atomic write
    status = ORC_ENOMEM;
  }
#pragma omp for schedule(dynamic, 64)
  for (int k = 0; k < nrows; ++k) {
    if (!bd || !bj) continue;
    knn_one(n, x, y, tag, q, rows ? rows[k] : k, per, bd, bj, idx + (int64_t)k * q);
  }
  free(bd); free(bj);
  }
  return status;
}

int orc_knn(int n, const double *x, const double *y, const int8_t *tag, int q, int32_t *idx) {
  return knn_rows(n, x, y, tag, q, n, NULL, NULL, idx);
}

/* Clouds of selected points only (spot checks of large problems). */
int orc_knn_rows(int n, const double *x, const double *y, const int8_t *tag, int q, int nrows,
                 const int32_t *rows, int32_t *idx) {
  return knn_rows(n, x, y, tag, q, nrows, rows, NULL, idx);
}

/* ------------------------------------------------------------------------ */
/* Dense LU with partial pivoting on an augmented matrix M (n rows, n+nr    */
/* columns, row-major, leading dimension ld).  Doolittle elimination; the   */
/* pivot is the largest |a| in the column, lowest row on a tie; an exactly  */
/* zero pivot is singular.  The nr right-hand sides are eliminated with the */
/* matrix and then back-substituted column by column.  Returns 0 or -1.     */
int orc_lu_solve(int n, int nr, double *M, int ld, double *sol /* n*nr, col-major by rhs */) {
  for (int k = 0; k < n; ++k) {
    int piv = k;
    double best = fabs(M[(int64_t)k * ld + k]);
    for (int i = k + 1; i < n; ++i) {
      double a = fabs(M[(int64_t)i * ld + k]);
      if (a > best) { best = a; piv = i; }
    }
    if (best == 0.0) return -1;
    if (piv != k)
      for (int j = 0; j < n + nr; ++j) {
        double t = M[(int64_t)k * ld + j];
        M[(int64_t)k * ld + j] = M[(int64_t)piv * ld + j];
        M[(int64_t)piv * ld + j] = t;
      }
    double akk = M[(int64_t)k * ld + k];
    for (int i = k + 1; i < n; ++i) {
      double l = M[(int64_t)i * ld + k] / akk;
      M[(int64_t)i * ld + k] = l;
      for (int j = k + 1; j < n + nr; ++j)
        M[(int64_t)i * ld + j] = M[(int64_t)i * ld + j] - l * M[(int64_t)k * ld + j];
    }
  }
  /* column-oriented back substitution U c = b' */
  for (int r = 0; r < nr; ++r) {
    double *c = sol + (int64_t)r * n;
    for (int i = 0; i < n; ++i) c[i] = M[(int64_t)i * ld + n + r];
    for (int j = n - 1; j >= 0; --j) {
      c[j] = c[j] / M[(int64_t)j * ld + j];
      for (int i = 0; i < j; ++i) c[i] = c[i] - M[(int64_t)i * ld + j] * c[j];
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Operator weights of one cloud, Sec. 2 Eqs. (RBF_interp_mat_vec) to        */
/* (RBF_interp_mat_vec_L_solve).  A = [Phi P; P^T 0] is symmetric, so the    */
/* row vector B = [L(Phi) L(P)] A^{-1} evaluated at the centre is the        */
/* transpose of the solution of A c = [L phi(|x_c - x_j|)]_j ++ [L P(x_c)];  */
/* B1 = its first q entries.  Local coordinates: xi = (x - x_c)/h with       */
/* h = max_j |x_j - x_c|; d/dx = (1/h) d/dxi, Laplacian = (1/h^2) that of xi. */
/* phi = r^3:  d/dxi phi(|xi - xi_j|) at xi = 0 is 3 r_j (0 - xi_j);         */
/*             the 2-D Laplacian of r^3 is 9 r.                              */
/* ops: bit 1 = d/dx, bit 2 = d/dy, bit 4 = Laplacian.                       */
/* One cloud: centre i, members cl[0..q-1].  Work arrays M (N*(N+3)),       */
/* sol (3N), xi, eta (q).  Returns 0, or -1 on an exactly zero pivot.        */
static int weights_one(const double *x, const double *y, int q, const int32_t *cl, int i, int m,
                       const int32_t *ax, const int32_t *ay, const double *per, double *M,
                       double *sol, double *xi, double *eta, double *wx, double *wy, double *wl) {
  int N = q + m, ld = N + 3;
  double xc = x[i], yc = y[i];
  double Lx = per ? per[0] : 0.0, Ly = per ? per[1] : 0.0;
  /* stencil radius (members at their nearest periodic image) */
  double d2max = 0.0;
  for (int a = 0; a < q; ++a) {
    double dx = pdiff(x[cl[a]], xc, Lx), dy = pdiff(y[cl[a]], yc, Ly);
    double d2 = dx * dx + dy * dy;
    if (d2 > d2max) d2max = d2;
  }
  double h = sqrt(d2max);
  if (h == 0.0) h = 1.0; /* a one-point cloud: nothing to scale */
  for (int a = 0; a < q; ++a) {
    xi[a] = pdiff(x[cl[a]], xc, Lx) / h;
    eta[a] = pdiff(y[cl[a]], yc, Ly) / h;
  }
  /* A = [Phi P; P^T 0] with the three right-hand sides appended */
  for (int a = 0; a < q; ++a) {
    for (int b = 0; b < q; ++b) {
      double dx = xi[a] - xi[b], dy = eta[a] - eta[b];
      double r = sqrt(dx * dx + dy * dy);
      M[(int64_t)a * ld + b] = r * r * r;
    }
    for (int l = 0; l < m; ++l) {
      double pv = ipow_seq(xi[a], ax[l]) * ipow_seq(eta[a], ay[l]);
      M[(int64_t)a * ld + q + l] = pv;
      M[(int64_t)(q + l) * ld + a] = pv;
    }
    double rj = sqrt(xi[a] * xi[a] + eta[a] * eta[a]);
    M[(int64_t)a * ld + N + 0] = 3.0 * rj * (0.0 - xi[a]);
    M[(int64_t)a * ld + N + 1] = 3.0 * rj * (0.0 - eta[a]);
    M[(int64_t)a * ld + N + 2] = 9.0 * rj;
  }
  for (int l = 0; l < m; ++l) {
    for (int b = 0; b < m; ++b) M[(int64_t)(q + l) * ld + q + b] = 0.0;
    M[(int64_t)(q + l) * ld + N + 0] = (ax[l] == 1 && ay[l] == 0) ? 1.0 : 0.0;
    M[(int64_t)(q + l) * ld + N + 1] = (ax[l] == 0 && ay[l] == 1) ? 1.0 : 0.0;
    M[(int64_t)(q + l) * ld + N + 2] =
        ((ax[l] == 2 && ay[l] == 0) || (ax[l] == 0 && ay[l] == 2)) ? 2.0 : 0.0;
  }
  if (orc_lu_solve(N, 3, M, ld, sol) != 0) {
    for (int a = 0; a < q; ++a) {
      if (wx) wx[a] = 0.0;
      if (wy) wy[a] = 0.0;
      if (wl) wl[a] = 0.0;
    }
    return -1;
  }
  double h2 = h * h;
  for (int a = 0; a < q; ++a) {
    if (wx) wx[a] = sol[a] / h;
    if (wy) wy[a] = sol[N + a] / h;
    if (wl) wl[a] = sol[2 * N + a] / h2;
  }
  return 0;
}

static int weights_rows(int n, const double *x, const double *y, int q, int nrows,
                        const int32_t *rows, const int32_t *idx, int degree, const double *per,
                        double *wx, double *wy, double *wl, int32_t *first_singular);

int orc_weights(int n, const double *x, const double *y, int q, const int32_t *idx,
                int degree, double *wx, double *wy, double *wl, int32_t *first_singular) {
  return weights_rows(n, x, y, q, n, NULL, idx, degree, NULL, wx, wy, wl, first_singular);
}

/* Weights of the clouds idx (nrows x q) centred at rows[k] (spot checks of */
/* large problems); first_singular reports the position k.                 */
int orc_weights_rows(int n, const double *x, const double *y, int q, int nrows,
                     const int32_t *rows, const int32_t *idx, int degree, double *wx, double *wy,
                     double *wl, int32_t *first_singular) {
  return weights_rows(n, x, y, q, nrows, rows, idx, degree, NULL, wx, wy, wl, first_singular);
}

static int weights_rows(int n, const double *x, const double *y, int q, int nrows,
                        const int32_t *rows, const int32_t *idx, int degree, const double *per,
                        double *wx, double *wy, double *wl, int32_t *first_singular) {
  int m = orc_num_monomials(degree);
  if (n <= 0 || q <= 0 || q > n || degree < 0 || q < m || nrows < 0) return ORC_EINVAL;
  int N = q + m;
  int32_t ax[64], ay[64];
  if (m > 64) return ORC_EINVAL;
  orc_monomial_exponents(degree, ax, ay);
  int status = ORC_OK, sing = -1;
#pragma omp parallel
  {
  double *M = (double *)malloc(sizeof(double) * (size_t)N * (N + 3));
  double *sol = (double *)malloc(sizeof(double) * (size_t)N * 3);
  double *xi = (double *)malloc(sizeof(double) * q);
  double *eta = (double *)malloc(sizeof(double) * q);
  int ok = M && sol && xi && eta;
  if (!ok) {
#pragma omp atomic write
    status = ORC_ENOMEM;
  }
#pragma omp for schedule(dynamic, 16)
  for (int i = 0; i < nrows; ++i) {
    if (!ok) continue;
    int64_t o = (int64_t)i * q;
    if (weights_one(x, y, q, idx + o, rows ? rows[i] : i, m, ax, ay, per, M, sol, xi, eta, wx ? wx + o : NULL,
                    wy ? wy + o : NULL, wl ? wl + o : NULL) != 0) {
#pragma omp critical(orc_singular)
      {
        if (sing < 0 || i < sing) sing = i;
      }
    }
  }
  free(M); free(sol); free(xi); free(eta);
  }
  if (first_singular) *first_singular = sing;
  if (status == ORC_OK && sing >= 0) status = ORC_ESINGULAR;
  return status;
}

/* ------------------------------------------------------------------------ */
/* CSR sparse matrix and y = A x (row order, serial sum in stored order).    */
typedef struct {
  int n;
  int64_t *rowptr;
  int32_t *col;
  double *val;
} csr_t;

static void csr_spmv(const csr_t *A, const double *xv, double *yv) {
#pragma omp parallel for schedule(static) if (A->n > 8192)
  for (int i = 0; i < A->n; ++i) {
    double s = 0.0;
    for (int64_t e = A->rowptr[i]; e < A->rowptr[i + 1]; ++e) s = s + A->val[e] * xv[A->col[e]];
    yv[i] = s;
  }
}

static double dot(int n, const double *a, const double *b) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) s = s + a[i] * b[i];
  return s;
}

/* ------------------------------------------------------------------------ */
/* Right-Jacobi-preconditioned BiCGSTAB (van der Vorst 1992), used by the    */
/* paper for both the momentum and the pressure-correction systems (Sec. 3). */
/* Stops when |r|_2 <= tol |b|_2, checked on s (half step) and on r.  On a   */
/* breakdown (rho == 0 or omega == 0) it restarts from the current x, at    */
/* most 3 times.  x holds the initial guess on entry.                       */
typedef struct {
  int iters;
  int restarts;
  double relres;
} krylov_stats_t;

static int bicgstab(const csr_t *A, const double *b, double *xv, double tol, int maxit,
                    krylov_stats_t *st) {
  int n = A->n;
  double *dg = (double *)malloc(sizeof(double) * n);
  double *r = (double *)malloc(sizeof(double) * n);
  double *rh = (double *)malloc(sizeof(double) * n);
  double *p = (double *)malloc(sizeof(double) * n);
  double *v = (double *)malloc(sizeof(double) * n);
  double *ph = (double *)malloc(sizeof(double) * n);
  double *s = (double *)malloc(sizeof(double) * n);
  double *sh = (double *)malloc(sizeof(double) * n);
  double *t = (double *)malloc(sizeof(double) * n);
  int ret = ORC_ENOCONV;
  st->iters = 0; st->restarts = 0; st->relres = 0.0;
  if (!dg || !r || !rh || !p || !v || !ph || !s || !sh || !t) { ret = ORC_ENOMEM; goto done; }
  for (int i = 0; i < n; ++i) {
    dg[i] = 0.0;
    for (int64_t e = A->rowptr[i]; e < A->rowptr[i + 1]; ++e)
      if (A->col[e] == i) dg[i] = dg[i] + A->val[e];
    if (dg[i] == 0.0) dg[i] = 1.0;
  }
  double bnorm = sqrt(dot(n, b, b));
  if (bnorm == 0.0) {
    for (int i = 0; i < n; ++i) xv[i] = 0.0;
    ret = ORC_OK;
    goto done;
  }
  for (;;) { /* (re)start */
    csr_spmv(A, xv, r);
    for (int i = 0; i < n; ++i) r[i] = b[i] - r[i];
    double rnorm = sqrt(dot(n, r, r));
    st->relres = rnorm / bnorm;
    if (!(st->relres == st->relres)) { ret = ORC_EDIVERGED; goto done; }
    if (st->relres <= tol) { ret = ORC_OK; goto done; }
    for (int i = 0; i < n; ++i) { rh[i] = r[i]; p[i] = 0.0; v[i] = 0.0; }
    double rho_prev = 1.0, alpha = 1.0, omega = 1.0;
    int first = 1, broke = 0;
    while (st->iters < maxit) {
      double rho = dot(n, rh, r);
      if (rho == 0.0) { broke = 1; break; }
      if (first) {
        for (int i = 0; i < n; ++i) p[i] = r[i];
        first = 0;
      } else {
        double beta = (rho / rho_prev) * (alpha / omega);
        for (int i = 0; i < n; ++i) p[i] = r[i] + beta * (p[i] - omega * v[i]);
      }
      for (int i = 0; i < n; ++i) ph[i] = p[i] / dg[i];
      csr_spmv(A, ph, v);
      alpha = rho / dot(n, rh, v);
      for (int i = 0; i < n; ++i) s[i] = r[i] - alpha * v[i];
      st->iters++;
      double snorm = sqrt(dot(n, s, s));
      if (!(snorm == snorm)) { ret = ORC_EDIVERGED; goto done; }
      if (snorm / bnorm <= tol) {
        for (int i = 0; i < n; ++i) xv[i] = xv[i] + alpha * ph[i];
        st->relres = snorm / bnorm;
        ret = ORC_OK;
        goto done;
      }
      for (int i = 0; i < n; ++i) sh[i] = s[i] / dg[i];
      csr_spmv(A, sh, t);
      double tt = dot(n, t, t);
      omega = tt == 0.0 ? 0.0 : dot(n, t, s) / tt;
      for (int i = 0; i < n; ++i) xv[i] = xv[i] + alpha * ph[i] + omega * sh[i];
      for (int i = 0; i < n; ++i) r[i] = s[i] - omega * t[i];
      rnorm = sqrt(dot(n, r, r));
      st->relres = rnorm / bnorm;
      if (!(rnorm == rnorm)) { ret = ORC_EDIVERGED; goto done; }
      if (st->relres <= tol) { ret = ORC_OK; goto done; }
      if (omega == 0.0) { broke = 1; break; }
      rho_prev = rho;
    }
    if (!broke) { ret = ORC_ENOCONV; goto done; }
    if (st->restarts >= 3) { ret = ORC_ENOCONV; goto done; }
    st->restarts++;
  }
done:
  free(dg); free(r); free(rh); free(p); free(v); free(ph); free(s); free(sh); free(t);
  return ret;
}

/* Stand-alone entry for tests: solve A x = b with A given as CSR. */
int orc_bicgstab_csr(int n, const int64_t *rowptr, const int32_t *col, const double *val,
                     const double *b, double *xv, double tol, int maxit, int32_t *iters,
                     double *relres) {
  csr_t A = {n, (int64_t *)rowptr, (int32_t *)col, (double *)val};
  krylov_stats_t st;
  int rc = bicgstab(&A, b, xv, tol, maxit, &st);
  if (iters) *iters = st.iters;
  if (relres) *relres = st.relres;
  return rc;
}

/* ------------------------------------------------------------------------ */
/* The flow problem.                                                         */
typedef struct {
  int n, q, degree, pin;
  double rho, mu;
  double per[2];   /* periods of x and y (0: not periodic), Sec. 3.1 */
  double force[2]; /* body force per unit volume, e.g. a mean pressure gradient */
  double *x, *y, *nx, *ny, *ubc, *vbc;
  int8_t *tag;
  int32_t *idx;
  double *wx, *wy, *wl;
  int64_t *rowptr;
  csr_t Dx, Dy, Dl, Pp, Am, Av; /* Pp: pressure correction; Am, Av: momentum u, v */
  /* compatibility of the pinned p' equation: left null vector psi of the  */
  /* pure-Neumann operator and psi . e_I (NULL / 0 when an outlet fixes p) */
  double *psi;
  double psi_eI;
  int psi_off; /* 1: compatibility switched off (orc_set_compat) */
  /* fields: iterate (u, v, p) and the two previous time levels */
  double *u, *v, *p, *un, *vn, *unm1, *vnm1;
  /* work */
  double *ut, *vt, *pc, *bu, *bv, *bp, *w1, *w2, *w3, *w4;
  /* Krylov settings */
  double ktol;
  int kmaxit;
} orc_problem;

#define FIELD_U 0
#define FIELD_V 1
#define FIELD_P 2
#define FIELD_UN 3
#define FIELD_VN 4
#define FIELD_UNM1 5
#define FIELD_VNM1 6
#define FIELD_UT 7
#define FIELD_VT 8
#define FIELD_PC 9
#define FIELD_UBC 10
#define FIELD_VBC 11

static double *dvec(int n) { return (double *)calloc((size_t)n, sizeof(double)); }

void orc_problem_destroy(orc_problem *P) {
  if (!P) return;
  free(P->x); free(P->y); free(P->nx); free(P->ny); free(P->ubc); free(P->vbc); free(P->tag);
  free(P->idx); free(P->wx); free(P->wy); free(P->wl); free(P->rowptr);
  free(P->Pp.val); free(P->Am.val); free(P->Av.val); free(P->psi);
  free(P->u); free(P->v); free(P->p); free(P->un); free(P->vn); free(P->unm1); free(P->vnm1);
  free(P->ut); free(P->vt); free(P->pc); free(P->bu); free(P->bv); free(P->bp);
  free(P->w1); free(P->w2); free(P->w3); free(P->w4);
  free(P);
}

/* ------------------------------------------------------------------------ */
/* Solvability of the pressure-correction equation (Sec. 3, Eq. (pressure   */
/* poisson) with the homogeneous Neumann rows of Sec. 3.1).  With Neumann   */
/* rows only (no outlet) the discrete operator L_N -- Laplacian weights at  */
/* interior rows, n.grad weights at boundary rows -- maps constants to zero */
/* (every row of weights sums to zero), so it is singular, and L_N p' = b  */
/* has a solution only when psi . b = 0 for the left null vector psi       */
/* (psi^T L_N = 0).  This is the discrete form of the condition that the    */
/* source of a Neumann problem integrate to the prescribed boundary flux   */
/* (zero here).  The divergence of u~ does not meet it exactly, so the      */
/* source is made compatible before the solve:                             */
/*     b~ = b - (psi . b / psi . e_I) e_I,   e_I = 1 at interior rows,      */
/* i.e. the part of the divergence that no pressure correction can remove  */
/* is a constant lambda over the interior rows.  The pin row (identity)     */
/* then only fixes the free constant of p'.                                 */
/* psi is computed once per problem.  With M = L_N with its pin row         */
/* replaced by the identity (the stored p' matrix) and l = the pin's        */
/* Neumann row, psi solves M^T psi = e_pin - l; then psi^T L_N = (1 -      */
/* psi_pin)(e_pin - l)^T, and applying both sides to the constant vector    */
/* (L_N 1 = 0, l . 1 = 0) gives psi_pin = 1, so psi^T L_N = 0.              */
static int compat_vector(orc_problem *P) {
  int n = P->n, q = P->q, pin = P->pin;
  int64_t nnz = (int64_t)n * q;
  /* M^T as CSR: column counts, prefix sums, then entries in row order */
  csr_t T;
  T.n = n;
  T.rowptr = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
  T.col = (int32_t *)malloc(sizeof(int32_t) * (size_t)nnz);
  T.val = (double *)malloc(sizeof(double) * (size_t)nnz);
  double *rhs = dvec(n);
  P->psi = dvec(n);
  int64_t *fill = (int64_t *)calloc((size_t)n, sizeof(int64_t));
  int rc = ORC_OK;
  if (!T.rowptr || !T.col || !T.val || !rhs || !P->psi || !fill) { rc = ORC_ENOMEM; goto out; }
  for (int64_t e = 0; e < nnz; ++e) T.rowptr[P->idx[e] + 1]++;
  for (int j = 0; j < n; ++j) T.rowptr[j + 1] = T.rowptr[j + 1] + T.rowptr[j];
  for (int i = 0; i < n; ++i)
    for (int64_t e = P->rowptr[i]; e < P->rowptr[i + 1]; ++e) {
      int j = P->idx[e];
      int64_t slot = T.rowptr[j] + fill[j]++;
      T.col[slot] = i;
      T.val[slot] = P->Pp.val[e];
    }
  /* right-hand side e_pin - l, l = n.grad weights of the pin's cloud */
  rhs[pin] = 1.0;
  for (int64_t e = P->rowptr[pin]; e < P->rowptr[pin + 1]; ++e)
    rhs[P->idx[e]] = rhs[P->idx[e]] - (P->nx[pin] * P->wx[e] + P->ny[pin] * P->wy[e]);
  krylov_stats_t st;
  rc = bicgstab(&T, rhs, P->psi, P->ktol, P->kmaxit, &st);
  if (rc) goto out;
  P->psi_eI = 0.0;
  for (int i = 0; i < n; ++i)
    if (P->tag[i] == TAG_INTERIOR) P->psi_eI = P->psi_eI + P->psi[i];
  if (P->psi_eI == 0.0) rc = ORC_ESINGULAR;
out:
  free(T.rowptr); free(T.col); free(T.val); free(rhs); free(fill);
  return rc;
}

/* Build stencils, weights, the operator CSR matrices and the pressure-      */
/* correction matrix (Sec. 3.1): interior rows = Laplacian weights; rows at  */
/* walls, inlets and symmetry lines = homogeneous Neumann n.grad p' = 0,     */
/* i.e. nx*Wx + ny*Wy; rows at fixed-pressure outlets = identity (p' = 0).   */
/* With Neumann rows only, p' is defined up to a constant; the Neumann row  */
/* of one boundary point (pin) is then replaced by the identity with a zero */
/* right-hand side, which fixes that constant.  pin = -1 is allowed when an */
/* outlet point exists.  Symmetry points need an axis-aligned normal (the   */
/* normal velocity component is then u or v).  per[2] (nullable): periods  */
/* of x and y, 0 for a bounded axis -- clouds and weights then use nearest */
/* periodic images (Sec. 3.1, periodic boundaries).  force[2] (nullable):   */
/* a body force added to the momentum equations, the paper's mean pressure */
/* gradient of periodic flows.                                              */
int orc_problem_create2(int n, int q, int degree, const double *x, const double *y,
                        const int8_t *tag, const double *nx, const double *ny,
                        const double *ubc, const double *vbc, int pin, double rho, double mu,
                        const double *per, const double *force, orc_problem **out,
                        int32_t *first_singular);

int orc_problem_create(int n, int q, int degree, const double *x, const double *y,
                       const int8_t *tag, const double *nx, const double *ny, const double *ubc,
                       const double *vbc, int pin, double rho, double mu, orc_problem **out,
                       int32_t *first_singular) {
  return orc_problem_create2(n, q, degree, x, y, tag, nx, ny, ubc, vbc, pin, rho, mu, NULL, NULL,
                             out, first_singular);
}

int orc_problem_create2(int n, int q, int degree, const double *x, const double *y,
                        const int8_t *tag, const double *nx, const double *ny,
                        const double *ubc, const double *vbc, int pin, double rho, double mu,
                        const double *per, const double *force, orc_problem **out,
                        int32_t *first_singular) {
  *out = NULL;
  if (per && (per[0] < 0.0 || per[1] < 0.0)) return ORC_EINVAL;
  int m = orc_num_monomials(degree);
  if (n <= 0 || q <= 0 || q > n || q < m || pin < -1 || pin >= n) return ORC_EINVAL;
  int n_out = 0;
  for (int i = 0; i < n; ++i) {
    if (tag[i] < TAG_INTERIOR || tag[i] > TAG_SYMMETRY) return ORC_EINVAL;
    if (tag[i] == TAG_OUTFLOW) n_out++;
    if (tag[i] == TAG_SYMMETRY && fabs(nx[i]) > 1e-12 && fabs(ny[i]) > 1e-12) return ORC_EINVAL;
  }
  if (pin < 0 && n_out == 0) return ORC_EINVAL;
  if (pin >= 0 && (tag[pin] == TAG_INTERIOR || tag[pin] == TAG_OUTFLOW)) return ORC_EINVAL;
  orc_problem *P = (orc_problem *)calloc(1, sizeof(orc_problem));
  if (!P) return ORC_ENOMEM;
  P->n = n; P->q = q; P->degree = degree; P->pin = pin; P->rho = rho; P->mu = mu;
  P->per[0] = per ? per[0] : 0.0; P->per[1] = per ? per[1] : 0.0;
  P->force[0] = force ? force[0] : 0.0; P->force[1] = force ? force[1] : 0.0;
  P->ktol = 1e-12; P->kmaxit = 10000;
  size_t nq = (size_t)n * q;
  P->x = dvec(n); P->y = dvec(n); P->nx = dvec(n); P->ny = dvec(n);
  P->ubc = dvec(n); P->vbc = dvec(n);
  P->tag = (int8_t *)calloc(n, 1);
  P->idx = (int32_t *)calloc(nq, sizeof(int32_t));
  P->wx = dvec((int)nq); P->wy = dvec((int)nq); P->wl = dvec((int)nq);
  P->rowptr = (int64_t *)calloc(n + 1, sizeof(int64_t));
  double *pval = dvec((int)nq), *mval = dvec((int)nq), *vval = dvec((int)nq);
  P->u = dvec(n); P->v = dvec(n); P->p = dvec(n); P->un = dvec(n); P->vn = dvec(n);
  P->unm1 = dvec(n); P->vnm1 = dvec(n);
  P->ut = dvec(n); P->vt = dvec(n); P->pc = dvec(n); P->bu = dvec(n); P->bv = dvec(n);
  P->bp = dvec(n); P->w1 = dvec(n); P->w2 = dvec(n); P->w3 = dvec(n); P->w4 = dvec(n);
  P->Pp.val = pval; P->Am.val = mval; P->Av.val = vval;
  if (!P->x || !P->y || !P->nx || !P->ny || !P->ubc || !P->vbc || !P->tag || !P->idx ||
      !P->wx || !P->wy || !P->wl || !P->rowptr || !pval || !mval || !vval || !P->u || !P->v ||
      !P->p ||
      !P->un || !P->vn || !P->unm1 || !P->vnm1 || !P->ut || !P->vt || !P->pc || !P->bu ||
      !P->bv || !P->bp || !P->w1 || !P->w2 || !P->w3 || !P->w4) {
    orc_problem_destroy(P);
    return ORC_ENOMEM;
  }
  memcpy(P->x, x, sizeof(double) * n); memcpy(P->y, y, sizeof(double) * n);
  memcpy(P->nx, nx, sizeof(double) * n); memcpy(P->ny, ny, sizeof(double) * n);
  memcpy(P->ubc, ubc, sizeof(double) * n); memcpy(P->vbc, vbc, sizeof(double) * n);
  memcpy(P->tag, tag, (size_t)n);
  int rc = knn_rows(n, P->x, P->y, P->tag, q, n, NULL, P->per, P->idx);
  if (rc) { orc_problem_destroy(P); return rc; }
  rc = weights_rows(n, P->x, P->y, q, n, NULL, P->idx, degree, P->per, P->wx, P->wy, P->wl,
                    first_singular);
  if (rc) { orc_problem_destroy(P); return rc; }
  for (int i = 0; i <= n; ++i) P->rowptr[i] = (int64_t)i * q;
  csr_t base = {n, P->rowptr, P->idx, NULL};
  P->Dx = base; P->Dx.val = P->wx;
  P->Dy = base; P->Dy.val = P->wy;
  P->Dl = base; P->Dl.val = P->wl;
  P->Pp.n = n; P->Pp.rowptr = P->rowptr; P->Pp.col = P->idx;
  P->Am.n = n; P->Am.rowptr = P->rowptr; P->Am.col = P->idx;
  P->Av.n = n; P->Av.rowptr = P->rowptr; P->Av.col = P->idx;
  for (int i = 0; i < n; ++i)
    for (int64_t e = P->rowptr[i]; e < P->rowptr[i + 1]; ++e) {
      double val;
      if (i == pin || tag[i] == TAG_OUTFLOW)
        val = (P->idx[e] == i) ? 1.0 : 0.0;
      else if (tag[i] == TAG_INTERIOR)
        val = P->wl[e];
      else
        val = nx[i] * P->wx[e] + ny[i] * P->wy[e];
      pval[e] = val;
    }
  if (pin >= 0) {
    rc = compat_vector(P);
    if (rc) { orc_problem_destroy(P); return rc; }
  }
  /* initial state: u = v = p = 0 in the interior, BC values on the boundary */
  for (int i = 0; i < n; ++i) {
    double u0 = tag[i] == TAG_INTERIOR ? 0.0 : ubc[i];
    double v0 = tag[i] == TAG_INTERIOR ? 0.0 : vbc[i];
    P->u[i] = P->un[i] = P->unm1[i] = u0;
    P->v[i] = P->vn[i] = P->vnm1[i] = v0;
  }
  *out = P;
  return ORC_OK;
}

static double *field_ptr(orc_problem *P, int which) {
  switch (which) {
    case FIELD_U: return P->u;
    case FIELD_V: return P->v;
    case FIELD_P: return P->p;
    case FIELD_UN: return P->un;
    case FIELD_VN: return P->vn;
    case FIELD_UNM1: return P->unm1;
    case FIELD_VNM1: return P->vnm1;
    case FIELD_UT: return P->ut;
    case FIELD_VT: return P->vt;
    case FIELD_PC: return P->pc;
    case FIELD_UBC: return P->ubc;
    case FIELD_VBC: return P->vbc;
    default: return NULL;
  }
}

int orc_get_field(orc_problem *P, int which, double *out) {
  double *f = field_ptr(P, which);
  if (!f) return ORC_EINVAL;
  memcpy(out, f, sizeof(double) * P->n);
  return ORC_OK;
}

int orc_set_field(orc_problem *P, int which, const double *in) {
  double *f = field_ptr(P, which);
  if (!f) return ORC_EINVAL;
  memcpy(f, in, sizeof(double) * P->n);
  return ORC_OK;
}

/* Weight arrays (n*q each, row-major by point) and stencil indices. */
int orc_get_operators(orc_problem *P, int32_t *idx, double *wx, double *wy, double *wl,
                      double *pval) {
  size_t nq = (size_t)P->n * P->q;
  if (idx) memcpy(idx, P->idx, nq * sizeof(int32_t));
  if (wx) memcpy(wx, P->wx, nq * sizeof(double));
  if (wy) memcpy(wy, P->wy, nq * sizeof(double));
  if (wl) memcpy(wl, P->wl, nq * sizeof(double));
  if (pval) memcpy(pval, P->Pp.val, nq * sizeof(double));
  return ORC_OK;
}

void orc_set_krylov(orc_problem *P, double tol, int maxit) {
  P->ktol = tol;
  P->kmaxit = maxit;
}

/* ------------------------------------------------------------------------ */
/* Kind of the momentum row of point i for velocity component c (0 = u,     */
/* 1 = v), Sec. 3.1: the equation itself inside; an identity row with the   */
/* boundary value where the component is prescribed (walls, inlets, the     */
/* normal component on a symmetry line); a zero normal derivative           */
/* n.grad = 0 at outlets and for the tangential component on a symmetry     */
/* line.                                                                    */
#define ROW_EQ 0
#define ROW_ID 1
#define ROW_NEU 2
static int row_kind(const orc_problem *P, int i, int c) {
  switch (P->tag[i]) {
    case TAG_INTERIOR: return ROW_EQ;
    case TAG_OUTFLOW: return ROW_NEU;
    case TAG_SYMMETRY: {
      int normal_c = fabs(P->nx[i]) > fabs(P->ny[i]) ? 0 : 1;
      return c == normal_c ? ROW_ID : ROW_NEU;
    }
    default: return ROW_ID;
  }
}

/* ------------------------------------------------------------------------ */
/* One outer iteration, Sec. 3.2 steps 2-7, BDF2 coefficients a1, a2, a3.   */
/* stats (nullable, 6 entries): momentum u iters, v iters, p' iters, and     */
/* their final relative residuals.                                           */
int orc_simple_iterate(orc_problem *P, double dt, double a1, double a2, double a3, double *delta,
                       double *stats) {
  int n = P->n;
  const double rho = P->rho, mu = P->mu;
  int64_t *rp = P->rowptr;
  int rc;
  /* Step 2, Eqs. (u:tilde), (v:tilde): linearised momentum, advection with  */
  /* the previous iterate u^r, diffusion implicit, pressure gradient at p^r. */
  /* Boundary rows by row_kind: identity with the BC value, or n.grad = 0.  */
  csr_spmv(&P->Dx, P->p, P->w1); /* (dp/dx)^r */
  csr_spmv(&P->Dy, P->p, P->w2); /* (dp/dy)^r */
  for (int i = 0; i < n; ++i) {
    for (int c = 0; c < 2; ++c) {
      int kind = row_kind(P, i, c);
      double *val = c == 0 ? P->Am.val : P->Av.val;
      for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
        double a;
        if (kind == ROW_EQ) {
          a = rho * P->u[i] * P->wx[e] + rho * P->v[i] * P->wy[e] - mu * P->wl[e];
          if (P->idx[e] == i) a = a + rho * a1 / dt;
        } else if (kind == ROW_NEU) {
          a = P->nx[i] * P->wx[e] + P->ny[i] * P->wy[e];
        } else {
          a = (P->idx[e] == i) ? 1.0 : 0.0;
        }
        val[e] = a;
      }
      double b;
      if (kind == ROW_EQ)
        b = c == 0 ? -rho * (a2 * P->un[i] + a3 * P->unm1[i]) / dt - P->w1[i] + P->force[0]
                   : -rho * (a2 * P->vn[i] + a3 * P->vnm1[i]) / dt - P->w2[i] + P->force[1];
      else if (kind == ROW_NEU)
        b = 0.0;
      else
        b = c == 0 ? P->ubc[i] : P->vbc[i];
      if (c == 0) P->bu[i] = b; else P->bv[i] = b;
    }
  }
  krylov_stats_t su, sv, sp;
  memcpy(P->ut, P->u, sizeof(double) * n); /* initial guess u^r */
  memcpy(P->vt, P->v, sizeof(double) * n);
  rc = bicgstab(&P->Am, P->bu, P->ut, P->ktol, P->kmaxit, &su);
  if (rc) return rc;
  rc = bicgstab(&P->Av, P->bv, P->vt, P->ktol, P->kmaxit, &sv);
  if (rc) return rc;
  /* Step 3, Eq. (pressure poisson): lap p' = (rho a1 / dt)(du~/dx + dv~/dy) */
  /* at interior rows; 0 at the Neumann rows, the outlet rows and the pin.  */
  csr_spmv(&P->Dx, P->ut, P->w1);
  csr_spmv(&P->Dy, P->vt, P->w2);
  for (int i = 0; i < n; ++i)
    P->bp[i] = P->tag[i] == TAG_INTERIOR ? (rho * a1 / dt) * (P->w1[i] + P->w2[i]) : 0.0;
  /* pure-Neumann p' (pinned): make the source compatible (compat_vector) */
  if (P->psi && !P->psi_off) {
    double cshift = dot(n, P->psi, P->bp) / P->psi_eI;
    for (int i = 0; i < n; ++i)
      if (P->tag[i] == TAG_INTERIOR) P->bp[i] = P->bp[i] - cshift;
  }
  for (int i = 0; i < n; ++i) P->pc[i] = 0.0;
  rc = bicgstab(&P->Pp, P->bp, P->pc, P->ktol, P->kmaxit, &sp);
  if (rc) return rc;
  /* Step 4, Eq. (p:correction) at interior points */
  for (int i = 0; i < n; ++i)
    if (P->tag[i] == TAG_INTERIOR) P->p[i] = P->p[i] + P->pc[i];
  /* Step 5, Eq. (normal momentum): boundary pressure.  For a boundary point */
  /* i, G = nx*Wx + ny*Wy (row i) and                                        */
  /*   sum_j G_ij p_j = N . [ -rho (a1 u~ + a2 u^n + a3 u^{n-1})/dt          */
  /*                          - rho (u~ . grad) u~ + mu lap u~ ]_i,          */
  /* solved for p_i with the other p_j at their current values (Jacobi).     */
  /* Outlet points keep their prescribed pressure.                           */
  csr_spmv(&P->Dx, P->ut, P->w1);
  csr_spmv(&P->Dy, P->ut, P->w2);
  csr_spmv(&P->Dl, P->ut, P->w3);
  double *gxu = P->w1, *gyu = P->w2, *lu = P->w3;
  double *gxv = (double *)malloc(sizeof(double) * n);
  double *gyv = (double *)malloc(sizeof(double) * n);
  double *lv = (double *)malloc(sizeof(double) * n);
  double *pnew = (double *)malloc(sizeof(double) * n);
  if (!gxv || !gyv || !lv || !pnew) { free(gxv); free(gyv); free(lv); free(pnew); return ORC_ENOMEM; }
  csr_spmv(&P->Dx, P->vt, gxv);
  csr_spmv(&P->Dy, P->vt, gyv);
  csr_spmv(&P->Dl, P->vt, lv);
  for (int i = 0; i < n; ++i) {
    pnew[i] = P->p[i];
    if (P->tag[i] == TAG_INTERIOR || P->tag[i] == TAG_OUTFLOW) continue;
    double fx = -rho * (a1 * P->ut[i] + a2 * P->un[i] + a3 * P->unm1[i]) / dt -
                rho * (P->ut[i] * gxu[i] + P->vt[i] * gyu[i]) + mu * lu[i] + P->force[0];
    double fy = -rho * (a1 * P->vt[i] + a2 * P->vn[i] + a3 * P->vnm1[i]) / dt -
                rho * (P->ut[i] * gxv[i] + P->vt[i] * gyv[i]) + mu * lv[i] + P->force[1];
    double rhs = P->nx[i] * fx + P->ny[i] * fy;
    double gii = 0.0, off = 0.0;
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
      double g = P->nx[i] * P->wx[e] + P->ny[i] * P->wy[e];
      if (P->idx[e] == i)
        gii = gii + g;
      else
        off = off + g * P->p[P->idx[e]];
    }
    pnew[i] = (rhs - off) / gii;
  }
  for (int i = 0; i < n; ++i) P->p[i] = pnew[i];
  free(gxv); free(gyv); free(lv); free(pnew);
  /* Step 6, Eqs. (u:correction), (v:correction), for every component that  */
  /* is not prescribed (interior, outlets, the tangential component on a    */
  /* symmetry line).  Step 7: Delta = mean|u^{r+1}-u^r| + mean|v^{r+1}-v^r|. */
  csr_spmv(&P->Dx, P->pc, P->w1);
  csr_spmv(&P->Dy, P->pc, P->w2);
  double c = dt / (rho * a1);
  double du = 0.0, dv = 0.0;
  for (int i = 0; i < n; ++i) {
    double unew = P->ut[i], vnew = P->vt[i];
    if (row_kind(P, i, 0) != ROW_ID) unew = P->ut[i] - c * P->w1[i];
    if (row_kind(P, i, 1) != ROW_ID) vnew = P->vt[i] - c * P->w2[i];
    du = du + fabs(unew - P->u[i]);
    dv = dv + fabs(vnew - P->v[i]);
    P->u[i] = unew;
    P->v[i] = vnew;
  }
  *delta = du / n + dv / n;
  if (stats) {
    stats[0] = su.iters; stats[1] = sv.iters; stats[2] = sp.iters;
    stats[3] = su.relres; stats[4] = sv.relres; stats[5] = sp.relres;
  }
  if (!(*delta == *delta)) return ORC_EDIVERGED;
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* One BDF2 time step (Sec. 3.2 steps 1-8): outer iterations from           */
/* [u^r, v^r, p^r] = [u^n, v^n, p^n] until Delta < tol_outer or max_outer,   */
/* then [u^{n-1}, u^n] <- [u^n, u^{n+1}].  change = mean|u^{n+1}-u^n| +      */
/* mean|v^{n+1}-v^n|, i.e. dt * eps_s of the adaptive tolerance.            */
int orc_time_step(orc_problem *P, double dt, double tol_outer, int max_outer, int32_t *outer_iters,
                  double *change, double *last_delta) {
  int n = P->n;
  const double a1 = 1.5, a2 = -2.0, a3 = 0.5;
  int it = 0, rc = ORC_OK;
  double delta = 0.0;
  /* step 1: the iterate starts at time level n (already so after rotation) */
  for (it = 0; it < max_outer;) {
    rc = orc_simple_iterate(P, dt, a1, a2, a3, &delta, NULL);
    ++it;
    if (rc) break;
    if (delta < tol_outer) break;
  }
  double cu = 0.0, cv = 0.0;
  for (int i = 0; i < n; ++i) {
    cu = cu + fabs(P->u[i] - P->un[i]);
    cv = cv + fabs(P->v[i] - P->vn[i]);
  }
  for (int i = 0; i < n; ++i) {
    P->unm1[i] = P->un[i]; P->un[i] = P->u[i];
    P->vnm1[i] = P->vn[i]; P->vn[i] = P->v[i];
  }
  if (outer_iters) *outer_iters = it;
  if (change) *change = cu / n + cv / n;
  if (last_delta) *last_delta = delta;
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Courant number of the explicit-Euler stability bound the paper quotes    */
/* (Sec. 3.2, the paragraph after the solution steps): lambda dt / 2, lambda */
/* the spectral radius of the discrete convection-diffusion operator        */
/*   C = rho (u Dx + v Dy) - mu Lap   at interior rows (other rows zero)    */
/* at the current velocity.  lambda by power iteration from a fixed start:   */
/* x_{k+1} = C x_k / |C x_k|_2, lambda = geometric mean of |C x_k|_2 / |x_k| */
/* over the second half of `iters` steps (robust to complex pairs, unlike    */
/* a Rayleigh quotient).  out: lambda, courant.                              */
int orc_courant(orc_problem *P, double dt, int iters, double *out) {
  int n = P->n;
  if (iters < 2) return ORC_EINVAL;
  double *x = dvec(n), *y = dvec(n), *gx = dvec(n), *gy = dvec(n), *gl = dvec(n);
  if (!x || !y || !gx || !gy || !gl) {
    free(x); free(y); free(gx); free(gy); free(gl);
    return ORC_ENOMEM;
  }
  for (int i = 0; i < n; ++i) x[i] = 1.0 + 0.5 * (double)((i * 7919) % 13) / 13.0;
  double nx = 0.0;
  for (int i = 0; i < n; ++i) nx = nx + x[i] * x[i];
  nx = sqrt(nx);
  for (int i = 0; i < n; ++i) x[i] = x[i] / nx;
  double logsum = 0.0;
  int counted = 0;
  for (int k = 0; k < iters; ++k) {
    csr_spmv(&P->Dx, x, gx);
    csr_spmv(&P->Dy, x, gy);
    csr_spmv(&P->Dl, x, gl);
    double ny = 0.0;
    for (int i = 0; i < n; ++i) {
      y[i] = P->tag[i] == TAG_INTERIOR
                 ? P->rho * (P->u[i] * gx[i] + P->v[i] * gy[i]) - P->mu * gl[i]
                 : 0.0;
      ny = ny + y[i] * y[i];
    }
    ny = sqrt(ny);
    if (!(ny > 0.0)) break;
    if (k >= iters / 2) {
      logsum = logsum + log(ny);
      counted++;
    }
    for (int i = 0; i < n; ++i) x[i] = y[i] / ny;
  }
  double lam = counted > 0 ? exp(logsum / counted) : 0.0;
  out[0] = lam;
  out[1] = lam * dt / 2.0;
  free(x); free(y); free(gx); free(gy); free(gl);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Steady relative residual of the discrete steady equations over the       */
/* interior rows (vector norms over both velocity components):              */
/*   r = rho (u.grad) u - mu lap u + grad p - f   (f: the body force)       */
/*   R_m = |r|_2 / (|rho (u.grad) u|_2 + |mu lap u|_2 + |grad p|_2 + |f|_2)  */
/*   d = Dx u + Dy v at interior rows;  lambda = mean of d                  */
/*   R_c = |d - lambda|_2 / |grad u|_2 when the p' equation is pinned (its   */
/*         source is made compatible, so a steady state satisfies           */
/*         continuity up to the constant lambda: compat_vector), else       */
/*         |d|_2 / |grad u|_2;  |grad u|^2 = sum of the squares of Dx u,     */
/*         Dy u, Dx v, Dy v                                                 */
/* out: R_m, R_c, R = max(R_m, R_c), lambda.                                 */
int orc_steady_residual(orc_problem *P, double *R4) {
  int n = P->n;
  double *gxu = dvec(n), *gyu = dvec(n), *lu = dvec(n), *gxv = dvec(n), *gyv = dvec(n),
         *lv = dvec(n), *gpx = dvec(n), *gpy = dvec(n);
  if (!gxu || !gyu || !lu || !gxv || !gyv || !lv || !gpx || !gpy) {
    free(gxu); free(gyu); free(lu); free(gxv); free(gyv); free(lv); free(gpx); free(gpy);
    return ORC_ENOMEM;
  }
  csr_spmv(&P->Dx, P->u, gxu); csr_spmv(&P->Dy, P->u, gyu); csr_spmv(&P->Dl, P->u, lu);
  csr_spmv(&P->Dx, P->v, gxv); csr_spmv(&P->Dy, P->v, gyv); csr_spmv(&P->Dl, P->v, lv);
  csr_spmv(&P->Dx, P->p, gpx); csr_spmv(&P->Dy, P->p, gpy);
  double nr = 0, sa = 0, sd = 0, sp = 0, sg = 0, sf = 0, sdiv = 0;
  int n_int = 0;
  const double fx = P->force[0], fy = P->force[1];
  for (int i = 0; i < n; ++i) {
    if (P->tag[i] != TAG_INTERIOR) continue;
    double au = P->rho * (P->u[i] * gxu[i] + P->v[i] * gyu[i]);
    double av = P->rho * (P->u[i] * gxv[i] + P->v[i] * gyv[i]);
    double du = P->mu * lu[i], dv = P->mu * lv[i];
    double ru = au - du + gpx[i] - fx, rv = av - dv + gpy[i] - fy;
    nr += ru * ru + rv * rv;
    sa += au * au + av * av;
    sd += du * du + dv * dv;
    sp += gpx[i] * gpx[i] + gpy[i] * gpy[i];
    sf += fx * fx + fy * fy;
    sdiv += gxu[i] + gyv[i];
    n_int++;
    sg += gxu[i] * gxu[i] + gyu[i] * gyu[i] + gxv[i] * gxv[i] + gyv[i] * gyv[i];
  }
  double lambda = n_int > 0 ? sdiv / n_int : 0.0;
  double shift = P->psi && !P->psi_off ? lambda : 0.0;
  double nc = 0;
  for (int i = 0; i < n; ++i) {
    if (P->tag[i] != TAG_INTERIOR) continue;
    double rc = gxu[i] + gyv[i] - shift;
    nc += rc * rc;
  }
  double den_m = sqrt(sa) + sqrt(sd) + sqrt(sp) + sqrt(sf);
  double den_c = sqrt(sg);
  R4[0] = den_m > 0 ? sqrt(nr) / den_m : sqrt(nr);
  R4[1] = den_c > 0 ? sqrt(nc) / den_c : sqrt(nc);
  R4[2] = R4[0] > R4[1] ? R4[0] : R4[1];
  R4[3] = lambda;
  free(gxu); free(gyu); free(lu); free(gxv); free(gyv); free(lv); free(gpx); free(gpy);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Steady driver: BDF2 pseudo-time marching from the current state.  Outer  */
/* tolerance 1e-4 for the first step, then min(1e-4, dt*eps_s) (Sec. 3.2).  */
/* Stops when R = max(R_m, R_c) <= resid_tol.  out (nullable, 4 entries):   */
/* steps taken, total outer iterations, final R, final change.             */
int orc_solve_steady_c(orc_problem *P, double dt, double resid_tol, int max_steps, int max_outer,
                       int criterion, double *out);
int orc_solve_steady(orc_problem *P, double dt, double resid_tol, int max_steps, int max_outer,
                     double *out) {
  return orc_solve_steady_c(P, dt, resid_tol, max_steps, max_outer, 0, out);
}

/* criterion 0: stop when R <= resid_tol; 1: the paper's steady error of
 * Sec. 4.1, (mean|u^{n+1}-u^n| + mean|v^{n+1}-v^n|) / dt <= resid_tol. */
int orc_solve_steady_c(orc_problem *P, double dt, double resid_tol, int max_steps, int max_outer,
                       int criterion, double *out) {
  double tol = 1e-4, R3[4], R = 1.0, change = 0.0;
  int steps = 0;
  long total_outer = 0;
  int rc = ORC_OK;
  while (steps < max_steps) {
    int32_t oi = 0;
    double last;
    rc = orc_time_step(P, dt, tol, max_outer, &oi, &change, &last);
    ++steps;
    total_outer += oi;
    if (rc) break;
    tol = change < 1e-4 ? change : 1e-4;
    orc_steady_residual(P, R3);
    R = R3[2];
    if (!(R == R)) { rc = ORC_EDIVERGED; break; }
    if (criterion == 1 ? change / dt <= resid_tol : R <= resid_tol) break;
  }
  if (out) {
    out[0] = steps; out[1] = (double)total_outer; out[2] = R; out[3] = change;
  }
  if (rc == ORC_OK && !(criterion == 1 ? change / dt <= resid_tol : R <= resid_tol))
    rc = ORC_ENOCONV;
  return rc;
}

/* Unsteady driver: n_steps BDF2 steps with the adaptive outer tolerance.   */
int orc_solve_unsteady(orc_problem *P, double dt, int n_steps, int max_outer, double *out) {
  double tol = 1e-4, change = 0.0;
  long total_outer = 0;
  int rc = ORC_OK, s;
  for (s = 0; s < n_steps; ++s) {
    int32_t oi = 0;
    double last;
    rc = orc_time_step(P, dt, tol, max_outer, &oi, &change, &last);
    total_outer += oi;
    if (rc) { ++s; break; }
    tol = change < 1e-4 ? change : 1e-4;
  }
  if (out) {
    out[0] = s; out[1] = (double)total_outer; out[2] = 0.0; out[3] = change;
  }
  return rc;
}

/* Number of host threads used by the loops over points and rows. */
int orc_set_threads(int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
  return omp_get_max_threads();
#else
  (void)nthreads;
  return 1;
#endif
}

/* y = W x for one of the stored operators (0 Dx, 1 Dy, 2 Lap, 3 p' matrix,  */
/* 4 u-momentum, 5 v-momentum; the two differ only on symmetry lines).      */
int orc_apply(orc_problem *P, int which, const double *xv, double *yv) {
  csr_t *A = which == 0 ? &P->Dx : which == 1 ? &P->Dy : which == 2 ? &P->Dl
           : which == 3 ? &P->Pp : which == 4 ? &P->Am : which == 5 ? &P->Av : NULL;
  if (!A) return ORC_EINVAL;
  csr_spmv(A, xv, yv);
  return ORC_OK;
}

/* The left null vector psi of the pure-Neumann p' operator (compat_vector); */
/* ORC_EINVAL when the problem has an outlet (no compatibility needed).      */
int orc_get_compat(orc_problem *P, double *out) {
  if (!P->psi) return ORC_EINVAL;
  memcpy(out, P->psi, sizeof(double) * P->n);
  return ORC_OK;
}

/* Switch the compatible p' source off (on = 0: the pin alone, whose dropped */
/* Neumann row is then violated whenever the source is incompatible) or     */
/* back on.  Used by the tests to plant that reading.                      */
int orc_set_compat(orc_problem *P, int on) {
  if (!P->psi) return ORC_EINVAL;
  P->psi_off = on ? 0 : 1;
  return ORC_OK;
}
