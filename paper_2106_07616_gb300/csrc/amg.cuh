// amg.cuh -- smoothed-aggregation algebraic multigrid hierarchy for the
// pressure-correction system, used as the preconditioner of its BiCGSTAB.
// The paper only says the p' system is solved by a preconditioned BiCGSTAB
// (Sec. 3); Jacobi is the default here, this hierarchy the alternative.
// It changes how many Krylov iterations a solve takes, not the solution
// the solve stops on (the same relative-residual test).
#pragma once
#include "common.cuh"

namespace rbffd {

constexpr int AMG_MAXLEV = 10;

// One level of the hierarchy (device pointers).  Level 0 is the p' matrix
// itself, kept in the problem's ELL arrays; its CSR fields are null.
struct AmgLevel {
  int n;  // rows
  const int32_t *a_ptr, *a_col;  // A_l, CSR (levels >= 1)
  const double *a_val;
  const double *wdinv;           // Jacobi smoother weight / diag(A_l)
  const int32_t *p_ptr, *p_col;  // P_l: n_l x n_{l+1} prolongation (not on the coarsest)
  const double *p_val;
  const int32_t *r_ptr, *r_col;  // R_l = P_l^T: n_{l+1} x n_l restriction
  const double *r_val;
  double *x;  // level iterate
  double *b;  // level right-hand side (levels >= 1)
  double *y;  // residual on the way down, smoothed result on the way up
};

struct AmgDev {
  int nlev;            // levels including the coarsest
  const double *cinv;  // inverse of the coarsest matrix, row-major nc x nc
  AmgLevel lev[AMG_MAXLEV];
};

struct AmgInfo {
  int nlev;
  int n[AMG_MAXLEV];
  long long nnz[AMG_MAXLEV];    // A_l
  long long nnz_p[AMG_MAXLEV];  // P_l (= R_l), 0 on the coarsest
  double omega[AMG_MAXLEV];
};

// Build the hierarchy of the packed p' matrix (ELL, column-major [q][ldn],
// device) on the host and upload it into one device allocation (*mem,
// *bytes; freed with dev_free).  *dev receives the device copy of the
// level table.  Errors: RBFFD_ESINGULAR if the coarsest matrix is singular,
// RBFFD_ENOMEM, RBFFD_ECUDA.
int amg_build(rbffd_ctx *ctx, int n, int q, int ldn, const int32_t *col, const double *val,
              void **mem, size_t *bytes, const AmgDev **dev, AmgDev *host_view, AmgInfo *info);

}  // namespace rbffd
