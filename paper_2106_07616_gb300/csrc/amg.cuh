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

// Arithmetic of the V-cycle (operators, dense inverse, level vectors).
// FP64: with amg_t = float the cycle's rounding (~1e-7 relative on every
// application, different for every input) breaks the short recurrences of
// the BiCGSTAB around it -- measured on the 200 x 200 cavity p' system:
// 1996 iterations to 1e-12 instead of 76 -- so the cycle stays in FP64
// although GB300 issues FP32 far faster.
using amg_t = double;

// A CSR matrix on the device, read with `grp` lanes per row.
struct AmgCsr {
  const int32_t *ptr, *col;
  const amg_t *val;
  int grp;  // 1, 2, 4, 8, 16 or 32
};

// One level of the hierarchy, with the V-cycle's smoothing folded into the
// transfer operators.  With W = w D^-1 (damped Jacobi) and a zero start, one
// V(1,1) cycle from level l is
//   z_l = S_l b_l,          S_l = 2 W - W A_l W          (both smoothings' b terms)
//   b_{l+1} = R~_l b_l,     R~_l = R_l (I - A_l W)       (restricted residual)
//   y_l = z_l + P~_l y_{l+1},  P~_l = (I - W A_l) P_l    (correction, post-smoothed)
// which needs one grid exchange per level on the way down and one on the
// way up.  Level 0's S lives in AmgDev::s0 in the solve's ELL layout.
struct AmgLevel {
  int n;       // rows
  AmgCsr S;    // levels >= 1
  AmgCsr R;    // n_{l+1} x n_l (not on the coarsest)
  AmgCsr P;    // n_l x n_{l+1} (not on the coarsest)
  amg_t *b;    // right-hand side (levels >= 1)
  amg_t *z;    // S_l b_l
  amg_t *y;    // the level's result
};

struct AmgDev {
  int nlev;            // levels including the coarsest
  const amg_t *cinv;   // inverse of the coarsest matrix, row-major nc x nc
  const amg_t *s0;     // level 0's S, ELL [q][ldn] on the solve's column array
  AmgLevel lev[AMG_MAXLEV];
};

struct AmgInfo {
  int nlev;
  int n[AMG_MAXLEV];
  long long nnz[AMG_MAXLEV];    // A_l
  long long nnz_r[AMG_MAXLEV];  // R~_l
  long long nnz_p[AMG_MAXLEV];  // P~_l
  double omega[AMG_MAXLEV];
  double setup_ms;              // host time of the hierarchy build
};

// Build the hierarchy of the packed p' matrix (ELL, column-major [q][ldn],
// device) on the host and upload it into one device allocation (*mem,
// *bytes; freed with dev_free).  *dev receives the device copy of the
// level table.  Errors: RBFFD_ESINGULAR if the coarsest matrix is singular,
// RBFFD_ENOMEM, RBFFD_ECUDA.
int amg_build(rbffd_ctx *ctx, int n, int q, int ldn, const int32_t *col, const double *val,
              void **mem, size_t *bytes, const AmgDev **dev, AmgDev *host_view, AmgInfo *info);

// The host part alone, on a CSR matrix (analysis and tests): level sizes
// and nonzeros in *info.
int amg_analyze(int n, const int32_t *rowptr, const int32_t *col, const double *val,
                AmgInfo *info);

}  // namespace rbffd
