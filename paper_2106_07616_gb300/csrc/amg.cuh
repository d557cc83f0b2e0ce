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
constexpr int AMG_CSR_CHUNK = 8;  // entries a lane loads before its gathers (CSR rows)

// Arithmetic of the V-cycle (operators, dense inverse, level vectors): a
// type parameter T; the vectors it reads and writes on level 0 may be FP64
// or T.  Inside BiCGSTAB the cycle is FP64: an FP32 cycle's
// rounding (~1e-7 relative on every application, different for every
// input) breaks BiCGSTAB's short recurrences, which assume one fixed linear
// preconditioner -- measured on the 200 x 200 cavity p' system: 1996
// iterations to 1e-12 instead of 76.  FGMRES keeps every preconditioned
// vector and minimises over them, so it takes an FP32 cycle (fgmres.cu).

// A CSR matrix on the device, read with `grp` lanes per row.
template <typename T>
struct AmgCsrT {
  const int32_t *ptr, *col;
  const T *val;
  int grp;  // 1, 2, 4, 8, 16 or 32
};

// One level of the hierarchy, with the V-cycle's smoothing folded into the
// transfer operators.  With W = w D^-1 (damped Jacobi) and a zero start, one
// V(1,1) cycle from level l is
//   z_l = S_l b_l,          S_l = 2 W - W A_l W          (both smoothings' b terms)
//   b_{l+1} = R~_l b_l,     R~_l = R_l (I - A_l W)       (restricted residual)
//   y_l = z_l + P~_l y_{l+1},  P~_l = (I - W A_l) P_l    (correction, post-smoothed)
// which needs one grid exchange per level on the way down and one on the
// way up.  Level 0's S lives in AmgDevT::s0 in the solve's ELL layout.
template <typename T>
struct AmgLevelT {
  int n;            // rows
  AmgCsrT<T> S;     // levels >= 1
  AmgCsrT<T> R;     // n_{l+1} x n_l (not on the coarsest)
  AmgCsrT<T> P;     // n_l x n_{l+1} (not on the coarsest)
  T *b;             // right-hand side (levels >= 1)
  T *z;             // S_l b_l
  T *y;             // the level's result
};

template <typename T>
struct AmgDevT {
  using value_type = T;
  int nlev;         // levels including the coarsest
  const T *cinv;    // inverse of the coarsest matrix, row-major nc x nc
  const T *s0;      // level 0's S, ELL [q][ldn] on the solve's column array
  int ts0;          // threads per row of level 0's S in the cycle (1..8)
  const T *a0;      // level 0's A rounded to T, same layout (FP32 only, else null)
  AmgLevelT<T> lev[AMG_MAXLEV];
};

using amg_t = double;  // the cycle inside BiCGSTAB
using AmgCsr = AmgCsrT<double>;
using AmgLevel = AmgLevelT<double>;
using AmgDev = AmgDevT<double>;
using AmgDevF = AmgDevT<float>;  // the cycle inside FGMRES

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
// *bytes; freed with dev_free).  nblocks x wpb: the CTAs and warps per CTA
// of the launch that will run the cycle (lanes per row are chosen for it;
// any launch runs it correctly).  *dev receives the device copy of the
// level table.  Errors: RBFFD_ESINGULAR if the coarsest matrix is singular,
// RBFFD_ENOMEM, RBFFD_ECUDA.
// T = double or float: the stored arithmetic of the cycle.
template <typename T>
int amg_build(rbffd_ctx *ctx, int n, int q, int ldn, const int32_t *col, const double *val,
              int nblocks, int wpb, void **mem, size_t *bytes, const AmgDevT<T> **dev,
              AmgDevT<T> *host_view, AmgInfo *info);

// The host part alone, on a CSR matrix (analysis and tests): level sizes
// and nonzeros in *info.
int amg_analyze(int n, const int32_t *rowptr, const int32_t *col, const double *val,
                AmgInfo *info);

}  // namespace rbffd
