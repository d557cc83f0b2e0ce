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
constexpr int AMG_RCHUNK = 32 * AMG_CSR_CHUNK;  // entries of a composed-restriction chunk

// Arithmetic of the V-cycle (operators, dense inverse, level vectors): a
// type parameter T; the vectors it reads and writes on level 0 may be FP64
// or T.  Inside BiCGSTAB the cycle is FP64: an FP32 cycle's
// rounding (~1e-7 relative on every application, different for every
// input) breaks BiCGSTAB's short recurrences, which assume one fixed linear
// preconditioner -- measured on the 200 x 200 cavity p' system: 1996
// iterations to 1e-12 instead of 76.  FGMRES keeps every preconditioned
// vector and minimises over them, so it takes an FP32 cycle (fgmres.cu).

// Priorities of level 0's MIS(2) aggregation (amg.cu: aggregate_mis2; the
// device build in amg_setup.cu takes the same): key(i) = (h(i) << 32 | i) + 1
// with h the 32-bit finaliser of MurmurHash3 (Appleby); 0 means "none".
__host__ __device__ inline uint32_t mis_hash(uint32_t x) {
  x ^= x >> 16;
  x *= 0x85ebca6bu;
  x ^= x >> 13;
  x *= 0xc2b2ae35u;
  x ^= x >> 16;
  return x;
}
__host__ __device__ inline uint64_t mis_key(int i) {
  return (((uint64_t)mis_hash((uint32_t)i) << 32) | (uint32_t)i) + 1;
}
// fixed non-constant start of the power iteration for rho(D^-1 A)
__host__ __device__ inline double rho_start(int i) {
  return 1.0 + 0.5 * (double)(((uint32_t)i * 7919u) % 13u) / 13.0;
}
constexpr double AMG_THETA = 0.08;  // strength threshold
constexpr double AMG_OMEGA = 2.0 / 3.0;

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

// The composed cycle.  The folded V-cycle above is one linear map; below
// level 1 it regroups as
//   y_1 = S_1 b_1 + sum_{l >= 2} Q_l b_l,   b_l = Rh_l b_1,
//   Rh_2 = R~_1,  Rh_l = R~_{l-1} Rh_{l-1}  (restriction straight from level 1),
//   Q_l = P~_1 ... P~_{l-1} S_l, and on the coarsest level
//   P~_1 ... P~_{L-2} A_{L-1}^-1            (corrections prolonged to level 1),
// four dependent phases instead of 2 L - 1: (A) z_0 = S_0 b_0 and
// b_1 = R~_0 b_0 as before; (B1) z_1 = S_1 b_1 and every deeper right-hand
// side at once, as partial sums of chunks of the stacked Rh (each chunk one
// warp's, AMG_RCHUNK entries at most); (B2) every CTA sums the chunks of all
// coarse entries into shared memory (the coarse vector c, nc entries) and
// y_1 = z_1 + Q c on level 1's rows, Q = [Q_2 | Q_3 | ...]; (C) the
// prolongation to level 0 as before.  Built on the host for three or more
// levels (amg.cu: compose); run by launches whose dynamic shared memory
// holds c, the others run the level-by-level cycle.
template <typename T>
struct AmgCompT {
  int nc;                      // coarse entries: rows of levels 2 .. L-1 (0: none)
  int nchunk;                  // chunks of the stacked Rh
  int nseg;                    // levels stacked
  int seg_off[AMG_MAXLEV + 1];  // level s + 2: entries [seg_off[s], seg_off[s + 1])
  int seg_grp[AMG_MAXLEV];     // lanes per entry summing its chunks (1..32)
  const int32_t *rcol;         // stacked Rh: column (level 1) and value of each entry
  const T *rval;
  const int32_t *cs;           // chunk c: entries [cs[c], cs[c + 1])
  const int32_t *kc;           // entry k: chunks [kc[k], kc[k + 1])
  AmgCsrT<T> Q;                // n_1 x nc
  T *part;                     // chunk sums (phase A)
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
  AmgCompT<T> comp;
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
  int comp_nc;                  // composed cycle: stacked coarse entries (0: not built)
  int comp_chunks;              // chunks of its stacked restriction
  long long comp_nnz_r;         // entries of the stacked restriction
  long long comp_nnz_q;         // entries of Q
  bool device_l0;               // level 0 was built on the device (amg_setup.cu)
};

// Build the hierarchy of the packed p' matrix (ELL, column-major [q][ldn],
// device) and upload it: the coarse levels in one device allocation (*mem,
// *bytes), level 0 in a second one when it was built on the device
// (*mem0, *bytes0; else null and 0); both freed with dev_free.  nblocks x
// wpb: the CTAs and warps per CTA of the launch that will run the cycle
// (lanes per row are chosen for it; any launch runs it correctly).  *dev
// receives the device copy of the level table.  Errors: RBFFD_ESINGULAR if
// the coarsest matrix is singular, RBFFD_ENOMEM, RBFFD_ECUDA.
// T = double or float: the stored arithmetic of the cycle.
template <typename T>
int amg_build(rbffd_ctx *ctx, int n, int q, int ldn, const int32_t *col, const double *val,
              int nblocks, int wpb, void **mem, size_t *bytes, void **mem0, size_t *bytes0,
              const AmgDevT<T> **dev, AmgDevT<T> *host_view, AmgInfo *info);

// The host part alone, on a CSR matrix (analysis and tests): level sizes
// and nonzeros in *info.
int amg_analyze(int n, const int32_t *rowptr, const int32_t *col, const double *val,
                AmgInfo *info);

// Level 0's aggregates of a CSR matrix on the host (aggregate_mis2 on its
// strength graph): agg[n], *naggs.
int amg_aggregates_host(int n, const int32_t *rowptr, const int32_t *col, const double *val,
                        int32_t *agg, int32_t *naggs);

// One cycle of the hierarchy of a CSR matrix applied to b on the host in
// FP64, level by level (out_levels) and composed (out_composed; zeros when
// the composed cycle is not built), n entries each.
int amg_cycle_host(int n, const int32_t *rowptr, const int32_t *col, const double *val,
                   const double *b, double *out_levels, double *out_composed, AmgInfo *info);

}  // namespace rbffd
