// problem.cuh -- device-resident state of one flow problem.
#pragma once
#include "common.cuh"
#include "amg.cuh"
#include "amg_job.cuh"
#include "knn.cuh"
#include "krylov.cuh"

// Outer-iteration record read back by the host once per outer iteration.
struct IterRecord {
  double delta;
  double change;
  double resid[4];  // R_m, R_c, R, lambda (rbffd_steady_residual)
  double pad[1];
  // total compatible shift c of the last p' solve (ops.cu: k_center,
  // compat_shift): the next solve takes it away from its right-hand side
  // first; zero after a build
  double cshift;
};

struct rbffd_problem {
  rbffd_ctx *ctx = nullptr;
  int n = 0, q = 0, degree = 0, pin = 0, precision = 0;
  int ldn = 0;  // padded row count of the column-major ELL arrays
  double rho = 1.0, mu = 1.0;
  double per[2] = {0.0, 0.0};    // periods of x and y (0: bounded)
  double force[2] = {0.0, 0.0};  // body force per unit volume
  // inputs
  double *x, *y, *nx, *ny, *ubc, *vbc;
  int8_t *tag;
  // clouds and weights, row-major n x q (as built)
  int32_t *idx_rm;
  double *wx_rm, *wy_rm, *wl_rm;
  // packed operators, column-major [q][ldn], one shared index array
  int32_t *col;
  double *Wx, *Wy, *Wl, *Pp, *Am;
  double *p_dinv, *m_dinv;
  // v~ matrix and its Jacobi diagonal, used only when symmetry lines exist
  // (the u~ and v~ rows differ there); otherwise Am serves both
  double *Am2, *m_dinv2;
  bool has_sym = false;
  // copies in the inner arithmetic of the mixed-precision solves (FP32 or
  // float-float; null in the FP64 path)
  int inner = 0;  // rbffd::INNER_F32 / INNER_FF
  void *Pin = nullptr, *Ain = nullptr, *pdin = nullptr, *mdin = nullptr;
  void *Ain2 = nullptr, *mdin2 = nullptr;
  rbffd::MixedVecs mv[2] = {};
  double *part64 = nullptr;
  void *partin = nullptr;
  // fields
  double *u, *v, *p, *p2, *un, *vn, *unm1, *vnm1, *ut, *vt, *pc, *bu, *bv, *bp;
  // compatible p' of a pinned problem (no outlet): z = M^{-1} e_I, solved
  // once per build by compat_ready, and the shifted p' of the iteration
  // (ops.cu: compat_shift)
  double *zc, *pcs;
  bool compat = false;   // pin >= 0: the p' equation has Neumann rows only
  // iterations of the last momentum [0] and p' [1] solves (the work
  // estimate of the batched work lists; 0 before any)
  int it_hist[2] = {0, 0};
  bool z_ready = false;  // zc holds z for the current build
  // Krylov workspace: 8 vectors x 2 right-hand sides
  rbffd::KrylovVecs kv[2];
  double *part;       // Krylov partials
  double *rpart;      // partials of the outer-loop reductions
  rbffd::GridBarrier *bar;
  unsigned int *flags;     // Krylov arrival counter (word 0)
  rbffd::KrylovOut *kout;  // [0..1] momentum, [2] pressure correction
  IterRecord *rec;         // device copy of the iteration record
  int *d_first_singular;
  // cloud-builder workspace
  void *knn_ws;
  rbffd::KnnLayout knn_lay;
  int kblocks1 = 0, kblocks2 = 0;  // cooperative grid sizes (1 and 2 RHS)
  int rblocks = 0;                 // grid of the row kernels with reductions
  // one allocation holds everything above
  void *mem = nullptr;
  size_t bytes = 0;
  // multigrid preconditioner of the p' solve (its own allocation), or none
  int precond = 0;
  // changes with every build (create or reload): what a captured batch
  // graph of this problem refers to (buffers, hierarchy) may have changed
  uint64_t gen = 0;
  void *amg_mem = nullptr;
  size_t amg_bytes = 0;
  void *amg0_mem = nullptr;  // level 0 built on the device (its own allocation), or null
  size_t amg0_bytes = 0;
  const rbffd::AmgDev *amg = nullptr;  // device copy of the level table
  rbffd::AmgDev amg_host{};             // host copy (device pointers)
  rbffd::AmgInfo amg_info{};
  // the hierarchy's host part while it is being built (amg_ready finishes it)
  rbffd::AmgJob *amg_job = nullptr;
  // status of a hierarchy build that failed for good (not for want of
  // device memory): every later p' solve returns it, until a reload
  int amg_err = 0;
  char amg_errmsg[160] = {0};
  // flexible GMRES with an FP32 hierarchy (RBFFD_PRECOND_AMG_FGMRES): the
  // FP32 level table and the basis / direction vectors and partials
  const rbffd::AmgDevF *amgf = nullptr;
  rbffd::AmgDevF amgf_host{};
  void *fg_mem = nullptr;
  size_t fg_bytes = 0;
  double *fgR = nullptr;                     // FP64 restart residual
  float *fgV = nullptr, *fgZ = nullptr;       // FP32 basis and directions
  void *fgpart = nullptr;
  int fg_m = 0, fg_blocks = 0;
};

namespace rbffd {
// End of a BDF2 time step (rotation of the time levels); change = mean
// |u - u^n| + mean |v - v^n| of the step.  Synchronises the stream.
int problem_step_end(rbffd_problem *P, double *change);
// Algorithmic bytes of an FP64 pressure-correction solve of `iters`
// iterations (the roofline numerator of the p' kernel statistics).
double pcorr_bytes(const rbffd_problem *P, int iters);
// Steady stopping test of solve_steady and of the request server.
bool steady_done(const rbffd_solve_params *s, double R, double change, int steps);
// Finish the multigrid hierarchy whose host part a build started (upload
// on the problem's stream); a no-op when none is pending.  Every use of
// the hierarchy calls it first.
int amg_ready(rbffd_problem *P);
// Solve z = M^{-1} e_I with the problem's p' solver once per build (pinned
// problems only; a no-op otherwise or when done).  Synchronises the stream:
// call it before any graph capture.
int compat_ready(rbffd_problem *P);
// tolerance, step cap and acceptance of the z solve (problem.cu)
double compat_tol(const rbffd_problem *P);
constexpr double compat_accept() { return 1e-9; }
int compat_maxit(const rbffd_problem *P);
// z solved again, from zero, with FP64 Jacobi BiCGSTAB to compat_accept()
// (up to 50 000 steps): for a multigrid solve of z that stalled.  Waits for
// it; *relres (nullable) receives its relative residual.
int compat_fallback(rbffd_problem *P, double *relres);
// partial-sum slots of the steady residual reduction (ops.cu: k_resid)
constexpr int RESID_SLOTS = 9;
}  // namespace rbffd
