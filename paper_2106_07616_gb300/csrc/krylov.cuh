// krylov.cuh -- internal interface of the persistent BiCGSTAB solver.
#pragma once
#include "amg.cuh"
#include "common.cuh"

namespace rbffd {

enum { KRY_RUNNING = 1, KRY_OK = 0, KRY_NOCONV = -4, KRY_DIVERGED = -5, KRY_TIMEOUT = -6 };

struct KrylovVecs {
  double *r, *rh, *p, *v, *ph, *s, *sh, *t;
  double *xb;  // the iterate with the smallest residual so far (restart point)
};

struct KrylovOut {
  int iters;
  int restarts;
  int status;
  int pad;
  double relres;
};

struct KrylovArgs {
  int n, q, ldn;
  const int32_t *col;   // ELL [q][ldn]
  const double *val;    // ELL [q][ldn]
  const double *dinv;   // 1 / diagonal
  const double *b[2];
  double *x[2];
  KrylovVecs w[2];
  double *part;         // krylov_partials_doubles(nr, nblocks)
  GridBarrier *bar;     // err word (bounded waits that gave up)
  unsigned int *flags;  // word 0: the arrival counter, zeroed per launch
  KrylovOut *out;       // nr entries
  double tol;
  int maxit;
  int tpr;              // threads per row in the SpMV phases (1..8)
  int nblocks;          // CTAs that share the solve (batched launches)
  const AmgDev *amg;    // multigrid preconditioner (one RHS), or null: Jacobi
};

constexpr int KB_NT = 256;  // threads per CTA of batched Krylov launches

// Inner arithmetic of the mixed-precision solve.
enum { INNER_F32 = 0, INNER_FF = 1 };

// Vectors of the mixed-precision solve, in the inner arithmetic's storage
// type (float for INNER_F32, a float pair for INNER_FF); d = the sweep's
// correction.
struct MixedVecs {
  void *r, *rh, *p0, *p1, *v0, *v1, *s, *t, *d;  // p, v double-buffered
};

struct MixedArgs {
  int n, q, ldn, tpr;
  int inner;             // INNER_F32 or INNER_FF
  int nblocks;           // CTAs of the system in a batched launch
  const int32_t *col;
  const double *val64;   // FP64 operator (residuals)
  const void *valin;     // operator in the inner arithmetic
  const void *dinvin;    // 1 / diagonal in the inner arithmetic
  const double *b[2];
  double *x[2];
  MixedVecs w[2];
  double *part64;        // krylov_ir_partials64(nr, nblocks)
  void *partin;          // krylov_ir_partials_inner_bytes(nr, nblocks, inner)
  GridBarrier *bar;
  unsigned int *flags;
  KrylovOut *out;        // iters = inner iterations, restarts = sweeps
  double tol;            // FP64 relative residual to reach
  int maxit;             // cap on inner iterations over all sweeps
  double inner_tol;      // relative reduction asked of each inner solve
  int inner_maxit;       // cap on inner iterations per sweep
  int max_sweeps;
};

int krylov_max_blocks(rbffd_ctx *ctx, int nr);
int krylov_ir_max_blocks(rbffd_ctx *ctx, int nr, int inner);
int krylov_ir_launch(rbffd_ctx *ctx, int nr, int nblocks, const MixedArgs &args);
// Batched: d_sys[s] (nblocks, flags, bar set) owns CTAs d_cta_first[s] ..;
// KB_NT threads per CTA; every system of one launch has the same inner
// arithmetic.
int krylov_ir_batch_max_ctas(rbffd_ctx *ctx, int nr, int inner);
int krylov_ir_batch_launch(rbffd_ctx *ctx, int nr, int inner, int nctas, const MixedArgs *d_sys,
                           const int *d_cta_sys, const int *d_cta_first);
size_t krylov_ir_partials64(int nr, int nblocks);
size_t krylov_ir_partials_inner_bytes(int nr, int nblocks, int inner);
int krylov_blocks_for(rbffd_ctx *ctx, int n, int nr);
int krylov_threads_per_row(int n, int nr, int nblocks);
int krylov_batch_max_ctas(rbffd_ctx *ctx, int nr);
// d_sys: device array of per-system arguments (nblocks, flags and partials
// sized for that many CTAs); d_cta_sys / d_cta_first: per CTA, its system
// and per system, its first CTA.  Flags and barrier words must be zeroed.
// amg: every system has a multigrid preconditioner (nr = 1).
int krylov_batch_launch(rbffd_ctx *ctx, int nr, int nctas, const KrylovArgs *d_sys,
                        const int *d_cta_sys, const int *d_cta_first, bool amg = false);
int krylov_launch(rbffd_ctx *ctx, int nr, int nblocks, const KrylovArgs &args);
size_t krylov_partials_doubles(int nr, int nblocks);

}  // namespace rbffd
