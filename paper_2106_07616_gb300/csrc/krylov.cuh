// krylov.cuh -- internal interface of the persistent BiCGSTAB solver.
#pragma once
#include "common.cuh"

namespace rbffd {

enum { KRY_RUNNING = 1, KRY_OK = 0, KRY_NOCONV = -4, KRY_DIVERGED = -5, KRY_TIMEOUT = -6 };

struct KrylovVecs {
  double *r, *rh, *p, *v, *ph, *s, *sh, *t;
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
  unsigned int *flags;  // one publish flag per block, zeroed per launch
  KrylovOut *out;       // nr entries
  double tol;
  int maxit;
  int tpr;              // threads per row in the SpMV phases (1, 2, 4 or 8)
};

// FP32 vectors of the mixed-precision solve (d = the sweep's correction).
struct MixedVecs {
  float *r, *rh, *p, *v, *ph, *s, *sh, *t, *d;
};

struct MixedArgs {
  int n, q, ldn, tpr;
  const int32_t *col;
  const double *val64;   // FP64 operator (residuals)
  const float *val32;    // FP32 copy (inner iterations)
  const float *dinv32;   // FP32 1 / diagonal
  const double *b[2];
  double *x[2];
  MixedVecs w[2];
  double *part64;        // krylov_ir_partials64(nr, nblocks)
  float *part32;         // krylov_ir_partials32(nr, nblocks)
  GridBarrier *bar;
  unsigned int *flags;
  KrylovOut *out;        // iters = inner iterations, restarts = sweeps
  double tol;            // FP64 relative residual to reach
  int maxit;             // cap on inner iterations over all sweeps
  double inner_tol;      // relative reduction asked of each FP32 solve
  int inner_maxit;       // cap on inner iterations per sweep
  int max_sweeps;
};

int krylov_max_blocks(rbffd_ctx *ctx, int nr);
int krylov_ir_max_blocks(rbffd_ctx *ctx, int nr);
int krylov_ir_launch(rbffd_ctx *ctx, int nr, int nblocks, const MixedArgs &args);
size_t krylov_ir_partials64(int nr, int nblocks);
size_t krylov_ir_partials32(int nr, int nblocks);
int krylov_blocks_for(rbffd_ctx *ctx, int n, int nr);
int krylov_threads_per_row(int n, int nr, int nblocks);
int krylov_launch(rbffd_ctx *ctx, int nr, int nblocks, const KrylovArgs &args);
size_t krylov_partials_doubles(int nr, int nblocks);

}  // namespace rbffd
