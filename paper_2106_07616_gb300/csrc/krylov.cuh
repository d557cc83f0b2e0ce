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
  GridBarrier *bar;
  KrylovOut *out;       // nr entries
  double tol;
  int maxit;
};

int krylov_max_blocks(rbffd_ctx *ctx, int nr);
int krylov_blocks_for(rbffd_ctx *ctx, int n, int nr);
int krylov_launch(rbffd_ctx *ctx, int nr, int nblocks, const KrylovArgs &args);
size_t krylov_partials_doubles(int nr, int nblocks);

}  // namespace rbffd
