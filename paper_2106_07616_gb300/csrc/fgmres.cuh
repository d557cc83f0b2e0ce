// fgmres.cuh -- interface of the persistent flexible GMRES solver of the
// pressure-correction system with an FP32 multigrid V-cycle preconditioner.
#pragma once
#include "amg.cuh"
#include "common.cuh"
#include "krylov.cuh"

namespace rbffd {

constexpr int FG_MAXM = 30;  // largest restart length

struct FgmresArgs {
  int n, q, ldn, tpr;   // rows, ELL width, leading dimension, threads per row
  int m;                // restart length, 1..FG_MAXM
  int nblocks;          // CTAs of the system in a batched launch
  const int32_t *col;   // ELL [q][ldn]
  const double *val;    // ELL [q][ldn], FP64: the true residual at each restart
  const float *val32;   // the same values rounded to FP32: the Arnoldi SpMVs
  const double *b;
  double *x;            // initial guess in, solution out
  double *r;            // n: b - A x at a restart
  float *V;             // (m + 1) x n Arnoldi basis
  float *Z;             // m x n preconditioned directions
  void *part;           // fgmres_partials_bytes(nblocks), 8-byte aligned
  GridBarrier *bar;     // err word (bounded waits that gave up)
  unsigned int *flags;  // word 0: the arrival counter, zeroed per launch
  KrylovOut *out;       // iters, restarts, status (KRY_*), relres (true residual)
  double tol;           // relative residual to reach
  int maxit;            // cap on Arnoldi steps over all restarts
  const AmgDevF *amg;   // the FP32 hierarchy
  int reorth;           // 1: classical Gram-Schmidt with one reorthogonalisation
                        // (two reductions a step); 0: one pass, the norm by
                        // Pythagoras (one reduction, one grid exchange fewer);
                        // 2: two passes, the second delayed to the next step's
                        // reduction (one reduction a step)
};

size_t fgmres_partials_bytes(int nblocks);
int fgmres_max_blocks(rbffd_ctx *ctx);
// rows per block fixed by nblocks; threads per row chosen inside
int fgmres_launch(rbffd_ctx *ctx, int nblocks, const FgmresArgs &args);
// Batched: d_sys[s] (with nblocks set) owns CTAs d_cta_first[s] ..; KB_NT
// threads per CTA; at most fgmres_batch_max_ctas CTAs in one launch.
int fgmres_batch_max_ctas(rbffd_ctx *ctx);
int fgmres_batch_launch(rbffd_ctx *ctx, int nctas, const FgmresArgs *d_sys,
                        const int *d_cta_sys, const int *d_cta_first);

}  // namespace rbffd
