// ops.cuh -- internal interface of the outer-iteration row kernels.
#pragma once
#include "problem.cuh"

namespace rbffd {
int ops_pack(rbffd_problem *P);
int ops_momentum(rbffd_problem *P, const rbffd_step_params *sp);
int ops_divergence(rbffd_problem *P, const rbffd_step_params *sp);
int ops_pressure(rbffd_problem *P, const rbffd_step_params *sp);
int ops_correct(rbffd_problem *P, const rbffd_step_params *sp);
int ops_rotate(rbffd_problem *P);
int ops_resid(rbffd_problem *P);
int ops_courant(rbffd_problem *P, int iters, double *logacc);
int ops_spmv(rbffd_problem *P, const double *val, const double *x, double *y);
// b = e_I (1 at interior rows), x = 0
int ops_interior_ones(rbffd_problem *P, double *b, double *x);
int ops_reduce_blocks(rbffd_ctx *ctx, int n);
int ops_to_inner(rbffd_problem *P, const double *src, void *dst, int64_t m);
}  // namespace rbffd
