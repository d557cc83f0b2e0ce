// weights.cuh -- internal interface of the weight generator.
#pragma once
#include "common.cuh"

namespace rbffd {
int weights_check_args(int n, int q, int degree);
int weights_config(int q, int degree, int *wpb, size_t *smem);
// d_first_singular: device int, must hold INT_MAX on entry; receives the
// lowest singular cloud index.
// Lx, Ly: periods of the axes (0: bounded); cloud members enter at their
// nearest periodic image.
int weights_run(rbffd_ctx *ctx, int n, const double *x, const double *y, int q,
                const int32_t *idx, int degree, double *wx, double *wy, double *wl,
                int *d_first_singular, double Lx, double Ly);
}  // namespace rbffd
