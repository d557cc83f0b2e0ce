// knn.cuh -- internal interface of the cloud builder.
#pragma once
#include <stddef.h>

#include "common.cuh"

namespace rbffd {

struct KnnLayout {
  int G, m;
  size_t off_bbox, off_err, off_cell, off_cnt, off_start, off_cursor, off_pts;
  size_t bytes;
};

int knn_workspace_bytes(int n, KnnLayout *lay);
// Lx, Ly: periods of the axes (0: bounded).
int knn_run(rbffd_ctx *ctx, void *ws, const KnnLayout &lay, int n, const double *x,
            const double *y, const int8_t *tag, int q, int32_t *idx, double Lx, double Ly);

}  // namespace rbffd
