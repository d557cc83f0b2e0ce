// batch.cuh -- advancing many problems together (used by the batch ABI and
// by the request server).
#pragma once
#include "common.cuh"
#include "krylov.cuh"

namespace rbffd {

// Device + pinned host scratch of batched outer iterations, grown on demand.
struct BatchScratch {
  rbffd_ctx *ctx = nullptr;
  int cap = 0, maxc = 0;
  void *dmem = nullptr, *hmem = nullptr;
  size_t dbytes = 0, hbytes = 0;
  size_t off_sys = 0, off_cta_sys = 0, off_cta_first = 0, off_flags = 0, off_bars = 0,
         off_recs = 0, off_kouts = 0, off_out = 0;
  int reserve(rbffd_ctx *c, int members);
  ~BatchScratch();
};

// One outer iteration (paper Sec. 3.2 steps 2-7) of the m problems P[0..m),
// all FP64 and on one context.  deltas, stats, status: host arrays of m
// (nullable).  With status, per-member solver failures are reported there
// and the call returns RBFFD_OK; without it, the first failure is returned.
// spv[i]: the step parameters of member i (dt may differ per member; the
// Krylov tolerance and cap of member 0 apply to all).
int batch_iterate(BatchScratch &S, rbffd_problem *const *P, int m,
                  const rbffd_step_params *const *spv, double *deltas, rbffd_iter_stats *stats,
                  int *status);

}  // namespace rbffd
