// batch.cuh -- advancing many problems together (used by the batch ABI and
// by the request server).
#pragma once
#include "common.cuh"
#include "krylov.cuh"

#include <vector>

namespace rbffd {

// Device + pinned host scratch of batched outer iterations, grown on demand,
// and the outer iteration captured as a CUDA graph.  Each of the (up to)
// nine Krylov launches of an outer iteration has its own table slot, so
// nothing is reused within an iteration and the whole iteration -- row
// kernels, table copies, barrier resets, the cooperative Krylov launches,
// the gather of the members' results -- is one stream-ordered sequence that
// a graph can hold.  A set of members, builds and step parameters runs
// directly the first time, is captured the second time, and is replayed
// from then on while it stays the same.
struct BatchScratch {
  static constexpr int NSLOT = 9;
  rbffd_ctx *ctx = nullptr;
  int cap = 0, maxc = 0;
  int team_words = 0;  // ints of one work-list table slot (4 per team + the lists)
  void *dmem = nullptr, *hmem = nullptr;
  size_t dbytes = 0, hbytes = 0;
  // per slot: sys args, CTA -> system, first CTA of each system (one
  // contiguous host -> device copy), flags, barriers
  size_t off_sys[NSLOT] = {}, off_cta_sys[NSLOT] = {}, off_cta_first[NSLOT] = {},
         off_flags[NSLOT] = {}, off_bars[NSLOT] = {};
  size_t off_recs = 0, off_kouts = 0, off_out = 0;
  cudaGraphExec_t exec = nullptr;
  std::vector<uint64_t> key;     // what the graph was captured for
  std::vector<uint64_t> seen;    // the last set run directly (captured when it returns)
  int64_t graph_launches = 0;    // kernels one replay launches
  bool graph_off = false;        // capture failed once: launch directly
  int64_t replays = 0, captures = 0;
  int reserve(rbffd_ctx *c, int members);
  void drop_graph();
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
