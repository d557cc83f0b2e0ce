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
  // Work-list autotuner (batch.cu: plan_teams), its iterations run
  // directly.  The batch's first iteration runs untimed at scale 1 (it pays
  // the one-time costs: module loading, first launches); the next 2 NCAND
  // each scale the planned team size of every launch slot by one
  // candidate, in the order 0 1 2 3 3 2 1 0 so that a drift of the work from
  // one iteration to the next cancels; each launch is timed with CUDA
  // events and its time divided by the work it did (rows x iterations of
  // its systems); the two costs of a candidate are averaged and every slot
  // keeps its cheapest scale (part of the graph key).
  static constexpr int NCAND = 4;
  static constexpr int NTUNE = 1 + 2 * NCAND;  // iterations the tuner takes
  static int tune_cand(int step) {             // candidate of a tuning step (-1: warm-up)
    return step == 0 ? -1 : (step <= NCAND ? step - 1 : 2 * NCAND - step);
  }
  double scale[NSLOT] = {1, 1, 1, 1, 1, 1, 1, 1, 1};  // current team-size scale
  double cost[NSLOT][NCAND] = {};  // ms per unit of work, per candidate
  int tune_step = 0;               // tuning iterations done
  bool tuned = false;
  bool tune_off = false;           // autotuner switched off: every scale 1
  bool timing = false;             // this iteration records per-slot events
  cudaEvent_t ev[NSLOT][2] = {};
  bool slot_used[NSLOT] = {};
  std::vector<std::pair<int, int>> slot_sys[NSLOT];  // (member, 0 momentum / 1 p') per system
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
