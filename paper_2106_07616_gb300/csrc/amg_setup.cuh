// amg_setup.cuh -- level 0 of the multigrid hierarchy built on the device
// (amg_setup.cu), handed to the host build of the coarse levels (amg.cu).
#pragma once
#include <vector>

#include "amg.cuh"

namespace rbffd {

// most distinct columns of one row of P, A P, A^T P or A_1 the device build
// holds; a wider row makes it give up (the host build runs instead)
constexpr int AMG_SETUP_DMAX = 96;
// the device build runs for p' matrices of at least this many rows (smaller
// ones take a few milliseconds on the host, off the device's way)
constexpr int AMG_SETUP_MIN_ROWS = 16384;

// What the device build leaves: level 0's cycle operators in one device
// allocation (offsets into `mem`, the cycle's type T), A_1 on the host.
struct AmgL0 {
  int n1 = 0;                         // aggregates
  double lam = 0.0;                   // rho(D^-1 A)
  double omega = 0.0;                 // the smoother's weight min(2/3, 4 / (3 lam))
  long long nnz_a = 0, nnz_r = 0, nnz_p = 0;  // A_0, R~_0, P~_0
  int maxlen_r = 0, maxlen_p = 0;     // longest rows of R~_0 and P~_0
  std::vector<int32_t> a1ptr, a1col;  // A_1 (CSR)
  std::vector<double> a1val;
  void *mem = nullptr;
  size_t bytes = 0;
  size_t o_s0 = 0, o_a0 = 0, o_rp = 0, o_rc = 0, o_rv = 0, o_pp = 0, o_pc = 0, o_pv = 0,
         o_z = 0, o_y = 0;
};

// Level 0 of the packed p' matrix (ELL [q][ldn] on the device, n rows) on
// stream st (the caller's); low: also A in FP32 (the flexible GMRES cycle).
// Synchronises st a few times (the MIS(2) rounds, the sizes of the
// products).  RBFFD_ENOTIMPL: the device build does not apply (q > 64, a
// row wider than AMG_SETUP_DMAX, a pattern the device's P~ or R~ does not
// cover, coarsening stalled); nothing is kept, the caller builds on the
// host.  RBFFD_ENOMEM, RBFFD_ECUDA.
template <typename T>
int amg_level0_device(rbffd_ctx *ctx, cudaStream_t st, int n, int q, int ldn,
                      const int32_t *col, const double *val, bool low, AmgL0 *out);

}  // namespace rbffd
