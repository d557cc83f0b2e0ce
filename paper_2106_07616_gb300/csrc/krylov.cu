// krylov.cu -- right-Jacobi-preconditioned BiCGSTAB (van der Vorst 1992),
// the solver the paper names for the momentum and pressure-correction
// systems (Sec. 3), as ONE persistent cooperative kernel per solve.
//
// Rows are spread over a grid that is resident all at once (cooperative
// launch, one 1024-thread block per SM for one right-hand side, 512 for
// two); the five grid-wide dependencies of an iteration are crossed with a
// bounded acquire/release grid barrier (common.cuh).  A solve of a few
// tens of thousands of rows is latency-bound, so the SpMV spreads each row
// over T threads (T = 1..8, chosen from the thread count per row) to keep
// many independent gathers in flight.
//
// Dot products: block partials, then a fixed-order sum that every block
// evaluates redundantly, so all blocks hold bit-identical scalars and a
// solve is deterministic run to run.  NR = 2 runs two independent
// recurrences (u~ and v~) that share the matrix: one pass over the ELL
// arrays feeds both SpMVs.
//
// Vectors written inside the kernel and gathered by other rows are read
// with __ldcg (L2, coherent across SMs); row-local vectors are only ever
// touched by the thread that owns the row; the matrix never changes during
// a solve and goes through the read-only path.
#include "amg_dev.cuh"
#include "common.cuh"
#include "krylov.cuh"
#include "krylov_dev.cuh"

namespace rbffd {

namespace {

// slots of the partials array (x NR for the right-hand sides)
enum { S_BB = 0, S_RR, S_RHV, S_SS, S_RHS, S_TT, S_TS, S_RHT, S_RHR, S_COUNT };

using kdev::MAXB;

}  // namespace

// Scalar state of one recurrence.  Thread 0 of each block updates it from
// the grid totals; the other threads read it after a __syncthreads, so the
// FP64 divisions and square roots run once per block, not once per thread
// (GB300 issues FP64 at a small fraction of its FP32 rate).
struct KScalars {
  double bnorm, rho, rho_prev, alpha, omega, beta, relres, snorm;
  double best;  // smallest relative residual of the solve so far
  int it, restarts, state, need_init, first, half, run;
  int save;     // the iterate entering the next update is the best so far
  int restore;  // restart from the best iterate (xb) instead of x
  int blowups;  // restarts from the best iterate so far
};

// Residual growth over the best that counts as a blow-up, and how many
// restarts from the best iterate a solve may make.  BiCGSTAB's residual is
// erratic: healthy solves were seen to rise 1.8e4-fold over their start in
// the first iterations and recover.  On the 200 x 200 cavity p' system with
// Jacobi (condition ~3e6) a rounding-dependent loss of the recurrence took
// the residual from below 1e-6 to 1e14 instead; a non-finite residual (a
// near-breakdown's division) is treated the same way.
constexpr double KRY_BLOWUP = 1e10;
constexpr int KRY_MAX_BLOWUPS = 8;

// One BiCGSTAB iteration as four grid exchanges:
//   A: v = A p^,            partial (r^, v)                -> alpha
//   B: s = r - alpha v, s^ = s/d  (rows only)               -> barrier
//   C: t = A s^,            partials (s,s) (t,t) (t,s) (r^,s) (r^,t)
//                                                           -> omega, rho' = (r^,s) - omega (r^,t)
//   D: x += alpha p^ + omega s^, r = s - omega t, and already the next
//      p = r + beta (p - omega v), p^ = p/d with beta = (rho'/rho)(alpha/omega);
//      partials (r, r), (r^, r)                            -> |r| test
// The next direction is formed before the |r| test; if the test stops the
// solve it is simply unused.  rho' equals (r^, r) in exact arithmetic; the
// directly summed (r^, r) replaces it for the next iteration (phase D).
// The solve of one system by the nb CTAs lb = 0..nb-1 that share it (the
// whole grid for a single system; a subrange of a batched launch).
// AMGP: the preconditioner is a V-cycle of the hierarchy A.amg instead of
// the Jacobi scaling (one right-hand side): p^ and s^ come from the cycle
// after p and s are published, not from the row loops.
template <int NR, int NT, bool AMGP = false>
__device__ __forceinline__ void bicgstab_body(const KrylovArgs &A, const int lb, const int nb) {
  static_assert(!AMGP || NR == 1, "the multigrid preconditioner serves one right-hand side");
  __shared__ double sred[5 * NR * NT];  // block_partials of up to 5 NR values
  __shared__ double stot[16];
  __shared__ KScalars ks[NR];
  __shared__ int s_flags[2];
  const int tid = lb * NT + threadIdx.x;
  const int stride = nb * NT;
  const int wglobal = tid >> 5, nwarps = stride >> 5;
  const int n = A.n, q = A.q, ldn = A.ldn, T = A.tpr;
  unsigned int epoch = 1;
  double *part = A.part;
  auto P = [&](int slot, int k) { return part + (size_t)(slot * NR + k) * nb; };
  const bool leader = threadIdx.x == 0;
  int *err = &A.bar->err;
  amgdev::Ctx actx{n,  q,  ldn,    T,      A.col,   A.flags, &A.bar->err,
                   lb, nb, tid, stride, wglobal, nwarps, stot};
  (void)actx;

  if (leader) {
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      KScalars &c = ks[k];
      c.bnorm = c.rho = c.rho_prev = c.alpha = c.omega = 1.0;
      c.beta = c.relres = c.snorm = 0.0;
      c.best = 1e300;
      c.save = c.restore = c.blowups = 0;
      c.it = c.restarts = 0;
      c.state = KRY_RUNNING;
      c.need_init = 1;
      c.first = 1;
      c.half = 0;
      c.run = 1;
    }
  }
  __syncthreads();
  bool ok = true;
  bool have_bnorm = false;

  for (;;) {
    // ---------------- (re)start: r = b - A x, r^ = r, p = r, p^ = r / d
    bool ini[NR], any_init = false, rst[NR], any_rst = false;
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      ini[k] = ks[k].state == KRY_RUNNING && ks[k].need_init;
      any_init |= ini[k];
      rst[k] = ini[k] && ks[k].restore;
      any_rst |= rst[k];
    }
    __syncthreads();
    if (any_rst) {
      // back to the best iterate, published before the restart's SpMV
      for (int i = tid; i < n; i += stride) {
#pragma unroll
        for (int k = 0; k < NR; ++k)
          if (rst[k]) A.x[k][i] = A.w[k].xb[i];
      }
      ok = kdev::exchange<0, double>(A.flags, err, epoch++, nullptr, nullptr, stot, lb, nb);
      if (!ok) break;
      if (leader) {
#pragma unroll
        for (int k = 0; k < NR; ++k)
          if (rst[k]) ks[k].restore = 0;
      }
    }
    if (any_init) {
      double acc[2 * NR];
#pragma unroll
      for (int k = 0; k < 2 * NR; ++k) acc[k] = 0.0;
      kdev::spmv_rows<NR, double>(n, q, ldn, T, A.col, A.val, A.x, wglobal, nwarps,
                    [&](int i, const double *ax) {
                      const double di = __ldg(A.dinv + i);
#pragma unroll
                      for (int k = 0; k < NR; ++k) {
                        if (!ini[k]) continue;
                        const double bi = A.b[k][i];
                        const double ri = bi - ax[k];
                        A.w[k].r[i] = ri;
                        A.w[k].rh[i] = ri;
                        A.w[k].p[i] = ri;
                        if constexpr (!AMGP) A.w[k].ph[i] = ri * di;
                        acc[2 * k] += bi * bi;
                        acc[2 * k + 1] += ri * ri;
                      }
                    });
      double *outs[2 * NR];
#pragma unroll
      for (int k = 0; k < NR; ++k) {
        outs[2 * k] = ini[k] ? P(S_BB, k) : nullptr;
        outs[2 * k + 1] = ini[k] ? P(S_RR, k) : nullptr;
      }
      kdev::block_partials<NT, 2 * NR>(acc, sred, outs, lb);
      double tot[2 * NR];
      ok = kdev::exchange<2 * NR>(A.flags, err, epoch++, outs, tot, stot, lb, nb);
      if (!ok) break;
      int zero_any = 0;
      if (leader) {
#pragma unroll
        for (int k = 0; k < NR; ++k) {
          KScalars &c = ks[k];
          if (!ini[k]) continue;
          c.need_init = 0;
          const double bb = tot[2 * k], rr = tot[2 * k + 1];
          if (c.it == 0 && c.restarts == 0) c.bnorm = sqrt(bb);
          if (c.bnorm == 0.0) {
            c.relres = 0.0;
            c.state = KRY_OK;
            zero_any |= 1 << k;
            continue;
          }
          c.relres = sqrt(rr) / c.bnorm;
          if (!(c.relres == c.relres)) { c.state = KRY_DIVERGED; continue; }
          if (c.relres <= A.tol) { c.state = KRY_OK; continue; }
          if (c.relres < c.best) {
            c.best = c.relres;
            c.save = 1;
          }
          c.rho = rr;  // (r^, r) with r^ = r
          if (c.rho == 0.0) c.state = KRY_NOCONV;
        }
        s_flags[1] = zero_any;
      }
      __syncthreads();
      zero_any = s_flags[1];
      if (zero_any) {
        for (int i = tid; i < n; i += stride) {
#pragma unroll
          for (int k = 0; k < NR; ++k)
            if (zero_any & (1 << k)) A.x[k][i] = 0.0;
        }
      }
      (void)have_bnorm;
    }
    if (leader) {
      int running = 0;
#pragma unroll
      for (int k = 0; k < NR; ++k) {
        ks[k].run = ks[k].state == KRY_RUNNING;
        running |= ks[k].run;
      }
      s_flags[0] = running;
    }
    __syncthreads();
    if (!s_flags[0]) break;
    bool run[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) run[k] = ks[k].run != 0;

    // ---------------- A: v = A p^, partial (r^, v)
    if constexpr (AMGP) {
      if (!amgdev::vcycle(A.amg, actx, A.w[0].p, A.w[0].ph, epoch)) {
        ok = false;
        break;
      }
    }
    {
      double acc[NR];
#pragma unroll
      for (int k = 0; k < NR; ++k) acc[k] = 0.0;
      double *phs[NR];
#pragma unroll
      for (int k = 0; k < NR; ++k) phs[k] = A.w[k].ph;
      kdev::spmv_rows<NR, double>(n, q, ldn, T, A.col, A.val, phs, wglobal, nwarps,
                    [&](int i, const double *av) {
#pragma unroll
                      for (int k = 0; k < NR; ++k) {
                        if (!run[k]) continue;
                        A.w[k].v[i] = av[k];
                        acc[k] += A.w[k].rh[i] * av[k];
                      }
                    });
      double *outs[NR];
#pragma unroll
      for (int k = 0; k < NR; ++k) outs[k] = run[k] ? P(S_RHV, k) : nullptr;
      kdev::block_partials<NT, NR>(acc, sred, outs, lb);
      double tot[NR];
      ok = kdev::exchange<NR>(A.flags, err, epoch++, outs, tot, stot, lb, nb);
      if (!ok) break;
      if (leader) {
#pragma unroll
        for (int k = 0; k < NR; ++k)
          if (run[k]) ks[k].alpha = ks[k].rho / tot[k];
      }
      __syncthreads();
    }

    // ---------------- B: s = r - alpha v; s^ = s / d
    {
      double alp[NR];
#pragma unroll
      for (int k = 0; k < NR; ++k) alp[k] = ks[k].alpha;
      for (int i = tid; i < n; i += stride) {
        const double di = __ldg(A.dinv + i);
#pragma unroll
        for (int k = 0; k < NR; ++k) {
          if (!run[k]) continue;
          const double si = A.w[k].r[i] - alp[k] * A.w[k].v[i];
          A.w[k].s[i] = si;
          if constexpr (!AMGP) A.w[k].sh[i] = si * di;
        }
      }
      ok = kdev::exchange<0, double>(A.flags, err, epoch++, nullptr, nullptr, stot, lb, nb);
      if (!ok) break;
      if constexpr (AMGP) {
        if (!amgdev::vcycle(A.amg, actx, A.w[0].s, A.w[0].sh, epoch)) {
          ok = false;
          break;
        }
      }
    }

    // ---------------- C: t = A s^, partials (s,s) (t,t) (t,s) (r^,s) (r^,t)
    {
      double acc[5 * NR];
#pragma unroll
      for (int k = 0; k < 5 * NR; ++k) acc[k] = 0.0;
      double *shs[NR];
#pragma unroll
      for (int k = 0; k < NR; ++k) shs[k] = A.w[k].sh;
      kdev::spmv_rows<NR, double>(n, q, ldn, T, A.col, A.val, shs, wglobal, nwarps,
                    [&](int i, const double *at) {
#pragma unroll
                      for (int k = 0; k < NR; ++k) {
                        if (!run[k]) continue;
                        const double si = A.w[k].s[i], rhi = A.w[k].rh[i];
                        A.w[k].t[i] = at[k];
                        acc[5 * k + 0] += si * si;
                        acc[5 * k + 1] += at[k] * at[k];
                        acc[5 * k + 2] += at[k] * si;
                        acc[5 * k + 3] += rhi * si;
                        acc[5 * k + 4] += rhi * at[k];
                      }
                    });
      double *outs[5 * NR];
#pragma unroll
      for (int k = 0; k < NR; ++k) {
        outs[5 * k + 0] = run[k] ? P(S_SS, k) : nullptr;
        outs[5 * k + 1] = run[k] ? P(S_TT, k) : nullptr;
        outs[5 * k + 2] = run[k] ? P(S_TS, k) : nullptr;
        outs[5 * k + 3] = run[k] ? P(S_RHS, k) : nullptr;
        outs[5 * k + 4] = run[k] ? P(S_RHT, k) : nullptr;
      }
      kdev::block_partials<NT, 5 * NR>(acc, sred, outs, lb);
      double tot[5 * NR];
      ok = kdev::exchange<5 * NR>(A.flags, err, epoch++, outs, tot, stot, lb, nb);
      if (!ok) break;
      if (leader) {
#pragma unroll
        for (int k = 0; k < NR; ++k) {
          KScalars &c = ks[k];
          c.half = 0;
          if (!run[k]) continue;
          const double ss = tot[5 * k + 0], tt = tot[5 * k + 1], ts = tot[5 * k + 2];
          const double rhs = tot[5 * k + 3], rht = tot[5 * k + 4];
          c.it++;
          c.snorm = sqrt(ss);
          if (!(c.snorm == c.snorm) || c.snorm > 1e300) {
            c.run = 0;  // phase D leaves this system alone; it restarts or ends there
            c.half = 2;
            continue;
          }
          if (c.snorm / c.bnorm <= A.tol) {
            c.half = 1;
            continue;
          }
          c.omega = tt == 0.0 ? 0.0 : ts / tt;
          const double rho_new = rhs - c.omega * rht;
          c.beta = (c.omega == 0.0) ? 0.0 : (rho_new / c.rho) * (c.alpha / c.omega);
          c.rho_prev = c.rho;
          c.rho = rho_new;
        }
      }
      __syncthreads();
    }

    // ---------------- D: x and r updates, next direction, partial (r, r)
    {
      bool half[NR], sav[NR];
      double alp[NR], omg[NR], bet[NR];
#pragma unroll
      bool bad[NR];
      for (int k = 0; k < NR; ++k) {
        bad[k] = ks[k].half == 2;  // non-finite s: restart from the best iterate
        run[k] = ks[k].run != 0;
        half[k] = ks[k].half == 1;
        sav[k] = ks[k].save != 0;
        alp[k] = ks[k].alpha;
        omg[k] = ks[k].omega;
        bet[k] = ks[k].beta;
      }
      __syncthreads();
      if (leader) {
#pragma unroll
        for (int k = 0; k < NR; ++k) ks[k].save = 0;
      }
      double acc[2 * NR];
#pragma unroll
      for (int k = 0; k < 2 * NR; ++k) acc[k] = 0.0;
      for (int i = tid; i < n; i += stride) {
        const double di = __ldg(A.dinv + i);
#pragma unroll
        for (int k = 0; k < NR; ++k) {
          if (!run[k]) continue;
          const double phi = A.w[k].ph[i];
          // x still holds the iterate whose residual was the best so far
          if (sav[k]) A.w[k].xb[i] = A.x[k][i];
          if (half[k]) {
            A.x[k][i] = A.x[k][i] + alp[k] * phi;
          } else {
            const double shi = A.w[k].sh[i];
            A.x[k][i] = A.x[k][i] + alp[k] * phi + omg[k] * shi;
            const double ri = A.w[k].s[i] - omg[k] * A.w[k].t[i];
            A.w[k].r[i] = ri;
            acc[k] += ri * ri;
            acc[NR + k] += A.w[k].rh[i] * ri;
            const double pi = ri + bet[k] * (A.w[k].p[i] - omg[k] * A.w[k].v[i]);
            A.w[k].p[i] = pi;
            if constexpr (!AMGP) A.w[k].ph[i] = pi * di;
          }
        }
      }
      double *outs[2 * NR];
#pragma unroll
      for (int k = 0; k < NR; ++k) {
        outs[k] = (run[k] && !half[k]) ? P(S_RR, k) : nullptr;
        outs[NR + k] = (run[k] && !half[k]) ? P(S_RHR, k) : nullptr;
      }
      kdev::block_partials<NT, 2 * NR>(acc, sred, outs, lb);
      double tot[2 * NR];
      ok = kdev::exchange<2 * NR>(A.flags, err, epoch++, outs, tot, stot, lb, nb);
      if (!ok) break;
      if (leader) {
#pragma unroll
        for (int k = 0; k < NR; ++k) {
          KScalars &c = ks[k];
          // the recurrence has run away (or produced a non-finite value):
          // restart from the best iterate, a bounded number of times
          auto blowup = [&](int final_state) {
            if (c.blowups >= KRY_MAX_BLOWUPS || c.it >= A.maxit) {
              c.state = final_state;
            } else {
              c.blowups++;
              c.restore = 1;
              c.need_init = 1;
            }
          };
          if (bad[k]) {
            c.half = 0;
            blowup(KRY_DIVERGED);
            continue;
          }
          if (!run[k]) continue;
          if (half[k]) {
            c.relres = c.snorm / c.bnorm;
            c.state = KRY_OK;
            continue;
          }
          const double rn = sqrt(tot[k]);
          c.relres = rn / c.bnorm;
          if (!(rn == rn) || rn > 1e300) {
            blowup(KRY_DIVERGED);
            continue;
          }
          if (c.relres <= A.tol) { c.state = KRY_OK; continue; }
          if (c.relres < c.best) {
            c.best = c.relres;
            c.save = 1;  // copied to xb when the next update reads x
          } else if (c.relres > KRY_BLOWUP * c.best) {
            blowup(KRY_NOCONV);
            continue;
          }
          if (c.omega == 0.0 || c.rho == 0.0) {
            // breakdown: restart from the current x (at most 3 times)
            if (c.restarts >= 3) {
              c.state = KRY_NOCONV;
            } else {
              c.restarts++;
              c.need_init = 1;
            }
            continue;
          }
          if (c.it >= A.maxit) { c.state = KRY_NOCONV; continue; }
          // The update took rho_new as (r^,s) - omega (r^,t), equal to
          // (r^, r) in exact arithmetic (it saves a grid exchange) but
          // summed from two products that cancel.  The next iteration uses
          // the directly summed (r^, r) instead: with the fused value alone,
          // the 200 x 200 cavity p' system with Jacobi (~3e6 condition)
          // diverged for some summation orders.  (Restarting whenever r^
          // and r were nearly orthogonal was tried too: it restarted every
          // few hundred iterations and stalled the 150k cylinder.)
          c.rho = tot[NR + k];
        }
      }
      __syncthreads();
    }
  }

  if (lb == 0 && leader) {
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      A.out[k].iters = ks[k].it;
      A.out[k].restarts = ks[k].restarts + ks[k].blowups;
      A.out[k].status = ok ? ks[k].state : KRY_TIMEOUT;
      A.out[k].relres = ks[k].relres;
    }
  }
}

template <int NR, int NT>
__global__ void __launch_bounds__(NT) k_bicgstab(KrylovArgs A) {
  bicgstab_body<NR, NT>(A, blockIdx.x, gridDim.x);
}

// One right-hand side, multigrid-preconditioned (A.amg set).
template <int NT>
__global__ void __launch_bounds__(NT) k_bicgstab_amg(KrylovArgs A) {
  bicgstab_body<1, NT, true>(A, blockIdx.x, gridDim.x);
}

// Many independent systems in one cooperative launch: CTA b works on system
// cta_sys[b]; the CTAs of one system are consecutive and synchronise only
// with each other, so systems progress (and finish) independently.
template <int NR, int NT>
__global__ void __launch_bounds__(NT) k_bicgstab_batch(const KrylovArgs *__restrict__ sys,
                                                       const int *__restrict__ cta_sys,
                                                       const int *__restrict__ cta_first) {
  __shared__ KrylovArgs A;
  // persistent work list (batch.cu: plan_teams): this CTA's team solves
  // the systems cta_first[j0 .. j1) one after another
  const int t = cta_sys[blockIdx.x];
  const int c0 = cta_first[4 * t], nc = cta_first[4 * t + 1];
  const int j0 = cta_first[4 * t + 2], j1 = cta_first[4 * t + 3];
  for (int j = j0; j < j1; ++j) {
    __syncthreads();
    if (threadIdx.x == 0) A = sys[cta_first[j]];
    __syncthreads();
    bicgstab_body<NR, NT>(A, blockIdx.x - c0, nc);
  }
}

// Batched launch of multigrid-preconditioned single-RHS systems.
template <int NT>
__global__ void __launch_bounds__(NT) k_bicgstab_batch_amg(const KrylovArgs *__restrict__ sys,
                                                           const int *__restrict__ cta_sys,
                                                           const int *__restrict__ cta_first) {
  __shared__ KrylovArgs A;
  // persistent work list (batch.cu: plan_teams): this CTA's team solves
  // the systems cta_first[j0 .. j1) one after another
  const int t = cta_sys[blockIdx.x];
  const int c0 = cta_first[4 * t], nc = cta_first[4 * t + 1];
  const int j0 = cta_first[4 * t + 2], j1 = cta_first[4 * t + 3];
  for (int j = j0; j < j1; ++j) {
    __syncthreads();
    if (threadIdx.x == 0) A = sys[cta_first[j]];
    __syncthreads();
    bicgstab_body<1, NT, true>(A, blockIdx.x - c0, nc);
  }
}

namespace {
constexpr int NT1 = 1024;  // threads per block, one right-hand side
constexpr int NT2 = 512;   // two right-hand sides (more registers per thread)

inline int nt_for(int nr) { return nr == 1 ? NT1 : NT2; }
}  // namespace

int krylov_max_blocks(rbffd_ctx *ctx, int nr) {
  int per_sm = 0;
  cudaError_t e;
  if (nr == 1) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bicgstab<1, NT1>, NT1, 0);
    int per_sm_amg = 0;
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_amg, k_bicgstab_amg<NT1>, NT1, 0);
    if (per_sm_amg < per_sm) per_sm = per_sm_amg;
  } else {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bicgstab<2, NT2>, NT2, 0);
  }
  if (e != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    return 0;
  }
  return per_sm * ctx->num_sms;
}

int krylov_blocks_for(rbffd_ctx *ctx, int n, int nr) {
  const int nt = nt_for(nr);
  int cap = krylov_max_blocks(ctx, nr);
  if (cap > ctx->num_sms) cap = ctx->num_sms;  // one block per SM
  if (cap > MAXB) cap = MAXB;
  // aim at 8 threads per row before spreading over fewer SMs
  long long want = ((long long)n * 8 + nt - 1) / nt;
  if (want < 1) want = 1;
  return (int)(want < cap ? want : cap);
}

// threads per row: the most that still cover a CTA's ceil(n / nblocks)
// rows (kdev::cta_rows) in one pass of its warps
int krylov_threads_per_row(int n, int nr, int nblocks) {
  const long long wpb = nt_for(nr) / 32;
  const long long R = (n + (long long)nblocks - 1) / nblocks;
  int best = 1;
  for (int T = 2; T <= 8; ++T)
    if ((32 / T) * wpb >= R) best = T;
  return best;
}

int krylov_launch(rbffd_ctx *ctx, int nr, int nblocks, const KrylovArgs &args) {
  if (nblocks < 1) {
    set_error("krylov_launch: no co-resident blocks available");
    return RBFFD_ECUDA;
  }
  if (nblocks > MAXB) {
    set_error("krylov_launch: %d blocks exceed the limit %d", nblocks, MAXB);
    return RBFFD_EINVAL;
  }
  RBFFD_TRY(reset_barriers(ctx, args.bar, 1));
  RBFFD_CK(cudaMemsetAsync(args.flags, 0, sizeof(unsigned int) * nblocks, ctx->stream));
  void *kargs[] = {(void *)&args};
  cudaError_t e;
  if (nr == 1 && args.amg)
    e = cudaLaunchCooperativeKernel((const void *)k_bicgstab_amg<NT1>, dim3(nblocks), dim3(NT1),
                                    kargs, 0, ctx->stream);
  else if (nr == 1)
    e = cudaLaunchCooperativeKernel((const void *)k_bicgstab<1, NT1>, dim3(nblocks), dim3(NT1),
                                    kargs, 0, ctx->stream);
  else
    e = cudaLaunchCooperativeKernel((const void *)k_bicgstab<2, NT2>, dim3(nblocks), dim3(NT2),
                                    kargs, 0, ctx->stream);
  ctx->launches++;
  if (e != cudaSuccess) {
    set_error("cooperative launch of k_bicgstab failed: %s", cudaGetErrorString(e));
    return RBFFD_ECUDA;
  }
  return RBFFD_OK;
}

size_t krylov_partials_doubles(int nr, int nblocks) { return (size_t)S_COUNT * nr * nblocks; }

int krylov_batch_max_ctas(rbffd_ctx *ctx, int nr) {
  int per_sm = 0;
  cudaError_t e;
  if (nr == 1) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bicgstab_batch<1, KB_NT>, KB_NT,
                                                      0);
    int per_sm_amg = 0;
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_amg,
                                                        k_bicgstab_batch_amg<KB_NT>, KB_NT, 0);
    if (per_sm_amg < per_sm) per_sm = per_sm_amg;
  } else
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bicgstab_batch<2, KB_NT>, KB_NT,
                                                      0);
  if (e != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    return 0;
  }
  return per_sm * ctx->num_sms;
}

int krylov_batch_launch(rbffd_ctx *ctx, int nr, int nctas, const KrylovArgs *d_sys,
                        const int *d_cta_sys, const int *d_cta_first, bool amg) {
  if (nctas < 1 || nctas > krylov_batch_max_ctas(ctx, nr)) {
    set_error("krylov_batch_launch: %d CTAs are not co-resident", nctas);
    return RBFFD_EINVAL;
  }
  void *kargs[] = {(void *)&d_sys, (void *)&d_cta_sys, (void *)&d_cta_first};
  const void *fn = amg ? (const void *)k_bicgstab_batch_amg<KB_NT>
                   : nr == 1 ? (const void *)k_bicgstab_batch<1, KB_NT>
                             : (const void *)k_bicgstab_batch<2, KB_NT>;
  cudaError_t e =
      cudaLaunchCooperativeKernel(fn, dim3(nctas), dim3(KB_NT), kargs, 0, ctx->stream);
  ctx->launches++;
  if (e != cudaSuccess) {
    set_error("cooperative launch of k_bicgstab_batch failed: %s", cudaGetErrorString(e));
    return RBFFD_ECUDA;
  }
  return RBFFD_OK;
}

}  // namespace rbffd
