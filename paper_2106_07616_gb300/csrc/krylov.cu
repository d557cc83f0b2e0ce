// krylov.cu -- right-Jacobi-preconditioned BiCGSTAB (van der Vorst 1992),
// the solver the paper names for the momentum and pressure-correction
// systems (Sec. 3), as ONE persistent cooperative kernel per solve.
//
// Rows are spread over a grid that is resident all at once (cooperative
// launch); the five grid-wide dependencies of an iteration are crossed with
// a bounded grid barrier (common.cuh).  Dot products are block partials
// followed by a fixed-order sum that every block evaluates redundantly, so
// all blocks hold bit-identical scalars and a solve is deterministic.
// NR = 2 runs two independent recurrences (u~ and v~) that share the
// matrix: one pass over the ELL arrays feeds both SpMVs.
//
// Vectors written inside the kernel are read with __ldcg (L2, coherent
// across SMs); the matrix, which never changes during a solve, goes
// through the read-only path.
#include "common.cuh"
#include "krylov.cuh"

namespace rbffd {

namespace {

constexpr int NT = 256;

// slots of the partials array (x NR for the right-hand sides)
enum { S_BB = 0, S_RR, S_RHV, S_SS, S_TT, S_TS, S_RHR, S_COUNT };

template <int NR>
struct RowSpmv {
  __device__ __forceinline__ static void run(int i, int q, int ldn, const int32_t *__restrict__ col,
                                             const double *__restrict__ val, double *const *xs,
                                             double *out) {
#pragma unroll
    for (int k = 0; k < NR; ++k) out[k] = 0.0;
#pragma unroll 4
    for (int j = 0; j < q; ++j) {
      const int64_t e = (int64_t)j * ldn + i;
      const int c = __ldg(col + e);
      const double a = __ldg(val + e);
#pragma unroll
      for (int k = 0; k < NR; ++k) out[k] += a * __ldcg(xs[k] + c);
    }
  }
};

}  // namespace

template <int NR>
__global__ void __launch_bounds__(NT) k_bicgstab(KrylovArgs A) {
  __shared__ double sred[NT / 32];
  const int nb = gridDim.x;
  const int tid = blockIdx.x * NT + threadIdx.x;
  const int stride = nb * NT;
  const int n = A.n, q = A.q, ldn = A.ldn;
  unsigned int gen = *(volatile unsigned int *)&A.bar->gen;
  double *part = A.part;
  auto P = [&](int slot, int k) { return part + (size_t)(slot * NR + k) * nb; };

  double bnorm[NR], rho[NR], rho_prev[NR], alpha[NR], omega[NR], relres[NR], snorm[NR];
  int it[NR], restarts[NR], state[NR];
  bool need_init[NR], first[NR], have_bnorm[NR], half[NR], zero_x[NR];
#pragma unroll
  for (int k = 0; k < NR; ++k) {
    bnorm[k] = rho[k] = rho_prev[k] = alpha[k] = omega[k] = 1.0;
    relres[k] = snorm[k] = 0.0;
    it[k] = restarts[k] = 0;
    state[k] = KRY_RUNNING;
    need_init[k] = true;
    first[k] = true;
    have_bnorm[k] = false;
    half[k] = false;
    zero_x[k] = false;
  }
  bool ok = true;

  for (;;) {
    // ---------------- (re)start: r = b - A x, r^ = r, p = v = 0
    bool any_init = false;
#pragma unroll
    for (int k = 0; k < NR; ++k) any_init |= (state[k] == KRY_RUNNING && need_init[k]);
    if (any_init) {
      double pbb[NR], prr[NR];
#pragma unroll
      for (int k = 0; k < NR; ++k) pbb[k] = prr[k] = 0.0;
      for (int i = tid; i < n; i += stride) {
        double ax[NR];
        RowSpmv<NR>::run(i, q, ldn, A.col, A.val, A.x, ax);
#pragma unroll
        for (int k = 0; k < NR; ++k) {
          if (state[k] != KRY_RUNNING || !need_init[k]) continue;
          const double bi = A.b[k][i];
          const double ri = bi - ax[k];
          A.w[k].r[i] = ri;
          A.w[k].rh[i] = ri;
          A.w[k].p[i] = 0.0;
          A.w[k].v[i] = 0.0;
          pbb[k] += bi * bi;
          prr[k] += ri * ri;
        }
      }
#pragma unroll
      for (int k = 0; k < NR; ++k) {
        if (state[k] != KRY_RUNNING || !need_init[k]) continue;
        double sb = block_sum<NT>(pbb[k], sred);
        double sr = block_sum<NT>(prr[k], sred);
        if (threadIdx.x == 0) {
          P(S_BB, k)[blockIdx.x] = sb;
          P(S_RR, k)[blockIdx.x] = sr;
        }
      }
      ok = grid_sync(A.bar, nb, gen);
      if (!ok) break;
      bool any_zero = false;
#pragma unroll
      for (int k = 0; k < NR; ++k) {
        if (state[k] != KRY_RUNNING || !need_init[k]) continue;
        need_init[k] = false;
        double bb = 0.0, rr = 0.0;
        if (threadIdx.x < 32) {
          bb = warp_sum_array(P(S_BB, k), nb);
          rr = warp_sum_array(P(S_RR, k), nb);
        }
        __syncthreads();
        if (threadIdx.x == 0) { sred[0] = bb; sred[1] = rr; }
        __syncthreads();
        bb = sred[0];
        rr = sred[1];
        __syncthreads();
        if (!have_bnorm[k]) {
          bnorm[k] = sqrt(bb);
          have_bnorm[k] = true;
        }
        if (bnorm[k] == 0.0) {
          zero_x[k] = true;
          relres[k] = 0.0;
          state[k] = KRY_OK;
          any_zero = true;
          continue;
        }
        const double rn = sqrt(rr);
        relres[k] = rn / bnorm[k];
        if (!(relres[k] == relres[k])) { state[k] = KRY_DIVERGED; continue; }
        if (relres[k] <= A.tol) { state[k] = KRY_OK; continue; }
        rho[k] = rr;  // (r^, r) with r^ = r
        first[k] = true;
      }
      if (any_zero) {
        for (int i = tid; i < n; i += stride) {
#pragma unroll
          for (int k = 0; k < NR; ++k)
            if (zero_x[k]) A.x[k][i] = 0.0;
        }
#pragma unroll
        for (int k = 0; k < NR; ++k) zero_x[k] = false;
      }
    }
    bool any_run = false;
#pragma unroll
    for (int k = 0; k < NR; ++k) any_run |= (state[k] == KRY_RUNNING);
    if (!any_run) break;

    // breakdown rho == 0: restart (at most 3 times)
    bool restart = false;
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      if (state[k] != KRY_RUNNING) continue;
      if (rho[k] == 0.0) {
        if (restarts[k] >= 3) {
          state[k] = KRY_NOCONV;
        } else {
          restarts[k]++;
          need_init[k] = true;
          restart = true;
        }
      }
    }
    if (restart) continue;

    // ---------------- P1: p = r + beta (p - omega v); p^ = p / d
    double beta[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k)
      beta[k] = first[k] ? 0.0 : (rho[k] / rho_prev[k]) * (alpha[k] / omega[k]);
    for (int i = tid; i < n; i += stride) {
      const double di = __ldg(A.dinv + i);
#pragma unroll
      for (int k = 0; k < NR; ++k) {
        if (state[k] != KRY_RUNNING) continue;
        const double ri = A.w[k].r[i];
        const double pi = first[k] ? ri : ri + beta[k] * (A.w[k].p[i] - omega[k] * A.w[k].v[i]);
        A.w[k].p[i] = pi;
        A.w[k].ph[i] = pi * di;
      }
    }
    ok = grid_sync(A.bar, nb, gen);
    if (!ok) break;

    // ---------------- P2: v = A p^, partial (r^, v)
    {
      double prv[NR];
#pragma unroll
      for (int k = 0; k < NR; ++k) prv[k] = 0.0;
      double *phs[NR];
#pragma unroll
      for (int k = 0; k < NR; ++k) phs[k] = A.w[k].ph;
      for (int i = tid; i < n; i += stride) {
        double av[NR];
        RowSpmv<NR>::run(i, q, ldn, A.col, A.val, phs, av);
#pragma unroll
        for (int k = 0; k < NR; ++k) {
          if (state[k] != KRY_RUNNING) continue;
          A.w[k].v[i] = av[k];
          prv[k] += A.w[k].rh[i] * av[k];
        }
      }
#pragma unroll
      for (int k = 0; k < NR; ++k) {
        if (state[k] != KRY_RUNNING) continue;
        double s = block_sum<NT>(prv[k], sred);
        if (threadIdx.x == 0) P(S_RHV, k)[blockIdx.x] = s;
      }
    }
    ok = grid_sync(A.bar, nb, gen);
    if (!ok) break;

    // ---------------- P3: alpha = rho / (r^, v); s = r - alpha v; s^ = s / d
    {
      double rv[NR];
#pragma unroll
      for (int k = 0; k < NR; ++k) {
        rv[k] = 0.0;
        if (state[k] != KRY_RUNNING) continue;
        double t = 0.0;
        if (threadIdx.x < 32) t = warp_sum_array(P(S_RHV, k), nb);
        __syncthreads();
        if (threadIdx.x == 0) sred[0] = t;
        __syncthreads();
        rv[k] = sred[0];
        __syncthreads();
        alpha[k] = rho[k] / rv[k];
      }
      double pss[NR];
#pragma unroll
      for (int k = 0; k < NR; ++k) pss[k] = 0.0;
      for (int i = tid; i < n; i += stride) {
        const double di = __ldg(A.dinv + i);
#pragma unroll
        for (int k = 0; k < NR; ++k) {
          if (state[k] != KRY_RUNNING) continue;
          const double si = A.w[k].r[i] - alpha[k] * A.w[k].v[i];
          A.w[k].s[i] = si;
          A.w[k].sh[i] = si * di;
          pss[k] += si * si;
        }
      }
#pragma unroll
      for (int k = 0; k < NR; ++k) {
        if (state[k] != KRY_RUNNING) continue;
        double s = block_sum<NT>(pss[k], sred);
        if (threadIdx.x == 0) P(S_SS, k)[blockIdx.x] = s;
      }
    }
    ok = grid_sync(A.bar, nb, gen);
    if (!ok) break;

    // ---------------- P4: t = A s^, partials (t, t), (t, s)
    {
      double ptt[NR], pts[NR];
#pragma unroll
      for (int k = 0; k < NR; ++k) ptt[k] = pts[k] = 0.0;
      double *shs[NR];
#pragma unroll
      for (int k = 0; k < NR; ++k) shs[k] = A.w[k].sh;
      for (int i = tid; i < n; i += stride) {
        double at[NR];
        RowSpmv<NR>::run(i, q, ldn, A.col, A.val, shs, at);
#pragma unroll
        for (int k = 0; k < NR; ++k) {
          if (state[k] != KRY_RUNNING) continue;
          A.w[k].t[i] = at[k];
          ptt[k] += at[k] * at[k];
          pts[k] += at[k] * A.w[k].s[i];
        }
      }
#pragma unroll
      for (int k = 0; k < NR; ++k) {
        if (state[k] != KRY_RUNNING) continue;
        double a = block_sum<NT>(ptt[k], sred);
        double b = block_sum<NT>(pts[k], sred);
        if (threadIdx.x == 0) {
          P(S_TT, k)[blockIdx.x] = a;
          P(S_TS, k)[blockIdx.x] = b;
        }
      }
    }
    ok = grid_sync(A.bar, nb, gen);
    if (!ok) break;

    // ---------------- P5: half-step test on |s|; omega; x and r updates
    {
#pragma unroll
      for (int k = 0; k < NR; ++k) {
        half[k] = false;
        if (state[k] != KRY_RUNNING) continue;
        double ss = 0.0, tt = 0.0, ts = 0.0;
        if (threadIdx.x < 32) {
          ss = warp_sum_array(P(S_SS, k), nb);
          tt = warp_sum_array(P(S_TT, k), nb);
          ts = warp_sum_array(P(S_TS, k), nb);
        }
        __syncthreads();
        if (threadIdx.x == 0) { sred[0] = ss; sred[1] = tt; sred[2] = ts; }
        __syncthreads();
        ss = sred[0];
        tt = sred[1];
        ts = sred[2];
        __syncthreads();
        it[k]++;
        snorm[k] = sqrt(ss);
        if (!(snorm[k] == snorm[k])) { state[k] = KRY_DIVERGED; continue; }
        if (snorm[k] / bnorm[k] <= A.tol) {
          half[k] = true;
        } else {
          omega[k] = tt == 0.0 ? 0.0 : ts / tt;
        }
      }
      double prr[NR], prh[NR];
#pragma unroll
      for (int k = 0; k < NR; ++k) prr[k] = prh[k] = 0.0;
      for (int i = tid; i < n; i += stride) {
#pragma unroll
        for (int k = 0; k < NR; ++k) {
          if (state[k] != KRY_RUNNING) continue;
          if (half[k]) {
            A.x[k][i] = A.x[k][i] + alpha[k] * A.w[k].ph[i];
          } else {
            A.x[k][i] = A.x[k][i] + alpha[k] * A.w[k].ph[i] + omega[k] * A.w[k].sh[i];
            const double ri = A.w[k].s[i] - omega[k] * A.w[k].t[i];
            A.w[k].r[i] = ri;
            prr[k] += ri * ri;
            prh[k] += A.w[k].rh[i] * ri;
          }
        }
      }
#pragma unroll
      for (int k = 0; k < NR; ++k) {
        if (state[k] != KRY_RUNNING || half[k]) continue;
        double a = block_sum<NT>(prr[k], sred);
        double b = block_sum<NT>(prh[k], sred);
        if (threadIdx.x == 0) {
          P(S_RR, k)[blockIdx.x] = a;
          P(S_RHR, k)[blockIdx.x] = b;
        }
      }
    }
    ok = grid_sync(A.bar, nb, gen);
    if (!ok) break;

    // ---------------- end of iteration: |r| test, next rho
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      if (state[k] != KRY_RUNNING) continue;
      if (half[k]) {
        relres[k] = snorm[k] / bnorm[k];
        state[k] = KRY_OK;
        continue;
      }
      double rr = 0.0, rh = 0.0;
      if (threadIdx.x < 32) {
        rr = warp_sum_array(P(S_RR, k), nb);
        rh = warp_sum_array(P(S_RHR, k), nb);
      }
      __syncthreads();
      if (threadIdx.x == 0) { sred[0] = rr; sred[1] = rh; }
      __syncthreads();
      rr = sred[0];
      rh = sred[1];
      __syncthreads();
      const double rn = sqrt(rr);
      relres[k] = rn / bnorm[k];
      if (!(rn == rn)) { state[k] = KRY_DIVERGED; continue; }
      if (relres[k] <= A.tol) { state[k] = KRY_OK; continue; }
      if (omega[k] == 0.0) {
        if (restarts[k] >= 3) {
          state[k] = KRY_NOCONV;
        } else {
          restarts[k]++;
          need_init[k] = true;
        }
        continue;
      }
      if (it[k] >= A.maxit) { state[k] = KRY_NOCONV; continue; }
      rho_prev[k] = rho[k];
      rho[k] = rh;
      first[k] = false;
    }
  }

  if (blockIdx.x == 0 && threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      A.out[k].iters = it[k];
      A.out[k].restarts = restarts[k];
      A.out[k].status = ok ? state[k] : KRY_TIMEOUT;
      A.out[k].relres = relres[k];
    }
  }
}

int krylov_max_blocks(rbffd_ctx *ctx, int nr) {
  int per_sm = 0;
  cudaError_t e;
  if (nr == 1)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bicgstab<1>, NT, 0);
  else
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bicgstab<2>, NT, 0);
  if (e != cudaSuccess || per_sm < 1) return 0;
  return per_sm * ctx->num_sms;
}

int krylov_blocks_for(rbffd_ctx *ctx, int n, int nr) {
  int cap = krylov_max_blocks(ctx, nr);
  int want = (n + NT - 1) / NT;
  if (want > ctx->num_sms) want = ctx->num_sms;
  if (want < 1) want = 1;
  return want < cap ? want : cap;
}

int krylov_launch(rbffd_ctx *ctx, int nr, int nblocks, const KrylovArgs &args) {
  if (nblocks < 1) {
    set_error("krylov_launch: no co-resident blocks available");
    return RBFFD_ECUDA;
  }
  RBFFD_CK(cudaMemsetAsync(args.bar, 0, sizeof(GridBarrier), ctx->stream));
  void *kargs[] = {(void *)&args};
  cudaError_t e;
  if (nr == 1)
    e = cudaLaunchCooperativeKernel((const void *)k_bicgstab<1>, dim3(nblocks), dim3(NT), kargs,
                                    0, ctx->stream);
  else
    e = cudaLaunchCooperativeKernel((const void *)k_bicgstab<2>, dim3(nblocks), dim3(NT), kargs,
                                    0, ctx->stream);
  ctx->launches++;
  if (e != cudaSuccess) {
    set_error("cooperative launch of k_bicgstab failed: %s", cudaGetErrorString(e));
    return RBFFD_ECUDA;
  }
  return RBFFD_OK;
}

size_t krylov_partials_doubles(int nr, int nblocks) { return (size_t)S_COUNT * nr * nblocks; }

}  // namespace rbffd
