// krylov_mixed.cu -- the mixed-precision Krylov solve: FP32 right-Jacobi
// BiCGSTAB inside FP64 defect correction (iterative refinement), as ONE
// persistent cooperative kernel per solve.
//
// A sweep computes the FP64 residual r = b - A x with the FP64 operator,
// stops when |r| <= tol |b| (the same test as the FP64 solver, so both
// paths stop at the same FP64 accuracy), and otherwise solves A d = r to a
// loose relative tolerance with BiCGSTAB on FP32 copies of the operator and
// Jacobi diagonal, FP32 vectors and FP32 dot products, then x += d in FP64.
// The refinement converges while cond(A) * eps_fp32 < 1; each sweep gains
// about -log10(max(inner_tol, cond * eps_fp32)) digits.
//
// Why on GB300: the FP64 pipe issues 2 lanes per clock per SM against 128
// for FP32, so FP64 SpMV and reductions are ALU-bound there; the inner
// iterations, which are nearly all the work, run entirely on the FP32 pipe
// and move half the bytes.
#include "common.cuh"
#include "krylov.cuh"
#include "krylov_dev.cuh"

namespace rbffd {

namespace {

enum { M_BB = 0, M_RR, M_COUNT64 };
enum { F_RHV = 0, F_SS, F_TT, F_TS, F_RHS, F_RHT, F_RR, F_COUNT32 };

struct IRS {
  double bnorm, relres, rho, alpha, omega, beta, r0, snorm;
  int state, sweeps, it, inner_it, in_sweep, inner, half, zero;
};

}  // namespace

template <int NR, int NT>
__global__ void __launch_bounds__(NT) k_bicgstab_ir(MixedArgs A) {
  __shared__ float sr32[5 * NR * NT];
  __shared__ double sr64[2 * NR * NT];
  __shared__ float st32[16];
  __shared__ double st64[16];
  __shared__ IRS ks[NR];
  __shared__ int s_any;
  const int tid = blockIdx.x * NT + threadIdx.x;
  const int stride = gridDim.x * NT;
  const int wglobal = tid >> 5, nwarps = stride >> 5;
  const int n = A.n, q = A.q, ldn = A.ldn, T = A.tpr;
  const int nb = gridDim.x;
  unsigned int epoch = 1;
  const bool leader = threadIdx.x == 0;
  int *err = &A.bar->err;
  auto P64 = [&](int slot, int k) { return A.part64 + (size_t)(slot * NR + k) * nb; };
  auto P32 = [&](int slot, int k) { return A.part32 + (size_t)(slot * NR + k) * nb; };

  if (leader) {
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      IRS &c = ks[k];
      c.bnorm = 1.0;
      c.relres = c.rho = c.alpha = c.omega = c.beta = c.r0 = c.snorm = 0.0;
      c.state = KRY_RUNNING;
      c.sweeps = c.it = c.inner_it = 0;
      c.in_sweep = c.inner = c.half = c.zero = 0;
    }
  }
  __syncthreads();
  bool ok = true;

  for (;;) {
    // ---------------- R: FP64 residual, r32 = r, r^ = r, p = r, p^ = r/d, d = 0
    bool part[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) part[k] = ks[k].state == KRY_RUNNING;
    __syncthreads();
    {
      double acc[2 * NR];
#pragma unroll
      for (int k = 0; k < 2 * NR; ++k) acc[k] = 0.0;
      kdev::spmv_rows<NR, double>(n, q, ldn, T, A.col, A.val64, A.x, wglobal, nwarps,
                                  [&](int i, const double *ax) {
                                    const float di = __ldg(A.dinv32 + i);
#pragma unroll
                                    for (int k = 0; k < NR; ++k) {
                                      if (!part[k]) continue;
                                      const double bi = A.b[k][i];
                                      const double ri = bi - ax[k];
                                      const float rf = (float)ri;
                                      A.w[k].r[i] = rf;
                                      A.w[k].rh[i] = rf;
                                      A.w[k].p[i] = rf;
                                      A.w[k].ph[i] = rf * di;
                                      A.w[k].d[i] = 0.0f;
                                      acc[2 * k] += bi * bi;
                                      acc[2 * k + 1] += ri * ri;
                                    }
                                  });
      double *outs[2 * NR];
#pragma unroll
      for (int k = 0; k < NR; ++k) {
        outs[2 * k] = part[k] ? P64(M_BB, k) : nullptr;
        outs[2 * k + 1] = part[k] ? P64(M_RR, k) : nullptr;
      }
      kdev::block_partials<NT, 2 * NR>(acc, sr64, outs);
      double tot[2 * NR];
      ok = kdev::exchange<2 * NR>(A.flags, err, epoch++, outs, tot, st64);
      if (!ok) break;
      if (leader) {
        int any = 0;
#pragma unroll
        for (int k = 0; k < NR; ++k) {
          IRS &c = ks[k];
          c.in_sweep = 0;
          c.zero = 0;
          if (!part[k]) continue;
          if (c.sweeps == 0) c.bnorm = sqrt(tot[2 * k]);
          if (c.bnorm == 0.0) {
            c.relres = 0.0;
            c.state = KRY_OK;
            c.zero = 1;
            continue;
          }
          const double rr = tot[2 * k + 1];
          c.relres = sqrt(rr) / c.bnorm;
          if (!(c.relres == c.relres)) { c.state = KRY_DIVERGED; continue; }
          if (c.relres <= A.tol) { c.state = KRY_OK; continue; }
          if (c.sweeps >= A.max_sweeps || c.it >= A.maxit) { c.state = KRY_NOCONV; continue; }
          c.in_sweep = 1;
          c.inner = 1;
          c.inner_it = 0;
          c.rho = rr;
          c.r0 = sqrt(rr);
          any = 1;
        }
        s_any = any;
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < NR; ++k)
        if (ks[k].zero) {
          for (int i = tid; i < n; i += stride) A.x[k][i] = 0.0;
        }
      if (!s_any) break;
    }

    // ---------------- inner FP32 BiCGSTAB on A d = r
    for (;;) {
      bool run[NR], anyrun = false;
#pragma unroll
      for (int k = 0; k < NR; ++k) {
        run[k] = ks[k].inner != 0;
        anyrun |= run[k];
      }
      __syncthreads();
      if (!anyrun) break;

      // A: v = A p^, partial (r^, v)
      {
        float acc[NR];
#pragma unroll
        for (int k = 0; k < NR; ++k) acc[k] = 0.f;
        float *phs[NR];
#pragma unroll
        for (int k = 0; k < NR; ++k) phs[k] = A.w[k].ph;
        kdev::spmv_rows<NR, float>(n, q, ldn, T, A.col, A.val32, phs, wglobal, nwarps,
                                   [&](int i, const float *av) {
#pragma unroll
                                     for (int k = 0; k < NR; ++k) {
                                       if (!run[k]) continue;
                                       A.w[k].v[i] = av[k];
                                       acc[k] += A.w[k].rh[i] * av[k];
                                     }
                                   });
        float *outs[NR];
#pragma unroll
        for (int k = 0; k < NR; ++k) outs[k] = run[k] ? P32(F_RHV, k) : nullptr;
        kdev::block_partials<NT, NR>(acc, sr32, outs);
        float tot[NR];
        ok = kdev::exchange<NR>(A.flags, err, epoch++, outs, tot, st32);
        if (!ok) break;
        if (leader) {
#pragma unroll
          for (int k = 0; k < NR; ++k) {
            if (!run[k]) continue;
            const double al = ks[k].rho / (double)tot[k];
            // a (near) breakdown of the FP32 recurrence ends the sweep with
            // the correction accumulated so far; FP64 refinement goes on
            if (!isfinite(al) || fabs(al) > 1e30) {
              ks[k].inner = 0;
              continue;
            }
            ks[k].alpha = al;
          }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < NR; ++k) run[k] = ks[k].inner != 0;
      }
      // B: s = r - alpha v, s^ = s / d
      {
        float alp[NR];
#pragma unroll
        for (int k = 0; k < NR; ++k) alp[k] = (float)ks[k].alpha;
        for (int i = tid; i < n; i += stride) {
          const float di = __ldg(A.dinv32 + i);
#pragma unroll
          for (int k = 0; k < NR; ++k) {
            if (!run[k]) continue;
            const float si = A.w[k].r[i] - alp[k] * A.w[k].v[i];
            A.w[k].s[i] = si;
            A.w[k].sh[i] = si * di;
          }
        }
        ok = kdev::exchange<0, float>(A.flags, err, epoch++, nullptr, nullptr, st32);
        if (!ok) break;
      }
      // C: t = A s^, partials (s,s) (t,t) (t,s) (r^,s) (r^,t)
      {
        float acc[5 * NR];
#pragma unroll
        for (int k = 0; k < 5 * NR; ++k) acc[k] = 0.f;
        float *shs[NR];
#pragma unroll
        for (int k = 0; k < NR; ++k) shs[k] = A.w[k].sh;
        kdev::spmv_rows<NR, float>(n, q, ldn, T, A.col, A.val32, shs, wglobal, nwarps,
                                   [&](int i, const float *at) {
#pragma unroll
                                     for (int k = 0; k < NR; ++k) {
                                       if (!run[k]) continue;
                                       const float si = A.w[k].s[i], rhi = A.w[k].rh[i];
                                       A.w[k].t[i] = at[k];
                                       acc[5 * k + 0] += si * si;
                                       acc[5 * k + 1] += at[k] * at[k];
                                       acc[5 * k + 2] += at[k] * si;
                                       acc[5 * k + 3] += rhi * si;
                                       acc[5 * k + 4] += rhi * at[k];
                                     }
                                   });
        float *outs[5 * NR];
#pragma unroll
        for (int k = 0; k < NR; ++k) {
          outs[5 * k + 0] = run[k] ? P32(F_SS, k) : nullptr;
          outs[5 * k + 1] = run[k] ? P32(F_TT, k) : nullptr;
          outs[5 * k + 2] = run[k] ? P32(F_TS, k) : nullptr;
          outs[5 * k + 3] = run[k] ? P32(F_RHS, k) : nullptr;
          outs[5 * k + 4] = run[k] ? P32(F_RHT, k) : nullptr;
        }
        kdev::block_partials<NT, 5 * NR>(acc, sr32, outs);
        float tot[5 * NR];
        ok = kdev::exchange<5 * NR>(A.flags, err, epoch++, outs, tot, st32);
        if (!ok) break;
        if (leader) {
#pragma unroll
          for (int k = 0; k < NR; ++k) {
            IRS &c = ks[k];
            c.half = 0;
            if (!run[k]) continue;
            const double ss = tot[5 * k + 0], tt = tot[5 * k + 1], ts = tot[5 * k + 2];
            const double rhs = tot[5 * k + 3], rht = tot[5 * k + 4];
            c.it++;
            c.inner_it++;
            c.snorm = sqrt(ss);
            if (!isfinite(c.snorm) || !isfinite(tt) || !isfinite(ts) || c.snorm > 1e3 * c.r0) {
              // the FP32 recurrence went astray: end the sweep, keep d
              c.inner = 0;
              continue;
            }
            if (c.snorm <= A.inner_tol * c.r0) {
              c.half = 1;
              continue;
            }
            c.omega = tt == 0.0 ? 0.0 : ts / tt;
            const double rho_new = rhs - c.omega * rht;
            double be = (c.omega == 0.0 || c.rho == 0.0)
                            ? 0.0
                            : (rho_new / c.rho) * (c.alpha / c.omega);
            if (!isfinite(be) || !isfinite(rho_new) || fabs(be) > 1e30) {
              // apply this step's update, then end the sweep
              be = 0.0;
              c.omega = isfinite(c.omega) ? c.omega : 0.0;
              c.half = 2;
            }
            c.beta = be;
            c.rho = rho_new;
          }
        }
        __syncthreads();
      }
      // D: d += alpha p^ + omega s^, r = s - omega t, next direction, partial (r, r)
      {
        bool half[NR];
        float alp[NR], omg[NR], bet[NR];
#pragma unroll
        for (int k = 0; k < NR; ++k) {
          run[k] = ks[k].inner != 0;
          half[k] = ks[k].half == 1;
          alp[k] = (float)ks[k].alpha;
          omg[k] = (float)ks[k].omega;
          bet[k] = (float)ks[k].beta;
        }
        float acc[NR];
#pragma unroll
        for (int k = 0; k < NR; ++k) acc[k] = 0.f;
        for (int i = tid; i < n; i += stride) {
          const float di = __ldg(A.dinv32 + i);
#pragma unroll
          for (int k = 0; k < NR; ++k) {
            if (!run[k]) continue;
            const float phi = A.w[k].ph[i];
            if (half[k]) {
              A.w[k].d[i] += alp[k] * phi;
            } else {
              A.w[k].d[i] += alp[k] * phi + omg[k] * A.w[k].sh[i];
              const float ri = A.w[k].s[i] - omg[k] * A.w[k].t[i];
              A.w[k].r[i] = ri;
              acc[k] += ri * ri;
              const float pi = ri + bet[k] * (A.w[k].p[i] - omg[k] * A.w[k].v[i]);
              A.w[k].p[i] = pi;
              A.w[k].ph[i] = pi * di;
            }
          }
        }
        float *outs[NR];
#pragma unroll
        for (int k = 0; k < NR; ++k) outs[k] = (run[k] && !half[k]) ? P32(F_RR, k) : nullptr;
        kdev::block_partials<NT, NR>(acc, sr32, outs);
        float tot[NR];
        ok = kdev::exchange<NR>(A.flags, err, epoch++, outs, tot, st32);
        if (!ok) break;
        if (leader) {
#pragma unroll
          for (int k = 0; k < NR; ++k) {
            IRS &c = ks[k];
            if (!run[k]) continue;
            if (half[k] || c.half == 2) {
              c.inner = 0;
              continue;
            }
            const double rn = sqrt((double)tot[k]);
            if (!isfinite(rn) || rn <= A.inner_tol * c.r0 || rn > 1e3 * c.r0 ||
                c.omega == 0.0 || c.rho == 0.0 || c.inner_it >= A.inner_maxit ||
                c.it >= A.maxit)
              c.inner = 0;  // end of this sweep (converged, breakdown or cap)
          }
        }
        __syncthreads();
      }
    }
    if (!ok) break;
    // ---------------- x += d (FP64)
    {
      bool upd[NR];
#pragma unroll
      for (int k = 0; k < NR; ++k) upd[k] = ks[k].in_sweep != 0;
      for (int i = tid; i < n; i += stride) {
#pragma unroll
        for (int k = 0; k < NR; ++k)
          if (upd[k]) A.x[k][i] = A.x[k][i] + (double)A.w[k].d[i];  // d is finite: every
          // step that could make it non-finite ended the sweep before its update
      }
      if (leader) {
#pragma unroll
        for (int k = 0; k < NR; ++k)
          if (upd[k]) ks[k].sweeps++;
      }
      ok = kdev::exchange<0, double>(A.flags, err, epoch++, nullptr, nullptr, st64);
      if (!ok) break;
    }
  }

  if (blockIdx.x == 0 && leader) {
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      A.out[k].iters = ks[k].it;
      A.out[k].restarts = ks[k].sweeps;
      A.out[k].status = ok ? ks[k].state : KRY_TIMEOUT;
      A.out[k].relres = ks[k].relres;
    }
  }
}

namespace {
constexpr int MT1 = 1024;
constexpr int MT2 = 512;
}  // namespace

int krylov_ir_max_blocks(rbffd_ctx *ctx, int nr) {
  int per_sm = 0;
  cudaError_t e;
  if (nr == 1)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bicgstab_ir<1, MT1>, MT1, 0);
  else
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bicgstab_ir<2, MT2>, MT2, 0);
  if (e != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    return 0;
  }
  return per_sm * ctx->num_sms;
}

int krylov_ir_launch(rbffd_ctx *ctx, int nr, int nblocks, const MixedArgs &args) {
  if (nblocks < 1 || nblocks > kdev::MAXB || nblocks > krylov_ir_max_blocks(ctx, nr)) {
    set_error("krylov_ir_launch: %d blocks not co-resident", nblocks);
    return RBFFD_EINVAL;
  }
  RBFFD_CK(cudaMemsetAsync(args.bar, 0, sizeof(GridBarrier), ctx->stream));
  RBFFD_CK(cudaMemsetAsync(args.flags, 0, sizeof(unsigned int) * nblocks, ctx->stream));
  void *kargs[] = {(void *)&args};
  cudaError_t e;
  if (nr == 1)
    e = cudaLaunchCooperativeKernel((const void *)k_bicgstab_ir<1, MT1>, dim3(nblocks), dim3(MT1),
                                    kargs, 0, ctx->stream);
  else
    e = cudaLaunchCooperativeKernel((const void *)k_bicgstab_ir<2, MT2>, dim3(nblocks), dim3(MT2),
                                    kargs, 0, ctx->stream);
  ctx->launches++;
  if (e != cudaSuccess) {
    set_error("cooperative launch of k_bicgstab_ir failed: %s", cudaGetErrorString(e));
    return RBFFD_ECUDA;
  }
  return RBFFD_OK;
}

size_t krylov_ir_partials64(int nr, int nblocks) { return (size_t)M_COUNT64 * nr * nblocks; }
size_t krylov_ir_partials32(int nr, int nblocks) { return (size_t)F_COUNT32 * nr * nblocks; }

}  // namespace rbffd
