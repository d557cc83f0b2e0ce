// krylov_mixed.cu -- the mixed-precision Krylov solve: FP32 right-Jacobi
// BiCGSTAB inside FP64 defect correction (iterative refinement), as ONE
// persistent cooperative kernel per solve.
//
// A sweep computes the FP64 residual r = b - A x with the FP64 operator,
// stops when |r| <= tol |b| (the same test as the FP64 solver, so both
// paths stop at the same FP64 accuracy), and otherwise solves A d = r to a
// looser relative tolerance with BiCGSTAB on a copy of the operator and
// Jacobi diagonal held in the inner arithmetic (inner_arith.cuh), then
// x += d in FP64.  The refinement converges while cond(A) * eps_inner < 1;
// each sweep gains about -log10(max(inner_tol, cond * eps_inner)) digits.
//   ArithF32: eps 6e-8 -- enough for well-conditioned systems (momentum);
//   ArithFF:  float-float, eps ~1e-14 -- converges like FP64 on the
//             pressure-correction systems too.
//
// Why on GB300: the FP64 pipe issues 2 lanes per clock per SM against 128
// for FP32, so FP64 SpMV and reductions are ALU-bound there; the inner
// iterations, which are nearly all the work, run entirely on the FP32 pipe
// and move half the bytes.
#include "common.cuh"
#include "krylov.cuh"
#include "inner_arith.cuh"
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

// y_k(i) = sum_j A(i,j) x_k(j) in the inner arithmetic IA, T threads per
// row; the same batching and group sums as kdev::spmv_rows.
template <int NR, class IA, typename F>
__device__ __forceinline__ void spmv_rows_ia(int n, int q, int ldn, int T,
                                             const int32_t *__restrict__ col,
                                             const typename IA::S *__restrict__ val,
                                             typename IA::S *const *xs, int wglobal, int nwarps,
                                             F &&f) {
  using S = typename IA::S;
  using AC = typename IA::A;
  constexpr int CH = kdev::CH;
  const int lane = threadIdx.x & 31;
  const int gpw = 32 / T;
  const int g = lane / T;
  const int lg = lane - g * T;
  const bool active = g < gpw;
  const int wpb = blockDim.x >> 5;
  int r0, r1, w;
  kdev::cta_rows(n, wglobal, nwarps, wpb, r0, r1, w);
  for (int base = r0 + w * gpw; base < r1; base += wpb * gpw) {
    const int i = base + g;
    const bool valid = active && i < r1;
    AC s[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) s[k] = IA::zero();
    if (valid) {
      for (int j0 = lg; j0 < q; j0 += CH * T) {
        int c[CH];
        S a[CH];
#pragma unroll
        for (int u = 0; u < CH; ++u) {
          const int j = j0 + u * T;
          const int64_t e = (int64_t)j * ldn + i;
          c[u] = j < q ? __ldg(col + e) : -1;
          a[u] = j < q ? IA::ldg(val + e) : IA::szero();
        }
#pragma unroll
        for (int u = 0; u < CH; ++u) {
          if (c[u] >= 0) {
#pragma unroll
            for (int k = 0; k < NR; ++k) IA::madd(s[k], a[u], IA::ldcg(xs[k] + c[u]));
          }
        }
      }
    }
    AC tot[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) tot[k] = s[k];
    for (int u = 1; u < T; ++u) {
#pragma unroll
      for (int k = 0; k < NR; ++k) tot[k] = IA::add(tot[k], IA::shfl(s[k], (lane + u) & 31));
    }
    if (valid && lg == 0) f(i, tot);
  }
}

// y_k(i) = sum_j A(i,j) g(k, j) where the operand g is formed on the fly
// from several gathered vectors (the "fused" SpMVs below).  Same thread
// layout as spmv_rows_ia; g runs once per stored entry.
template <int NR, class IA, typename G, typename F>
__device__ __forceinline__ void spmv_rows_gen(int n, int q, int ldn, int T,
                                              const int32_t *__restrict__ col,
                                              const typename IA::S *__restrict__ val, G &&g,
                                              int wglobal, int nwarps, F &&f) {
  using S = typename IA::S;
  using AC = typename IA::A;
  constexpr int CH = kdev::CH;
  const int lane = threadIdx.x & 31;
  const int gpw = 32 / T;
  const int gi = lane / T;
  const int lg = lane - gi * T;
  const bool active = gi < gpw;
  const int wpb = blockDim.x >> 5;
  int r0, r1, w;
  kdev::cta_rows(n, wglobal, nwarps, wpb, r0, r1, w);
  // With dynamic shared memory (kdev::win_init ran), the operand is formed
  // once per entry of this CTA's column window into shared memory (one
  // coalesced pass over its source vectors) and gathered from there: one
  // shared-memory read per stored entry instead of the source vectors'
  // gathers from L2.  Columns outside the window form it directly.  Either
  // way g computes the same value.
  const kdev::RowWindow rw = kdev::row_window();
  const int wlen = kdev::win_cap() > 0 ? rw.w1 - rw.w0 : 0;
  S *wb[NR];
  if (wlen > 0) {
    __syncthreads();  // the buffers' previous use
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      wb[k] = reinterpret_cast<S *>(kdev::kdev_dyn + (size_t)k * kdev::win_cap() * 8);
      for (int t = threadIdx.x; t < wlen; t += blockDim.x) wb[k][t] = g(k, rw.w0 + t);
    }
    __syncthreads();
  }
  auto gw = [&](int k, int c) -> S {
    const unsigned int o = (unsigned int)(c - rw.w0);
    return o < (unsigned int)wlen ? wb[k][o] : g(k, c);
  };
  for (int base = r0 + w * gpw; base < r1; base += wpb * gpw) {
    const int i = base + gi;
    const bool valid = active && i < r1;
    AC s[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) s[k] = IA::zero();
    if (valid) {
      for (int j0 = lg; j0 < q; j0 += CH * T) {
        int c[CH];
        S a[CH];
#pragma unroll
        for (int u = 0; u < CH; ++u) {
          const int j = j0 + u * T;
          const int64_t e = (int64_t)j * ldn + i;
          c[u] = j < q ? __ldg(col + e) : -1;
          a[u] = j < q ? IA::ldg(val + e) : IA::szero();
        }
#pragma unroll
        for (int u = 0; u < CH; ++u) {
          if (c[u] >= 0) {
#pragma unroll
            for (int k = 0; k < NR; ++k) IA::madd(s[k], a[u], gw(k, c[u]));
          }
        }
      }
    }
    AC tot[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) tot[k] = s[k];
    for (int u = 1; u < T; ++u) {
#pragma unroll
      for (int k = 0; k < NR; ++k) tot[k] = IA::add(tot[k], IA::shfl(s[k], (lane + u) & 31));
    }
    if (valid && lg == 0) f(i, tot);
  }
}

// The solve of one system (NR right-hand sides) by the nb CTAs that share
// it; this CTA is number lb among them.
template <int NR, int NT, class IA>
__device__ __forceinline__ void bicgstab_ir_body(const MixedArgs &A, const int lb, const int nb) {
  using S = typename IA::S;
  using AC = typename IA::A;
  using PT = typename IA::P;
  using CF = typename IA::C;
  // block-partial staging for the inner sums (5 NR values) and the FP64
  // residual sums (2 NR values); never live at the same time
  constexpr size_t SB = (5 * NR * NT * sizeof(PT) > 2 * NR * NT * sizeof(double))
                            ? 5 * NR * NT * sizeof(PT)
                            : 2 * NR * NT * sizeof(double);
  __shared__ __align__(16) unsigned char sbuf[SB];
  PT *sr32 = reinterpret_cast<PT *>(sbuf);
  double *sr64 = reinterpret_cast<double *>(sbuf);
  __shared__ PT st32[16];
  __shared__ double st64[16];
  __shared__ IRS ks[NR];
  __shared__ int s_any;
  const int tid = lb * NT + threadIdx.x;
  const int stride = nb * NT;
  const int wglobal = tid >> 5, nwarps = stride >> 5;
  const int n = A.n, q = A.q, ldn = A.ldn, T = A.tpr;
  unsigned int epoch = 1;
  const bool leader = threadIdx.x == 0;
  int *err = &A.bar->err;
  const S *val = reinterpret_cast<const S *>(A.valin);
  const S *dinv = reinterpret_cast<const S *>(A.dinvin);
  // p and v are double-buffered: an iteration reads the previous direction
  // of its neighbours while it writes its own new one
  S *r[NR], *rh[NR], *pb[2][NR], *vb[2][NR], *sv[NR], *t[NR], *d[NR];
#pragma unroll
  for (int k = 0; k < NR; ++k) {
    r[k] = (S *)A.w[k].r;
    rh[k] = (S *)A.w[k].rh;
    pb[0][k] = (S *)A.w[k].p0;
    pb[1][k] = (S *)A.w[k].p1;
    vb[0][k] = (S *)A.w[k].v0;
    vb[1][k] = (S *)A.w[k].v1;
    sv[k] = (S *)A.w[k].s;
    t[k] = (S *)A.w[k].t;
    d[k] = (S *)A.w[k].d;
  }
  PT *part32 = reinterpret_cast<PT *>(A.partin);
  auto P64 = [&](int slot, int k) { return A.part64 + (size_t)(slot * NR + k) * nb; };
  auto P32 = [&](int slot, int k) { return part32 + (size_t)(slot * NR + k) * nb; };

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
    // ---------------- R: FP64 residual, then r = r^ = p = residual, p^ = r/d, d = 0
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
                                    const S di = IA::ldg(dinv + i);
#pragma unroll
                                    for (int k = 0; k < NR; ++k) {
                                      if (!part[k]) continue;
                                      const double bi = A.b[k][i];
                                      const double ri = bi - ax[k];
                                      const S rf = IA::from_double(ri);
                                      (void)di;
                                      // the first inner iteration forms
                                      // r = s - 0 t and p = r + 0 (p - 0 v)
                                      sv[k][i] = rf;
                                      rh[k][i] = rf;
                                      t[k][i] = IA::szero();
                                      pb[0][k][i] = IA::szero();
                                      vb[0][k][i] = IA::szero();
                                      d[k][i] = IA::szero();
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
      kdev::block_partials<NT, 2 * NR>(acc, sr64, outs, lb);
      double tot[2 * NR];
      ok = kdev::exchange<2 * NR>(A.flags, err, epoch++, outs, tot, st64, lb, nb);
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
          c.alpha = c.omega = c.beta = 0.0;
          c.half = 0;
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

    // ---------------- inner BiCGSTAB on A d = r in the inner arithmetic,
    // two grid exchanges per iteration:
    //   A: with alpha, omega of the previous iteration and the new beta,
    //      each row forms r = s - omega t, advances d by alpha p^ + omega s^,
    //      forms p = r + beta (p - omega v), and the SpMV builds
    //      p^_j = d_j (s_j - omega t_j + beta (p_j - omega v_j)) on the fly
    //      from its neighbours' previous vectors: v = A p^; partials (r^,v), (r,r)
    //   C: s = r - alpha v; t = A s^ with s^_j = d_j (r_j - alpha v_j) formed
    //      on the fly; partials (s,s) (t,t) (t,s) (r^,s) (r^,t) give omega,
    //      rho' = (r^,s) - omega (r^,t) and beta.
    // On the FP32 pipe the extra operand arithmetic is cheap; what it saves
    // is two of the four grid-wide round trips of the textbook order.
    int pv = 0;  // buffer holding the previous p and v
    for (;;) {
      bool run[NR], anyrun = false;
#pragma unroll
      for (int k = 0; k < NR; ++k) {
        run[k] = ks[k].inner != 0;
        anyrun |= run[k];
      }
      __syncthreads();
      if (!anyrun) break;
      const int cu = pv ^ 1;

      // A
      {
        CF alp[NR], omg[NR], nomg[NR], bet[NR];
#pragma unroll
        for (int k = 0; k < NR; ++k) {
          alp[k] = IA::coef(ks[k].alpha);
          omg[k] = IA::coef(ks[k].omega);
          nomg[k] = IA::coef(-ks[k].omega);
          bet[k] = IA::coef(ks[k].beta);
        }
        AC acc[2 * NR];
#pragma unroll
        for (int k = 0; k < 2 * NR; ++k) acc[k] = IA::zero();
        auto g = [&](int k, int j) {
          const S rj = IA::axpy(IA::ldcg(sv[k] + j), nomg[k], IA::ldcg(t[k] + j));
          const S qj = IA::axpy(IA::ldcg(pb[pv][k] + j), nomg[k], IA::ldcg(vb[pv][k] + j));
          return IA::mul(IA::axpy(rj, bet[k], qj), IA::ldg(dinv + j));
        };
        spmv_rows_gen<NR, IA>(n, q, ldn, T, A.col, val, g, wglobal, nwarps,
                              [&](int i, const AC *av) {
                                const S di = IA::ldg(dinv + i);
#pragma unroll
                                for (int k = 0; k < NR; ++k) {
                                  if (!run[k]) continue;
                                  const S si = sv[k][i], ti = t[k][i];
                                  const S pi = pb[pv][k][i], vi = vb[pv][k][i];
                                  const S ri = IA::axpy(si, nomg[k], ti);
                                  r[k][i] = ri;
                                  d[k][i] = IA::axpy(IA::axpy(d[k][i], alp[k], IA::mul(pi, di)),
                                                     omg[k], IA::mul(si, di));
                                  pb[cu][k][i] = IA::axpy(ri, bet[k], IA::axpy(pi, nomg[k], vi));
                                  const S vn = IA::from_acc(av[k]);
                                  vb[cu][k][i] = vn;
                                  IA::madd(acc[2 * k], rh[k][i], vn);
                                  IA::madd(acc[2 * k + 1], ri, ri);
                                }
                              });
        PT pa[2 * NR];
        PT *outs[2 * NR];
#pragma unroll
        for (int k = 0; k < NR; ++k) {
          pa[2 * k] = IA::part(acc[2 * k]);
          pa[2 * k + 1] = IA::part(acc[2 * k + 1]);
          outs[2 * k] = run[k] ? P32(F_RHV, k) : nullptr;
          outs[2 * k + 1] = run[k] ? P32(F_RR, k) : nullptr;
        }
        kdev::block_partials<NT, 2 * NR>(pa, sr32, outs, lb);
        PT tot[2 * NR];
        ok = kdev::exchange<2 * NR>(A.flags, err, epoch++, outs, tot, st32, lb, nb);
        if (!ok) break;
        if (leader) {
#pragma unroll
          for (int k = 0; k < NR; ++k) {
            IRS &c = ks[k];
            if (!run[k]) continue;
            const double rn = sqrt(IA::pd(tot[2 * k + 1]));
            // d now holds every step up to the previous iteration
            if (!isfinite(rn) || (c.inner_it > 0 && rn <= A.inner_tol * c.r0) ||
                rn > 1e3 * c.r0 || c.inner_it >= A.inner_maxit || c.it >= A.maxit) {
              c.inner = 0;
              continue;
            }
            const double al = c.rho / IA::pd(tot[2 * k]);
            if (!isfinite(al) || fabs(al) > 1e30) {
              c.inner = 0;  // breakdown: keep the correction so far
              continue;
            }
            c.alpha = al;
          }
        }
        __syncthreads();
        pv = cu;
#pragma unroll
        for (int k = 0; k < NR; ++k) run[k] = ks[k].inner != 0;
      }
      bool anyc = false;
#pragma unroll
      for (int k = 0; k < NR; ++k) anyc |= run[k];
      if (!anyc) continue;

      // C
      {
        CF nalp[NR];
#pragma unroll
        for (int k = 0; k < NR; ++k) nalp[k] = IA::coef(-ks[k].alpha);
        AC acc[5 * NR];
#pragma unroll
        for (int k = 0; k < 5 * NR; ++k) acc[k] = IA::zero();
        auto g = [&](int k, int j) {
          return IA::mul(IA::axpy(IA::ldcg(r[k] + j), nalp[k], IA::ldcg(vb[pv][k] + j)),
                         IA::ldg(dinv + j));
        };
        spmv_rows_gen<NR, IA>(n, q, ldn, T, A.col, val, g, wglobal, nwarps,
                              [&](int i, const AC *at) {
#pragma unroll
                                for (int k = 0; k < NR; ++k) {
                                  if (!run[k]) continue;
                                  const S si = IA::axpy(r[k][i], nalp[k], vb[pv][k][i]);
                                  sv[k][i] = si;
                                  const S ti = IA::from_acc(at[k]);
                                  t[k][i] = ti;
                                  const S rhi = rh[k][i];
                                  IA::madd(acc[5 * k + 0], si, si);
                                  IA::madd(acc[5 * k + 1], ti, ti);
                                  IA::madd(acc[5 * k + 2], ti, si);
                                  IA::madd(acc[5 * k + 3], rhi, si);
                                  IA::madd(acc[5 * k + 4], rhi, ti);
                                }
                              });
        PT pa[5 * NR];
        PT *outs[5 * NR];
#pragma unroll
        for (int k = 0; k < NR; ++k) {
#pragma unroll
          for (int j = 0; j < 5; ++j) pa[5 * k + j] = IA::part(acc[5 * k + j]);
          outs[5 * k + 0] = run[k] ? P32(F_SS, k) : nullptr;
          outs[5 * k + 1] = run[k] ? P32(F_TT, k) : nullptr;
          outs[5 * k + 2] = run[k] ? P32(F_TS, k) : nullptr;
          outs[5 * k + 3] = run[k] ? P32(F_RHS, k) : nullptr;
          outs[5 * k + 4] = run[k] ? P32(F_RHT, k) : nullptr;
        }
        kdev::block_partials<NT, 5 * NR>(pa, sr32, outs, lb);
        PT tot[5 * NR];
        ok = kdev::exchange<5 * NR>(A.flags, err, epoch++, outs, tot, st32, lb, nb);
        if (!ok) break;
        if (leader) {
#pragma unroll
          for (int k = 0; k < NR; ++k) {
            IRS &c = ks[k];
            c.half = 0;
            if (!run[k]) continue;
            const double ss = IA::pd(tot[5 * k + 0]), tt = IA::pd(tot[5 * k + 1]);
            const double ts = IA::pd(tot[5 * k + 2]);
            const double rhs = IA::pd(tot[5 * k + 3]), rht = IA::pd(tot[5 * k + 4]);
            c.it++;
            c.inner_it++;
            c.snorm = sqrt(ss);
            const double om = tt == 0.0 ? 0.0 : ts / tt;
            const double rho_new = rhs - om * rht;
            const double be = (om == 0.0 || c.rho == 0.0) ? 0.0 : (rho_new / c.rho) * (c.alpha / om);
            if (!isfinite(c.snorm) || c.snorm > 1e3 * c.r0 || c.snorm <= A.inner_tol * c.r0 ||
                !isfinite(om) || !isfinite(be) || fabs(be) > 1e30 || om == 0.0 ||
                rho_new == 0.0) {
              // stop after the half step d += alpha p^ (valid whenever alpha
              // is finite); a non-finite s drops the step altogether
              c.half = isfinite(c.snorm) && c.snorm <= 1e3 * c.r0 ? 1 : 2;
              c.inner = 0;
              continue;
            }
            c.omega = om;
            c.beta = be;
            c.rho = rho_new;
          }
        }
        __syncthreads();
        // half step of the iterations that stopped here
        bool fin[NR], anyfin = false;
#pragma unroll
        for (int k = 0; k < NR; ++k) {
          fin[k] = run[k] && ks[k].half == 1;
          anyfin |= fin[k];
        }
        if (anyfin) {
          CF alp[NR];
#pragma unroll
          for (int k = 0; k < NR; ++k) alp[k] = IA::coef(ks[k].alpha);
          const int lane = threadIdx.x & 31, gi = lane / T, lg = lane - gi * T;
          // the rows this thread owns are the ones its SpMV leader lane wrote
          int r0, r1, wb;
          kdev::cta_rows(n, wglobal, nwarps, NT >> 5, r0, r1, wb);
          for (int base = r0 + wb * (32 / T); base < r1; base += (32 / T) * (NT >> 5)) {
            const int i = base + gi;
            if (gi < 32 / T && lg == 0 && i < r1) {
              const S di = IA::ldg(dinv + i);
#pragma unroll
              for (int k = 0; k < NR; ++k)
                if (fin[k]) d[k][i] = IA::axpy(d[k][i], alp[k], IA::mul(pb[pv][k][i], di));
            }
          }
        }
      }
    }
    if (!ok) break;
    // ---------------- x += d (FP64); every step that could make d non-finite
    // ended the sweep before its update
    {
      bool upd[NR];
#pragma unroll
      for (int k = 0; k < NR; ++k) upd[k] = ks[k].in_sweep != 0;
      {
        // d of a row was written by its SpMV leader lane: update x there too
        const int lane = threadIdx.x & 31, gi = lane / T, lg = lane - gi * T;
        int r0, r1, wb;
        kdev::cta_rows(n, wglobal, nwarps, NT >> 5, r0, r1, wb);
        for (int base = r0 + wb * (32 / T); base < r1; base += (32 / T) * (NT >> 5)) {
          const int i = base + gi;
          if (gi < 32 / T && lg == 0 && i < r1) {
#pragma unroll
            for (int k = 0; k < NR; ++k)
              if (upd[k]) A.x[k][i] = A.x[k][i] + IA::to_double(d[k][i]);
          }
        }
      }
      if (leader) {
#pragma unroll
        for (int k = 0; k < NR; ++k)
          if (upd[k]) ks[k].sweeps++;
      }
      ok = kdev::exchange<0, double>(A.flags, err, epoch++, nullptr, nullptr, st64, lb, nb);
      if (!ok) break;
    }
  }

  if (lb == 0 && leader) {
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      A.out[k].iters = ks[k].it;
      A.out[k].restarts = ks[k].sweeps;
      A.out[k].status = ok ? ks[k].state : KRY_TIMEOUT;
      A.out[k].relres = ks[k].relres;
    }
  }
}

template <int NR, int NT, class IA>
__global__ void __launch_bounds__(NT) k_bicgstab_ir(MixedArgs A) {
  // this CTA's column window for the staged SpMV operands (kdev::win_init)
  {
    const int wpb = NT / 32;
    int r0, r1, w;
    kdev::cta_rows(A.n, blockIdx.x * wpb, gridDim.x * wpb, wpb, r0, r1, w);
    kdev::win_init(A.n, A.q, A.ldn, A.col, r0, r1);
  }
  bicgstab_ir_body<NR, NT, IA>(A, blockIdx.x, gridDim.x);
}

// Batched launch: system cta_sys[b] owns the consecutive CTAs from
// cta_first[s] and synchronises only with them.
template <int NR, int NT, class IA>
__global__ void __launch_bounds__(NT) k_bicgstab_ir_batch(const MixedArgs *__restrict__ sys,
                                                          const int *__restrict__ cta_sys,
                                                          const int *__restrict__ cta_first) {
  __shared__ MixedArgs A;
  // persistent work list (batch.cu: plan_teams): this CTA's team solves
  // the systems cta_first[j0 .. j1) one after another
  const int t = cta_sys[blockIdx.x];
  const int c0 = cta_first[4 * t], nc = cta_first[4 * t + 1];
  const int j0 = cta_first[4 * t + 2], j1 = cta_first[4 * t + 3];
  for (int j = j0; j < j1; ++j) {
    __syncthreads();
    if (threadIdx.x == 0) A = sys[cta_first[j]];
    __syncthreads();
    bicgstab_ir_body<NR, NT, IA>(A, blockIdx.x - c0, nc);
  }
}

namespace {
constexpr int MT1 = 1024;
constexpr int MT2 = 512;
// dynamic shared memory of the single-problem launch: the staged column
// windows (kdev::win_cap: two 8-byte slots an entry, 4 096 entries)
constexpr int IR_WIN_BYTES = 64 * 1024;

template <class IA>
int max_blocks_ia(rbffd_ctx *ctx, int nr) {
  int per_sm = 0;
  cudaError_t e;
  if (nr == 1) {
    cudaFuncSetAttribute(k_bicgstab_ir<1, MT1, IA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         IR_WIN_BYTES);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bicgstab_ir<1, MT1, IA>, MT1,
                                                      IR_WIN_BYTES);
  } else {
    cudaFuncSetAttribute(k_bicgstab_ir<2, MT2, IA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         IR_WIN_BYTES);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bicgstab_ir<2, MT2, IA>, MT2,
                                                      IR_WIN_BYTES);
  }
  if (e != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    return 0;
  }
  return per_sm * ctx->num_sms;
}
}  // namespace

int krylov_ir_max_blocks(rbffd_ctx *ctx, int nr, int inner) {
  return inner == INNER_FF ? max_blocks_ia<ArithFF>(ctx, nr) : max_blocks_ia<ArithF32>(ctx, nr);
}

int krylov_ir_launch(rbffd_ctx *ctx, int nr, int nblocks, const MixedArgs &args) {
  if (nblocks < 1 || nblocks > kdev::MAXB || nblocks > krylov_ir_max_blocks(ctx, nr, args.inner)) {
    set_error("krylov_ir_launch: %d blocks not co-resident", nblocks);
    return RBFFD_EINVAL;
  }
  RBFFD_TRY(reset_barriers(ctx, args.bar, 1));
  RBFFD_CK(cudaMemsetAsync(args.flags, 0, sizeof(unsigned int) * nblocks, ctx->stream));
  void *kargs[] = {(void *)&args};
  const void *fn;
  const int nt = nr == 1 ? MT1 : MT2;
  if (args.inner == INNER_FF)
    fn = nr == 1 ? (const void *)k_bicgstab_ir<1, MT1, ArithFF>
                 : (const void *)k_bicgstab_ir<2, MT2, ArithFF>;
  else
    fn = nr == 1 ? (const void *)k_bicgstab_ir<1, MT1, ArithF32>
                 : (const void *)k_bicgstab_ir<2, MT2, ArithF32>;
  cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(nblocks), dim3(nt), kargs, IR_WIN_BYTES,
                                              ctx->stream);
  ctx->launches++;
  if (e != cudaSuccess) {
    set_error("cooperative launch of k_bicgstab_ir failed: %s", cudaGetErrorString(e));
    return RBFFD_ECUDA;
  }
  return RBFFD_OK;
}

namespace {
template <int NR, class IA>
const void *ir_batch_fn() {
  return (const void *)k_bicgstab_ir_batch<NR, KB_NT, IA>;
}
const void *ir_batch_kernel(int nr, int inner) {
  if (inner == INNER_FF) return nr == 1 ? ir_batch_fn<1, ArithFF>() : ir_batch_fn<2, ArithFF>();
  return nr == 1 ? ir_batch_fn<1, ArithF32>() : ir_batch_fn<2, ArithF32>();
}
}  // namespace

int krylov_ir_batch_max_ctas(rbffd_ctx *ctx, int nr, int inner) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ir_batch_kernel(nr, inner), KB_NT,
                                                    0) != cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    return 0;
  }
  return per_sm * ctx->num_sms;
}

int krylov_ir_batch_launch(rbffd_ctx *ctx, int nr, int inner, int nctas, const MixedArgs *d_sys,
                           const int *d_cta_sys, const int *d_cta_first) {
  if (nctas < 1 || nctas > krylov_ir_batch_max_ctas(ctx, nr, inner)) {
    set_error("krylov_ir_batch_launch: %d CTAs are not co-resident", nctas);
    return RBFFD_EINVAL;
  }
  void *kargs[] = {(void *)&d_sys, (void *)&d_cta_sys, (void *)&d_cta_first};
  cudaError_t e = cudaLaunchCooperativeKernel(ir_batch_kernel(nr, inner), dim3(nctas),
                                              dim3(KB_NT), kargs, 0, ctx->stream);
  ctx->launches++;
  if (e != cudaSuccess) {
    set_error("cooperative launch of k_bicgstab_ir_batch failed: %s", cudaGetErrorString(e));
    return RBFFD_ECUDA;
  }
  return RBFFD_OK;
}

size_t krylov_ir_partials64(int nr, int nblocks) { return (size_t)M_COUNT64 * nr * nblocks; }
// bytes of the inner partials (double for float-float, float for FP32)
size_t krylov_ir_partials_inner_bytes(int nr, int nblocks, int inner) {
  return (size_t)F_COUNT32 * nr * nblocks * (inner == INNER_FF ? sizeof(double) : sizeof(float));
}

}  // namespace rbffd
