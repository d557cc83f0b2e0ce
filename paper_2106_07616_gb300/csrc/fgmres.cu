// fgmres.cu -- restarted flexible GMRES(m) for the pressure-correction
// system, right-preconditioned by one FP32 multigrid V-cycle per Arnoldi
// step, as ONE persistent cooperative kernel per solve.
//
// The paper solves the p' equation with a preconditioned BiCGSTAB and does
// not fix the preconditioner (Sec. 3).  On GB300 an FP64 warp instruction
// occupies the FP64 pipe for ~32 cycles, against one for FP32, so the solve
// keeps FP64 only where the answer's accuracy lives:
//
//   * each restart computes the true residual r = b - A x in FP64 and ends
//     by x += Z y in FP64: the restarts are an FP64 iterative refinement
//     (GMRES-based refinement, Carson & Higham 2018), and the solve stops
//     only when the FP64 relative residual is at the tolerance;
//   * inside a restart the Arnoldi process runs in FP32 -- basis V,
//     directions Z, w = A z_j with the FP32 copy of A, classical
//     Gram-Schmidt with one reorthogonalisation, the cycle -- which only has
//     to reduce the residual by the restart's factor (~1e-3), far above
//     FP32 rounding;
//   * the small Hessenberg least-squares problem (Givens rotations, the
//     triangular solve) runs on one thread in FP32 like the Arnoldi
//     entries it holds, on the system scaled by 1 / beta (g_0 = 1), so its
//     range does not depend on the residual's size; beta multiplies back
//     in the FP64 update of x.
//
// Flexible GMRES (Saad 1993) keeps every preconditioned direction
// z_j = M_j^-1 v_j, so a cycle whose rounding differs per input only slows
// it (BiCGSTAB cannot take that cycle, see amg.cuh).
//
// Per Arnoldi step: the cycle (2L - 1 grid exchanges), w = A z_j with the
// dot products (w, v_i) (one exchange: SpMV and dots use this block's
// contiguous rows), the reorthogonalised w' with its dots (one exchange),
// and v_{j+1} = w'' / h_{j+1,j} published (one exchange) while thread 0
// applies the Givens rotations.  Reductions run in a fixed order, so every
// block holds bit-identical scalars and takes the same branches.
#include "amg_dev.cuh"
#include "fgmres.cuh"
#include "krylov_dev.cuh"

namespace rbffd {

namespace {

constexpr int FNT = 1024;
constexpr int FG_D = FG_MAXM + 2;  // dot products one exchange reduces (2 FG_D delayed)
constexpr int LDH = FG_MAXM + 1;   // leading dimension of the Hessenberg matrix
constexpr int GB = 8;              // loads a lane keeps in flight in the loops below
// dynamic shared memory of the single-problem launch: windows of up to
// 4 096 entries (two FP64 vectors' worth; kdev::win_cap)
constexpr int FG_WIN_BYTES = 64 * 1024;
using kdev::MAXB;

// barrier `id` among the first `nthreads` threads that reach it (a multiple
// of 32); id 0 with the whole block is __syncthreads
__device__ __forceinline__ void bar_sync(int id, int nthreads) {
  if (id == 0)
    __syncthreads();
  else
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// (A x)_i for the rows [r0, r1) of this block, T threads per row, summed in
// AT: f(i, Ax_i) on the row's first lane.  Gathers of x go through L2
// (written in this launch).
template <typename AT, typename VT, typename XT, typename F>
__device__ __forceinline__ void block_spmv(int r0, int r1, int q, int ldn, int T,
                                           const int32_t *__restrict__ col,
                                           const VT *__restrict__ val, const XT *x, F &&f) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int gpw = 32 / T, g = lane / T, lg = lane - g * T;
  const bool active = g < gpw;
  // x's window over this block's rows, staged in shared memory (win_init)
  const kdev::RowWindow rw = kdev::row_window();
  const int wlen = kdev::win_cap() > 0 ? rw.w1 - rw.w0 : 0;
  const XT *wb = wlen > 0 ? kdev::win_stage<XT>(x, rw.w0, rw.w1) : nullptr;
  for (int base = r0 + warp * gpw; base < r1; base += nw * gpw) {
    const int i = base + g;
    const bool valid = active && i < r1;
    AT s = AT(0);
    if (valid) {
      for (int j0 = lg; j0 < q; j0 += kdev::CH * T) {
        int c[kdev::CH];
        VT a[kdev::CH];
#pragma unroll
        for (int u = 0; u < kdev::CH; ++u) {
          const int j = j0 + u * T;
          const int64_t e = (int64_t)j * ldn + i;
          c[u] = j < q ? __ldg(col + e) : -1;
          a[u] = j < q ? __ldg(val + e) : VT(0);
        }
#pragma unroll
        for (int u = 0; u < kdev::CH; ++u)
          if (c[u] >= 0) s += AT(a[u]) * AT(kdev::win_get<XT>(wb, rw.w0, wlen, x, c[u]));
      }
    }
    AT tot = s;
    for (int u = 1; u < T; ++u) tot += __shfl_sync(0xffffffffu, s, (lane + u) & 31);
    if (valid && lg == 0) f(i, tot);
  }
}

// Block partials of the FP32 dot products (w, u_d), d <= nv, over rows
// [r0, r1): warp d takes product d (u_d = V_d for d < nv, u_d = w for
// d = nv), each lane GB rows per round.  Partial d of block lb goes to
// part[d * MAXB + lb].
__device__ __forceinline__ void block_dots(int r0, int r1, int n, const float *w,
                                           const float *V, int nv, float *part, int lb) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int d = warp; d <= nv; d += nw) {
    const float *u = d < nv ? V + (size_t)d * n : w;
    float t = 0.0f;
    for (int r = r0 + lane; r < r1; r += 32 * GB) {
      float a[GB], b[GB];
#pragma unroll
      for (int k = 0; k < GB; ++k) {
        const int rr = r + 32 * k;
        a[k] = rr < r1 ? __ldcg(w + rr) : 0.0f;
        b[k] = rr < r1 ? __ldcg(u + rr) : 0.0f;
      }
#pragma unroll
      for (int k = 0; k < GB; ++k) t += a[k] * b[k];
    }
    t = kdev::wsum(t);
    if (lane == 0) part[d * MAXB + lb] = t;
  }
}

// The one reduction of a step with delayed reorthogonalisation: over rows
// [r0, r1), the products (u, V_i) for i < j, (w, V_i) for i < j, (u, u) and
// (u, w), 2 j + 2 in all, partial d of block lb to part[d * MAXB + lb]
// (u: the step's once-orthogonalised basis vector, w = A z_j).
__device__ __forceinline__ void block_dots2(int r0, int r1, int n, const float *u,
                                            const float *w, const float *V, int j, float *part,
                                            int lb) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int d = warp; d < 2 * j + 2; d += nw) {
    const float *x = d < j ? u : (d < 2 * j ? w : u);
    const float *y = d < j ? V + (size_t)d * n
                           : (d < 2 * j ? V + (size_t)(d - j) * n : (d == 2 * j ? u : w));
    float t = 0.0f;
    for (int r = r0 + lane; r < r1; r += 32 * GB) {
      float a[GB], b[GB];
#pragma unroll
      for (int k = 0; k < GB; ++k) {
        const int rr = r + 32 * k;
        a[k] = rr < r1 ? __ldcg(x + rr) : 0.0f;
        b[k] = rr < r1 ? __ldcg(y + rr) : 0.0f;
      }
#pragma unroll
      for (int k = 0; k < GB; ++k) t += a[k] * b[k];
    }
    t = kdev::wsum(t);
    if (lane == 0) part[d * MAXB + lb] = t;
  }
}

// After every block has published its partials: exchange, then the D totals
// in a fixed order into tot[0..D).  False if a wait gave up.
template <typename T>
__device__ __forceinline__ bool reduce_all(const amgdev::Ctx &c, const T *part, int D, T *tot,
                                           unsigned int &epoch) {
  if (!amgdev::sync(c, epoch)) return false;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int d = warp; d < D; d += nw) {
    T t = T(0);
    for (int b = lane; b < c.nb; b += 32) t += __ldcg(part + d * MAXB + b);
    t = kdev::wsum(t);
    if (lane == 0) tot[d] = t;
  }
  __syncthreads();
  return true;
}

// out_r = (base_r + sgn * sum_{i<k} coef_i U_i[r]) * scale, summed in AT,
// for the rows [r0, r1) of this block (U_i = U + i n), run by the nthr
// threads t0 .. t0 + nthr - 1, which meet at barrier bid.  With R = r1 - r0
// rows and g = nthr / R > 1, g threads share a row, each taking every g-th
// vector, and their partial sums meet in red[] (nthr entries) in a fixed
// order; every thread keeps GB loads in flight.  out may alias base.
template <typename AT, typename UT, typename CT, typename BT, typename OT>
__device__ __forceinline__ void block_combine(int r0, int r1, int n, const UT *U, int k,
                                              const CT *coef, const BT *base, OT *out, AT sgn,
                                              AT scale, AT *red, int t0, int nthr, int bid) {
  const int R = r1 - r0;
  const int tid = (int)threadIdx.x - t0;
  int g = R > 0 ? nthr / R : 1;
  g = g < 1 ? 1 : (g > GB ? GB : g);
  const int sub = g > 1 ? tid / R : 0;
  const int rl0 = g > 1 ? tid - sub * R : tid;
  // the combining thread of a row loads its base value with the vectors
  const AT bv = (g > 1 && tid < R) ? AT(__ldcg(base + r0 + tid)) : AT(0);
  for (int rl = rl0; rl < R && sub < g; rl += (g > 1 ? R : nthr)) {
    const int r = r0 + rl;
    const AT b1 = g == 1 ? AT(__ldcg(base + r)) : AT(0);
    AT t = AT(0);
    for (int i0 = sub; i0 < k; i0 += GB * g) {
      UT a[GB];
#pragma unroll
      for (int u = 0; u < GB; ++u) {
        const int i = i0 + u * g;
        a[u] = i < k ? __ldcg(U + (size_t)i * n + r) : UT(0);
      }
#pragma unroll
      for (int u = 0; u < GB; ++u) {
        const int i = i0 + u * g;
        if (i < k) t += AT(coef[i]) * AT(a[u]);
      }
    }
    if (g == 1) {
      out[r] = OT((b1 + sgn * t) * scale);
    } else {
      red[tid] = t;
      break;  // g > 1: one row per thread
    }
  }
  bar_sync(bid, nthr);
  if (g > 1 && tid < R) {
    AT t = red[tid];
    for (int q = 1; q < g; ++q) t += red[q * R + tid];
    out[r0 + tid] = OT((bv + sgn * t) * scale);
  }
  bar_sync(bid, nthr);
}

struct FgState {
  double bnorm, beta, scale, relres;
  float hn, hinv, hjj;
  int it, restarts, state, k, stop;
};

}  // namespace

// The solve of one system by the nb CTAs that share it; this CTA is number
// lb among them.
template <int NT>
__device__ __forceinline__ void fgmres_body(const FgmresArgs &A, const int lb, const int nb) {
  __shared__ float H[LDH * FG_MAXM];
  __shared__ float cs[FG_MAXM], sn[FG_MAXM], g[FG_MAXM + 1], y[FG_MAXM];
  __shared__ float tot[2 * FG_D];  // up to 2 m + 2 totals (delayed reorthogonalisation)
  __shared__ double tot64[2];
  __shared__ double stot[16];
  __shared__ double sred[2 * NT];
  __shared__ FgState st;
  const int tid = lb * NT + threadIdx.x, stride = nb * NT;
  const int n = A.n, m = A.m;
  const bool leader = threadIdx.x == 0;
  amgdev::Ctx c{n,  A.q, A.ldn,  A.tpr,         A.col,  A.flags, &A.bar->err,
                lb, nb,  tid,    stride,        tid >> 5, stride >> 5, stot};
  unsigned int epoch = 1;
  // this block's row range and its threads per row
  const int R = (n + nb - 1) / nb;
  const int r0 = min(n, lb * R), r1 = min(n, r0 + R);
  int Tb = 1;
  for (int t = 2; t <= 8; ++t)
    if ((32 / t) * (NT / 32) >= R) Tb = t;
  // the column window of this block's rows for the staged gathers of every
  // level-0 SpMV (the solve's own and the cycle's smoother share the columns)
  kdev::win_init(n, A.q, A.ldn, A.col, r0, r1);
  double *p64 = (double *)A.part;  // 2 x MAXB
  float *part0 = (float *)(p64 + 2 * MAXB), *part1 = part0 + FG_D * MAXB;
  float *fred = reinterpret_cast<float *>(sred);
  float *V = A.V, *Z = A.Z;
  bool ok = true;

  if (leader) {
    st.bnorm = st.beta = 0.0;
    st.relres = 1.0;
    st.it = st.restarts = 0;
    st.state = KRY_RUNNING;
    st.stop = 0;
  }
  __syncthreads();

  // ---- r = b - A x (FP64) with (b, b) and (r, r)
  auto residual = [&](bool first) -> bool {
    double bb = 0.0, rr = 0.0;
    block_spmv<double>(r0, r1, A.q, A.ldn, Tb, A.col, A.val, A.x, [&](int i, double ax) {
      const double bi = A.b[i], ri = bi - ax;
      A.r[i] = ri;
      bb += bi * bi;
      rr += ri * ri;
    });
    double v2[2] = {bb, rr};
    double *outs[2] = {p64, p64 + MAXB};
    kdev::block_partials<NT, 2>(v2, sred, outs, lb);
    if (!reduce_all(c, p64, 2, tot64, epoch)) return false;
    if (leader) {
      if (first) st.bnorm = sqrt(tot64[0]);
      st.beta = sqrt(tot64[1]);
      st.scale = st.beta > 0.0 ? 1.0 / st.beta : 0.0;
      st.relres = st.bnorm > 0.0 ? st.beta / st.bnorm : 0.0;
      if (st.bnorm == 0.0) st.state = KRY_OK;
      else if (!(st.relres == st.relres)) st.state = KRY_DIVERGED;
      else if (st.relres <= A.tol) st.state = KRY_OK;
      else if (st.it >= A.maxit) st.state = KRY_NOCONV;
    }
    __syncthreads();
    return true;
  };

  if (!residual(true)) ok = false;
  if (ok && st.bnorm == 0.0) {
    for (int i = tid; i < n; i += stride) A.x[i] = 0.0;
  }

  while (ok && st.state == KRY_RUNNING) {
    // ---- start of a restart: v_0 = r / beta in FP32, published
    {
      const double sc = st.scale;
      for (int i = r0 + (int)threadIdx.x; i < r1; i += NT) V[i] = float(__ldcg(A.r + i) * sc);
      if (leader) {
        g[0] = 1.0f;
        for (int k = 1; k <= FG_MAXM; ++k) g[k] = 0.0f;
        st.k = 0;
      }
      if (!amgdev::sync(c, epoch)) { ok = false; break; }
    }
    int j = 0;
    // column jc of H rotated by the previous Givens rotations and a new one
    // (hn: its subdiagonal entry), the residual estimate updated (thread 0)
    auto rotate = [&](int jc, float hn) {
      float hc = H[LDH * jc];
      for (int i = 0; i < jc; ++i) {
        const float b = H[i + 1 + LDH * jc];
        H[i + LDH * jc] = cs[i] * hc + sn[i] * b;
        hc = -sn[i] * hc + cs[i] * b;
      }
      const float a = hc, b = hn;
      const float rr = sqrtf(a * a + b * b);
      const float ri = rr > 0.0f ? 1.0f / rr : 0.0f;
      cs[jc] = rr > 0.0f ? a * ri : 1.0f;
      sn[jc] = rr > 0.0f ? b * ri : 0.0f;
      H[jc + LDH * jc] = rr;
      H[jc + 1 + LDH * jc] = 0.0f;
      g[jc + 1] = -sn[jc] * g[jc];
      g[jc] = cs[jc] * g[jc];
      st.it++;
      st.k = jc + 1;
      const double est = fabs((double)g[jc + 1]) * st.beta / st.bnorm;
      st.stop = !(est == est) ? 2 : (est <= A.tol || hn == 0.0f || st.it >= A.maxit) ? 1 : 0;
    };
    if (A.reorth == 2) {
      // Delayed reorthogonalisation (DCGS2, Bielich et al. 2022), one
      // reduction a step.  Slot j holds u_j, orthogonalised once and not
      // normalised; z_j = M^-1 u_j (flexible GMRES takes any direction: only
      // w = A z_j must be expanded in the orthonormal basis).  The step's
      // reduction gives a = V^T u_j, b = V^T w, (u_j, u_j), (u_j, w); then
      // v_j = (u_j - V a) / alpha completes column j - 1 (+ a, alpha below
      // the diagonal), column j gets b and h_jj = ((u_j, w) - a.b) / alpha,
      // and u_{j+1} = w - V b - h_jj v_j.  The last column of a restart is
      // completed by one more reduction.
      bool last = true;  // the loop ran to m: column m - 1 still to complete
      for (; j < m; ++j) {
        float *uj = V + (size_t)j * n, *w = V + (size_t)(j + 1) * n, *zj = Z + (size_t)j * n;
        if (!amgdev::vcycle(A.amg, c, uj, zj, epoch)) { ok = false; break; }
        block_spmv<float>(r0, r1, A.q, A.ldn, Tb, A.col, A.val32, zj,
                          [&](int i, float az) { w[i] = az; });
        __syncthreads();
        block_dots2(r0, r1, n, uj, w, V, j, part0, lb);
        if (!reduce_all(c, part0, 2 * j + 2, tot, epoch)) { ok = false; break; }
        if (threadIdx.x < 32) {
          float aa = 0.0f, ab = 0.0f;
          for (int i = threadIdx.x; i < j; i += 32) {
            aa += tot[i] * tot[i];
            ab += tot[i] * tot[j + i];
          }
          aa = kdev::wsum(aa);
          ab = kdev::wsum(ab);
          if (leader) {
            float al = 1.0f;  // v_0 = r / beta is normalised already
            if (j > 0) {
              const float al2 = tot[2 * j] - aa;
              al = al2 > 0.0f ? sqrtf(al2) : 0.0f;
            }
            st.hn = al;
            st.hinv = al > 0.0f ? 1.0f / al : 0.0f;
            st.hjj = al > 0.0f ? (tot[2 * j + 1] - ab) / al : 0.0f;
            st.stop = 0;
            if (j > 0) {
              for (int i = 0; i < j; ++i) H[i + LDH * (j - 1)] += tot[i];
              rotate(j - 1, al);
            }
          }
        }
        __syncthreads();
        if (st.stop == 2) {
          if (leader) st.state = KRY_DIVERGED;
          __syncthreads();
          last = false;
          break;
        }
        if (st.stop) {
          last = false;
          break;
        }
        // v_j = (u_j - sum a_i v_i) / alpha in place (v_0 as it is)
        if (j > 0) block_combine<float>(r0, r1, n, V, j, tot, uj, uj, -1.0f, st.hinv, fred, 0, NT, 0);
        // column j: b_i above, h_jj on the diagonal; coefficients of u_{j+1}
        if ((int)threadIdx.x <= j) {
          const float h = (int)threadIdx.x < j ? tot[j + threadIdx.x] : st.hjj;
          H[threadIdx.x + LDH * j] = h;
          y[threadIdx.x] = h;
        }
        __syncthreads();
        // u_{j+1} = w - sum_{i <= j} h_ij v_i
        block_combine<float>(r0, r1, n, V, j + 1, y, w, w, -1.0f, 1.0f, fred, 0, NT, 0);
        if (j + 1 == m) break;
        if (!amgdev::sync(c, epoch)) { ok = false; break; }
      }
      if (!ok || st.state != KRY_RUNNING) break;
      if (last) {
        // column m - 1: (u_m, v_i), i < m, and (u_m, u_m)
        float *um = V + (size_t)m * n;
        block_dots(r0, r1, n, um, V, m, part0, lb);
        if (!reduce_all(c, part0, m + 1, tot, epoch)) { ok = false; break; }
        if (threadIdx.x < 32) {
          float aa = 0.0f;
          for (int i = threadIdx.x; i < m; i += 32) aa += tot[i] * tot[i];
          aa = kdev::wsum(aa);
          if (leader) {
            const float al2 = tot[m] - aa;
            const float al = al2 > 0.0f ? sqrtf(al2) : 0.0f;
            for (int i = 0; i < m; ++i) H[i + LDH * (m - 1)] += tot[i];
            rotate(m - 1, al);
          }
        }
        __syncthreads();
        if (st.stop == 2) {
          if (leader) st.state = KRY_DIVERGED;
          __syncthreads();
          break;
        }
      }
    } else {
    for (; j < m; ++j) {
      float *vj = V + (size_t)j * n, *w = V + (size_t)(j + 1) * n, *zj = Z + (size_t)j * n;
      // z_j = M^-1 v_j (FP32 cycle), published by its last exchange
      if (!amgdev::vcycle(A.amg, c, vj, zj, epoch)) { ok = false; break; }
      // w = A z_j on this block's rows; dots (w, v_i), i <= j, and (w, w)
      block_spmv<float>(r0, r1, A.q, A.ldn, Tb, A.col, A.val32, zj,
                        [&](int i, float az) { w[i] = az; });
      __syncthreads();
      block_dots(r0, r1, n, w, V, j + 1, part0, lb);
      if (!reduce_all(c, part0, j + 2, tot, epoch)) { ok = false; break; }
      if ((int)threadIdx.x <= j) H[threadIdx.x + LDH * j] = tot[threadIdx.x];
      if (A.reorth) {
        // w' = w - sum h_i v_i; reorthogonalisation dots (w', v_i), (w', w')
        block_combine<float>(r0, r1, n, V, j + 1, tot, w, w, -1.0f, 1.0f, fred, 0, NT, 0);
        block_dots(r0, r1, n, w, V, j + 1, part1, lb);
        if (!reduce_all(c, part1, j + 2, tot, epoch)) { ok = false; break; }
        // column j += the reorthogonalisation coefficients c_i
        if ((int)threadIdx.x <= j) H[threadIdx.x + LDH * j] += tot[threadIdx.x];
      }
      // h_{j+1,j} = sqrt((w', w') - sum c_i^2) by warp 0 in a fixed order
      // (one pass: sqrt((w, w) - sum h_i^2), and v_{j+1} below from w)
      if (threadIdx.x < 32) {
        float q2 = 0.0f;
        for (int i = threadIdx.x; i <= j; i += 32) q2 += tot[i] * tot[i];
        q2 = kdev::wsum(q2);
        if (leader) {
          const float hn2 = tot[j + 1] - q2;
          st.hn = hn2 > 0.0f ? sqrtf(hn2) : 0.0f;
          st.hinv = st.hn > 0.0f ? 1.0f / st.hn : 0.0f;
        }
      }
      __syncthreads();
      if (threadIdx.x < 32) {
        // thread 0: the previous rotations on column j (the rotated entry
        // i + 1 carried in a register), a new one, the residual estimate
        if (leader) {
          const float hn = st.hn;
          float hc = H[LDH * j];
          for (int i = 0; i < j; ++i) {
            const float b = H[i + 1 + LDH * j];
            H[i + LDH * j] = cs[i] * hc + sn[i] * b;
            hc = -sn[i] * hc + cs[i] * b;
          }
          const float a = hc, b = hn;
          const float rr = sqrtf(a * a + b * b);
          const float ri = rr > 0.0f ? 1.0f / rr : 0.0f;
          cs[j] = rr > 0.0f ? a * ri : 1.0f;
          sn[j] = rr > 0.0f ? b * ri : 0.0f;
          H[j + LDH * j] = rr;
          H[j + 1 + LDH * j] = 0.0f;
          g[j + 1] = -sn[j] * g[j];
          g[j] = cs[j] * g[j];
          st.it++;
          st.k = j + 1;
          // estimated relative residual: |g_{j+1}| beta / |b|
          const double est = fabs((double)g[j + 1]) * st.beta / st.bnorm;
          st.stop = !(est == est) ? 2 : (est <= A.tol || hn == 0.0f || st.it >= A.maxit) ? 1 : 0;
        }
      } else {
        // warps 1..: v_{j+1} = (w' - sum c_i v_i) / h_{j+1,j} meanwhile (not
        // used when the restart ends at this step)
        block_combine<float>(r0, r1, n, V, j + 1, tot, w, w, -1.0f, st.hinv, fred, 32, NT - 32,
                             1);
      }
      __syncthreads();
      if (st.stop == 2) {
        if (leader) st.state = KRY_DIVERGED;
        __syncthreads();
        break;
      }
      if (st.stop || j + 1 == m) break;
      if (!amgdev::sync(c, epoch)) { ok = false; break; }
    }
    }
    if (!ok || st.state != KRY_RUNNING) break;
    // ---- y = H^-1 g on the k columns (upper triangular), x += beta Z y in FP64
    if (leader) {
      const int k = st.k;
      for (int i = k - 1; i >= 0; --i) {
        float t = g[i];
        for (int l = i + 1; l < k; ++l) t -= H[i + LDH * l] * y[l];
        y[i] = t / H[i + LDH * i];
      }
    }
    __syncthreads();
    block_combine<double>(r0, r1, n, Z, st.k, y, A.x, A.x, st.beta, 1.0, sred, 0, NT, 0);
    if (!amgdev::sync(c, epoch)) { ok = false; break; }
    if (leader) st.restarts++;
    __syncthreads();
    // ---- true residual; stop or restart from it
    if (!residual(false)) { ok = false; break; }
  }

  if (lb == 0 && leader) {
    A.out->iters = st.it;
    A.out->restarts = st.restarts;
    A.out->status = ok ? st.state : KRY_TIMEOUT;
    A.out->relres = st.relres;
  }
}

template <int NT>
__global__ void __launch_bounds__(NT) k_fgmres(FgmresArgs A) {
  fgmres_body<NT>(A, blockIdx.x, gridDim.x);
}

// Batched launch: system cta_sys[b] owns the consecutive CTAs from
// cta_first[s]; each synchronises only with its system's CTAs.
template <int NT>
__global__ void __launch_bounds__(NT) k_fgmres_batch(const FgmresArgs *__restrict__ sys,
                                                     const int *__restrict__ cta_sys,
                                                     const int *__restrict__ cta_first) {
  __shared__ FgmresArgs A;
  // persistent work list (batch.cu: plan_teams): this CTA's team solves
  // the systems cta_first[j0 .. j1) one after another
  const int t = cta_sys[blockIdx.x];
  const int c0 = cta_first[4 * t], nc = cta_first[4 * t + 1];
  const int j0 = cta_first[4 * t + 2], j1 = cta_first[4 * t + 3];
  for (int j = j0; j < j1; ++j) {
    __syncthreads();
    if (threadIdx.x == 0) A = sys[cta_first[j]];
    __syncthreads();
    fgmres_body<NT>(A, blockIdx.x - c0, nc);
  }
}

size_t fgmres_partials_bytes(int nblocks) {
  (void)nblocks;
  return sizeof(double) * 2 * MAXB + sizeof(float) * 2 * FG_D * MAXB;
}

int fgmres_max_blocks(rbffd_ctx *ctx) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fgmres<FNT>, FNT, 0) !=
          cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    return 0;
  }
  int cap = per_sm * ctx->num_sms;
  if (cap > ctx->num_sms) cap = ctx->num_sms;
  if (cap > MAXB) cap = MAXB;
  return cap;
}

int fgmres_batch_max_ctas(rbffd_ctx *ctx) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fgmres_batch<KB_NT>, KB_NT, 0) !=
          cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    return 0;
  }
  return per_sm * ctx->num_sms;
}

int fgmres_batch_launch(rbffd_ctx *ctx, int nctas, const FgmresArgs *d_sys,
                        const int *d_cta_sys, const int *d_cta_first) {
  if (nctas < 1 || nctas > fgmres_batch_max_ctas(ctx)) {
    set_error("fgmres_batch_launch: %d CTAs are not co-resident", nctas);
    return RBFFD_EINVAL;
  }
  void *kargs[] = {(void *)&d_sys, (void *)&d_cta_sys, (void *)&d_cta_first};
  cudaError_t e = cudaLaunchCooperativeKernel((const void *)k_fgmres_batch<KB_NT>, dim3(nctas),
                                              dim3(KB_NT), kargs, 0, ctx->stream);
  ctx->launches++;
  if (e != cudaSuccess) {
    set_error("cooperative launch of k_fgmres_batch failed: %s", cudaGetErrorString(e));
    return RBFFD_ECUDA;
  }
  return RBFFD_OK;
}

int fgmres_launch(rbffd_ctx *ctx, int nblocks, const FgmresArgs &args) {
  if (nblocks < 1 || nblocks > MAXB || args.m < 1 || args.m > FG_MAXM || !args.amg ||
      !args.val32 || ((uintptr_t)args.part & 7) != 0) {
    set_error("fgmres_launch: bad arguments (blocks %d, m %d)", nblocks, args.m);
    return RBFFD_EINVAL;
  }
  RBFFD_TRY(reset_barriers(ctx, args.bar, 1));
  RBFFD_CK(cudaMemsetAsync(args.flags, 0, sizeof(unsigned int) * nblocks, ctx->stream));
  // shared memory for the staged windows of the gathered vectors
  // (kdev::win_init); one CTA per SM either way (1024 threads)
  RBFFD_CK(cudaFuncSetAttribute((const void *)k_fgmres<FNT>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, FG_WIN_BYTES));
  void *kargs[] = {(void *)&args};
  cudaError_t e = cudaLaunchCooperativeKernel((const void *)k_fgmres<FNT>, dim3(nblocks),
                                              dim3(FNT), kargs, FG_WIN_BYTES, ctx->stream);
  ctx->launches++;
  if (e != cudaSuccess) {
    set_error("cooperative launch of k_fgmres failed: %s", cudaGetErrorString(e));
    return RBFFD_ECUDA;
  }
  return RBFFD_OK;
}

}  // namespace rbffd
