// ops.cu -- row kernels of the outer iteration (paper Sec. 3) on the packed
// operators: packing (S3), momentum assembly (S4), divergence right-hand
// side (S6), pressure update + boundary pressure (S8/S9), velocity
// correction with the Delta partials (S8/S10), time-level rotation, the
// steady residual and a plain SpMV.
//
// Layout: every operator is an ELL array in column-major order [q][ldn]
// (entry j of row i at j*ldn + i), so a warp reading slot j of 32
// consecutive rows issues one coalesced 256-byte load; all operators share
// one int32 column array because they share the clouds.  Slot 0 of every
// row is the point itself (the clouds put it first).
#include "common.cuh"
#include "ops.cuh"

namespace rbffd {

constexpr int RT = 256;

// Kind of the momentum row of a point for velocity component c (0 = u,
// 1 = v), paper Sec. 3.1: the equation inside (ROW_EQ); an identity row with
// the boundary value where the component is prescribed (walls, inlets, the
// normal component on a symmetry line); a zero normal derivative n . grad
// at outlets and for the tangential component on a symmetry line.
enum { ROW_EQ = 0, ROW_ID = 1, ROW_NEU = 2 };

__device__ __forceinline__ int row_kind(int t, double nxi, double nyi, int c) {
  if (t == RBFFD_TAG_INTERIOR) return ROW_EQ;
  if (t == RBFFD_TAG_OUTFLOW) return ROW_NEU;
  if (t == RBFFD_TAG_SYMMETRY) return c == (fabs(nxi) > fabs(nyi) ? 0 : 1) ? ROW_ID : ROW_NEU;
  return ROW_ID;
}

__global__ void k_pack(int n, int q, int ldn, int pin, const int32_t *__restrict__ idx_rm,
                       const double *__restrict__ wx_rm, const double *__restrict__ wy_rm,
                       const double *__restrict__ wl_rm, const int8_t *__restrict__ tag,
                       const double *__restrict__ nx, const double *__restrict__ ny,
                       int32_t *__restrict__ col, double *__restrict__ Wx,
                       double *__restrict__ Wy, double *__restrict__ Wl,
                       double *__restrict__ Pp, double *__restrict__ pdinv) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ldn) return;
  if (i >= n) {  // padding rows: self-loops with zero weight, never read
    for (int j = 0; j < q; ++j) {
      int64_t e = (int64_t)j * ldn + i;
      col[e] = 0;
      Wx[e] = Wy[e] = Wl[e] = Pp[e] = 0.0;
    }
    pdinv[i] = 1.0;
    return;
  }
  const bool interior = tag[i] == 0;
  const double ni = nx[i], mi = ny[i];
  double diag = 0.0;
  for (int j = 0; j < q; ++j) {
    int64_t r = (int64_t)i * q + j, e = (int64_t)j * ldn + i;
    int c = idx_rm[r];
    double a = wx_rm[r], b = wy_rm[r], l = wl_rm[r];
    col[e] = c;
    Wx[e] = a;
    Wy[e] = b;
    Wl[e] = l;
    double pv;
    if (i == pin || tag[i] == RBFFD_TAG_OUTFLOW)
      pv = (c == i) ? 1.0 : 0.0;
    else if (interior)
      pv = l;
    else
      pv = ni * a + mi * b;
    Pp[e] = pv;
    if (c == i) diag += pv;
  }
  pdinv[i] = 1.0 / (diag == 0.0 ? 1.0 : diag);
}

// S4: momentum matrix and right-hand sides, Eqs. (u:tilde), (v:tilde):
//   rho a1/dt u~ + rho u^r Dx u~ + rho v^r Dy u~ - mu Lap u~
//       = -rho (a2 u^n + a3 u^{n-1}) / dt - (Dx p^r) + f_x
// at interior rows (f: the body force, e.g. the mean pressure gradient of
// a periodic flow); boundary rows by row_kind (identity with the boundary
// value, or n . grad with a zero right-hand side).  Am serves u~ (and v~
// too when Am2 is null: no symmetry rows); Am2, when given, is the v~
// matrix, equal to Am except on symmetry lines.  The initial guesses of the
// momentum solve are set to the current iterate.
__global__ void k_momentum(int n, int q, int ldn, const int32_t *__restrict__ col,
                           const double *__restrict__ Wx, const double *__restrict__ Wy,
                           const double *__restrict__ Wl, const int8_t *__restrict__ tag,
                           const double *__restrict__ u, const double *__restrict__ v,
                           const double *__restrict__ p, const double *__restrict__ un,
                           const double *__restrict__ vn, const double *__restrict__ unm1,
                           const double *__restrict__ vnm1, const double *__restrict__ ubc,
                           const double *__restrict__ vbc, const double *__restrict__ nx,
                           const double *__restrict__ ny, double rho, double mu, double dt,
                           double a1, double a2, double a3, double fx, double fy,
                           double *__restrict__ Am,
                           double *__restrict__ mdinv, double *__restrict__ Am2,
                           double *__restrict__ mdinv2, double *__restrict__ bu,
                           double *__restrict__ bv, double *__restrict__ ut,
                           double *__restrict__ vt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int t = tag[i];
  const double ui = u[i], vi = v[i];
  ut[i] = ui;
  vt[i] = vi;
  if (t != RBFFD_TAG_INTERIOR) {
    const double ni = nx[i], mi = ny[i];
    const int ku = row_kind(t, ni, mi, 0), kv = row_kind(t, ni, mi, 1);
    const bool neu = ku == ROW_NEU || kv == ROW_NEU;
    double gd = 0.0;
    for (int j = 0; j < q; ++j) {
      const int64_t e = (int64_t)j * ldn + i;
      const double id = (j == 0) ? 1.0 : 0.0;  // slot 0 is the point itself
      const double g = neu ? ni * Wx[e] + mi * Wy[e] : 0.0;
      if (j == 0) gd = g;
      Am[e] = ku == ROW_ID ? id : g;
      if (Am2) Am2[e] = kv == ROW_ID ? id : g;
    }
    const double gi = 1.0 / (gd == 0.0 ? 1.0 : gd);
    mdinv[i] = ku == ROW_ID ? 1.0 : gi;
    if (Am2) mdinv2[i] = kv == ROW_ID ? 1.0 : gi;
    bu[i] = ku == ROW_ID ? ubc[i] : 0.0;
    bv[i] = kv == ROW_ID ? vbc[i] : 0.0;
    return;
  }
  const double ru = rho * ui, rv = rho * vi, dd = rho * a1 / dt;
  double gx = 0.0, gy = 0.0, diag = 0.0;
#pragma unroll 4
  for (int j = 0; j < q; ++j) {
    int64_t e = (int64_t)j * ldn + i;
    const int c = col[e];
    const double a = Wx[e], b = Wy[e];
    const double pc = p[c];
    gx += a * pc;
    gy += b * pc;
    double val = ru * a + rv * b - mu * Wl[e];
    if (c == i) {
      val += dd;
      diag += val;
    }
    Am[e] = val;
    if (Am2) Am2[e] = val;
  }
  mdinv[i] = 1.0 / (diag == 0.0 ? 1.0 : diag);
  if (Am2) mdinv2[i] = mdinv[i];
  bu[i] = -rho * (a2 * un[i] + a3 * unm1[i]) / dt - gx + fx;
  bv[i] = -rho * (a2 * vn[i] + a3 * vnm1[i]) / dt - gy + fy;
}

// S6: right-hand side of Eq. (pressure poisson) at interior rows, zero at
// the Neumann rows and at the pinned row, with the block partials of the
// sum of the right-hand side and of the interior row count (for k_center).
__global__ void __launch_bounds__(RT) k_divergence(
    int n, int q, int ldn, const int32_t *__restrict__ col, const double *__restrict__ Wx,
    const double *__restrict__ Wy, const int8_t *__restrict__ tag,
    const double *__restrict__ ut, const double *__restrict__ vt, double coef,
    double *__restrict__ bp, double *__restrict__ pc, double *__restrict__ part) {
  __shared__ double sred[RT / 32];
  double sb = 0.0, sn = 0.0;
  for (int i = blockIdx.x * RT + threadIdx.x; i < n; i += gridDim.x * RT) {
    pc[i] = 0.0;  // initial guess of the p' solve
    if (tag[i] != 0) {
      bp[i] = 0.0;
      continue;
    }
    double dx = 0.0, dy = 0.0;
#pragma unroll 4
    for (int j = 0; j < q; ++j) {
      int64_t e = (int64_t)j * ldn + i;
      const int c = col[e];
      dx += Wx[e] * ut[c];
      dy += Wy[e] * vt[c];
    }
    const double b = coef * (dx + dy);
    bp[i] = b;
    sb += b;
    sn += 1.0;
  }
  sb = block_sum<RT>(sb, sred);
  sn = block_sum<RT>(sn, sred);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = sb;
    part[gridDim.x + blockIdx.x] = sn;
  }
}

// Pinned problems: take c0 e_I away from the interior rows of the p'
// right-hand side before the solve, c0 = the total shift c of the last p'
// solve (rec->cshift; 0 after a build).  This is the first, approximate
// part of the compatible shift c e_I (compat_shift removes the rest
// exactly, so c0 only has to be close): after one compatible correction
// the divergence left in u is about (dt / rho a1) c e_I, so the next
// right-hand side is about c e_I plus what changed.  Without it the
// right-hand side tends to c e_I near convergence, which is incompatible,
// and the pinned solve of it is dominated by the pin's large response
// (the p' solve's accuracy floor grows with |x|, and an FP32 inner solve
// cannot resolve it).  The plain interior mean is no substitute: psi
// weights the rows roughly by the area around each point.
__global__ void __launch_bounds__(RT) k_center(int n, const int8_t *__restrict__ tag,
                                               double *__restrict__ bp,
                                               const IterRecord *__restrict__ rec) {
  const double c0 = rec->cshift;
  for (int i = blockIdx.x * RT + threadIdx.x; i < n; i += gridDim.x * RT)
    if (tag[i] == RBFFD_TAG_INTERIOR) bp[i] -= c0;
}

// Compatible pressure correction (pinned problems: no outlet fixes the
// pressure level).  The p' equation with Neumann rows only is singular and
// solvable only for a right-hand side b with psi . b = 0 (psi: its left
// null vector); the divergence of u~ does not meet that exactly.  Its
// compatible solution is p' = M^{-1} (b - c e_I), e_I = 1 at interior rows,
// M = the stored p' matrix (pin row = identity), with c such that the
// pin's own Neumann row holds as well.  k_center has already taken c0 e_I
// away (b' = b - c0 e_I is what the solve saw), so by linearity
//   p' = M^{-1} b' - c1 z,   z = M^{-1} e_I (solved once per build),
//   c1 = (G_pin . M^{-1} b') / (G_pin . z),   G_pin = the pin's n . grad row,
// since G_pin . p' = 0 is the dropped equation; c = c0 + c1 is stored for
// the next solve.  Warp 0 of every block computes c1 in the same order
// (bit-identical in all blocks); z == null (an outlet fixes the level)
// gives c1 = 0.
__device__ __forceinline__ double compat_shift(int q, int ldn, int pin,
                                               const int32_t *__restrict__ col,
                                               const double *__restrict__ Wx,
                                               const double *__restrict__ Wy, double npx,
                                               double npy, const double *__restrict__ pc,
                                               const double *__restrict__ z, double *s_c) {
  if (threadIdx.x < 32) {
    double a = 0.0, b = 0.0;
    if (z) {
      for (int j = threadIdx.x; j < q; j += 32) {
        const int64_t e = (int64_t)j * ldn + pin;
        const double g = npx * Wx[e] + npy * Wy[e];
        const int c = col[e];
        a += g * pc[c];
        b += g * z[c];
      }
      a = warp_sum(a);
      b = warp_sum(b);
    }
    if (threadIdx.x == 0) *s_c = z ? a / b : 0.0;
  }
  __syncthreads();
  return *s_c;
}

// S8 (p += p' inside) fused with S9 (boundary pressure, Eq. normal momentum;
// outlets keep their prescribed pressure):
// for a boundary point i with G = nx Wx + ny Wy (row i),
//   sum_j G_ij p_j = N . [ -rho (a1 u~ + a2 u^n + a3 u^{n-1})/dt
//                          - rho (u~ . grad) u~ + mu Lap u~ ]_i,
// solved for p_i with every other p_j at its value after the interior
// update (p_j + p'_j inside, old p_j on the boundary).  Writes p_out and
// the compatible p' (compat_shift) to pcs; pc and z are only read.
__global__ void __launch_bounds__(RT) k_pressure(
    int n, int q, int ldn, const int32_t *__restrict__ col, const double *__restrict__ Wx,
    const double *__restrict__ Wy, const double *__restrict__ Wl,
    const int8_t *__restrict__ tag, const double *__restrict__ nx,
    const double *__restrict__ ny, const double *__restrict__ p,
    const double *__restrict__ pc, const double *__restrict__ z, int pin,
    const double *__restrict__ ut, const double *__restrict__ vt,
    const double *__restrict__ un, const double *__restrict__ vn,
    const double *__restrict__ unm1, const double *__restrict__ vnm1, double rho, double mu,
    double dt, double a1, double a2, double a3, double fx, double fy,
    double *__restrict__ p_out, double *__restrict__ pcs, IterRecord *__restrict__ rec) {
  __shared__ double s_c;
  const double cs = compat_shift(q, ldn, pin, col, Wx, Wy, z ? nx[pin] : 0.0,
                                 z ? ny[pin] : 0.0, pc, z, &s_c);
  // only this thread touches cshift in this kernel (k_center read it before)
  if (z && blockIdx.x == 0 && threadIdx.x == 0) rec->cshift += cs;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double pci = z ? pc[i] - cs * z[i] : pc[i];
  pcs[i] = pci;
  if (tag[i] == RBFFD_TAG_INTERIOR) {
    p_out[i] = p[i] + pci;
    return;
  }
  if (tag[i] == RBFFD_TAG_OUTFLOW) {
    p_out[i] = p[i];
    return;
  }
  const double ni = nx[i], mi = ny[i];
  double gxu = 0, gyu = 0, lu = 0, gxv = 0, gyv = 0, lv = 0, gii = 0, off = 0;
  for (int j = 0; j < q; ++j) {
    int64_t e = (int64_t)j * ldn + i;
    const int c = col[e];
    const double a = Wx[e], b = Wy[e], l = Wl[e];
    const double uc = ut[c], vc = vt[c];
    gxu += a * uc;
    gyu += b * uc;
    lu += l * uc;
    gxv += a * vc;
    gyv += b * vc;
    lv += l * vc;
    const double g = ni * a + mi * b;
    if (c == i) {
      gii += g;
    } else {
      const double pj = tag[c] == 0 ? p[c] + (z ? pc[c] - cs * z[c] : pc[c]) : p[c];
      off += g * pj;
    }
  }
  const double uti = ut[i], vti = vt[i];
  const double mx = -rho * (a1 * uti + a2 * un[i] + a3 * unm1[i]) / dt -
                    rho * (uti * gxu + vti * gyu) + mu * lu + fx;
  const double my = -rho * (a1 * vti + a2 * vn[i] + a3 * vnm1[i]) / dt -
                    rho * (uti * gxv + vti * gyv) + mu * lv + fy;
  p_out[i] = (ni * mx + mi * my - off) / gii;
}

// S8 velocity correction, Eqs. (u:correction), (v:correction), of every
// component that is not prescribed (row_kind != ROW_ID: interior, outlets,
// the tangential component on symmetry lines), with the block partials of
// sum|du| and sum|dv| for Delta (S10).  pcs: the compatible p' that
// k_pressure wrote; it is also copied into pc (the p' field of the step).
__global__ void __launch_bounds__(RT) k_correct(
    int n, int q, int ldn, const int32_t *__restrict__ col, const double *__restrict__ Wx,
    const double *__restrict__ Wy, const int8_t *__restrict__ tag,
    const double *__restrict__ nx, const double *__restrict__ ny,
    const double *__restrict__ pcs, double *__restrict__ pc, const double *__restrict__ ut,
    const double *__restrict__ vt, double c, double *__restrict__ u, double *__restrict__ v,
    const double *__restrict__ pnew, double *__restrict__ p, double *__restrict__ part) {
  __shared__ double sred[RT / 32];
  double su = 0.0, sv = 0.0;
  for (int i = blockIdx.x * RT + threadIdx.x; i < n; i += gridDim.x * RT) {
    // the pressure k_pressure wrote beside p becomes p (no pointer swap:
    // the buffers an outer iteration uses stay the same, so it can be
    // captured and replayed)
    p[i] = pnew[i];
    pc[i] = pcs[i];
    double unew = ut[i], vnew = vt[i];
    const int t = tag[i];
    if (t != RBFFD_TAG_DIRICHLET) {
      double gx = 0.0, gy = 0.0;
#pragma unroll 4
      for (int j = 0; j < q; ++j) {
        int64_t e = (int64_t)j * ldn + i;
        const double pj = pcs[col[e]];
        gx += Wx[e] * pj;
        gy += Wy[e] * pj;
      }
      bool cu = true, cv = true;
      if (t == RBFFD_TAG_SYMMETRY) {
        const double ni = nx[i], mi = ny[i];
        cu = row_kind(t, ni, mi, 0) != ROW_ID;
        cv = row_kind(t, ni, mi, 1) != ROW_ID;
      }
      if (cu) unew = unew - c * gx;
      if (cv) vnew = vnew - c * gy;
    }
    su += fabs(unew - u[i]);
    sv += fabs(vnew - v[i]);
    u[i] = unew;
    v[i] = vnew;
  }
  su = block_sum<RT>(su, sred);
  sv = block_sum<RT>(sv, sred);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = su;
    part[gridDim.x + blockIdx.x] = sv;
  }
}

// End of a time step: change partials (sum|u - u^n|, sum|v - v^n|), then
// u^{n-1} <- u^n, u^n <- u, row by row in place (the buffers keep their
// roles, so captured outer iterations stay valid across time steps).
__global__ void __launch_bounds__(RT) k_rotate(int n, const double *__restrict__ u,
                                               const double *__restrict__ v,
                                               double *__restrict__ un, double *__restrict__ vn,
                                               double *__restrict__ unm1,
                                               double *__restrict__ vnm1,
                                               double *__restrict__ part) {
  __shared__ double sred[RT / 32];
  double su = 0.0, sv = 0.0;
  for (int i = blockIdx.x * RT + threadIdx.x; i < n; i += gridDim.x * RT) {
    const double a = u[i], b = v[i], on = un[i], ovn = vn[i];
    su += fabs(a - on);
    sv += fabs(b - ovn);
    unm1[i] = on;
    vnm1[i] = ovn;
    un[i] = a;
    vn[i] = b;
  }
  su = block_sum<RT>(su, sred);
  sv = block_sum<RT>(sv, sred);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = su;
    part[gridDim.x + blockIdx.x] = sv;
  }
}

// Steady residual partials over interior rows (see rbffd_steady_residual):
// slots 0 |r|^2, 1 |rho (u.grad)u|^2, 2 |mu Lap u|^2, 3 |grad p|^2,
// 4 |div u|^2, 5 |grad u|^2, 6 |f|^2, 7 sum div u, 8 interior rows.
__global__ void __launch_bounds__(RT) k_resid(int n, int q, int ldn,
                                              const int32_t *__restrict__ col,
                                              const double *__restrict__ Wx,
                                              const double *__restrict__ Wy,
                                              const double *__restrict__ Wl,
                                              const int8_t *__restrict__ tag,
                                              const double *__restrict__ u,
                                              const double *__restrict__ v,
                                              const double *__restrict__ p, double rho,
                                              double mu, double fx, double fy,
                                              double *__restrict__ part) {
  __shared__ double sred[RT / 32];
  double acc[RESID_SLOTS] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int i = blockIdx.x * RT + threadIdx.x; i < n; i += gridDim.x * RT) {
    if (tag[i] != 0) continue;
    double gxu = 0, gyu = 0, lu = 0, gxv = 0, gyv = 0, lv = 0, gpx = 0, gpy = 0;
    for (int j = 0; j < q; ++j) {
      int64_t e = (int64_t)j * ldn + i;
      const int c = col[e];
      const double a = Wx[e], b = Wy[e], l = Wl[e];
      const double uc = u[c], vc = v[c], pcv = p[c];
      gxu += a * uc; gyu += b * uc; lu += l * uc;
      gxv += a * vc; gyv += b * vc; lv += l * vc;
      gpx += a * pcv; gpy += b * pcv;
    }
    const double ui = u[i], vi = v[i];
    const double au = rho * (ui * gxu + vi * gyu), av = rho * (ui * gxv + vi * gyv);
    const double du = mu * lu, dv = mu * lv;
    const double ru = au - du + gpx - fx, rv = av - dv + gpy - fy;
    acc[0] += ru * ru + rv * rv;
    acc[6] += fx * fx + fy * fy;
    acc[1] += au * au + av * av;
    acc[2] += du * du + dv * dv;
    acc[3] += gpx * gpx + gpy * gpy;
    const double dc = gxu + gyv;
    acc[4] += dc * dc;
    acc[7] += dc;
    acc[8] += 1.0;
    acc[5] += gxu * gxu + gyu * gyu + gxv * gxv + gyv * gyv;
  }
#pragma unroll
  for (int s = 0; s < RESID_SLOTS; ++s) {
    double t = block_sum<RT>(acc[s], sred);
    if (threadIdx.x == 0) part[s * gridDim.x + blockIdx.x] = t;
  }
}

// Fixed-order sums of the partials into the iteration record.
// mode 0: delta = (S0 + S1) / n   mode 1: change = (S0 + S1) / n
// mode 2: steady residual from the sums of k_resid; compat (pinned
// problems, whose compatible p' leaves continuity satisfied up to a
// constant lambda = mean interior divergence): R_c of d - lambda, with
// |d - lambda|^2 = S4 - S7^2 / S8.
__global__ void k_finalize(const double *__restrict__ part, int nb, int n, int mode,
                           IterRecord *rec, int compat = 0) {
  if (threadIdx.x >= 32) return;
  if (mode == 0 || mode == 1) {
    double a = warp_sum_array(part, nb);
    double b = warp_sum_array(part + nb, nb);
    if (threadIdx.x == 0) {
      double d = a / n + b / n;
      if (mode == 0)
        rec->delta = d;
      else
        rec->change = d;
    }
  } else {
    double s[RESID_SLOTS];
    for (int k = 0; k < RESID_SLOTS; ++k) s[k] = warp_sum_array(part + k * nb, nb);
    if (threadIdx.x == 0) {
      const double lambda = s[8] > 0 ? s[7] / s[8] : 0.0;
      double nc = s[4];
      if (compat && s[8] > 0) {
        nc = s[4] - s[7] * (s[7] / s[8]);
        if (nc < 0.0) nc = 0.0;
      }
      double dm = sqrt(s[1]) + sqrt(s[2]) + sqrt(s[3]) + sqrt(s[6]);
      double dc = sqrt(s[5]);
      double rm = dm > 0 ? sqrt(s[0]) / dm : sqrt(s[0]);
      double rc = dc > 0 ? sqrt(nc) / dc : sqrt(nc);
      rec->resid[0] = rm;
      rec->resid[1] = rc;
      rec->resid[2] = rm > rc ? rm : rc;
      rec->resid[3] = lambda;
    }
  }
}

// FP64 array -> the inner arithmetic of the mixed-precision solve: FP32
// (round to nearest) or float-float (hi = rn(v), lo = rn(v - hi)).
__global__ void k_to_inner(int64_t m, const double *__restrict__ src, void *__restrict__ dst,
                           int ff) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const double v = src[i];
  const float h = __double2float_rn(v);
  if (ff)
    reinterpret_cast<float2 *>(dst)[i] = make_float2(h, __double2float_rn(v - (double)h));
  else
    reinterpret_cast<float *>(dst)[i] = h;
}

__global__ void k_spmv(int n, int q, int ldn, const int32_t *__restrict__ col,
                       const double *__restrict__ val, const double *__restrict__ x,
                       double *__restrict__ y) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
#pragma unroll 4
  for (int j = 0; j < q; ++j) {
    int64_t e = (int64_t)j * ldn + i;
    s += val[e] * x[col[e]];
  }
  y[i] = s;
}

// Courant helper: y = C x with C = rho (u Dx + v Dy) - mu Lap at interior
// rows (zero elsewhere), plus the block partials of sum y^2.
__global__ void __launch_bounds__(RT) k_cd_apply(
    int n, int q, int ldn, const int32_t *__restrict__ col, const double *__restrict__ Wx,
    const double *__restrict__ Wy, const double *__restrict__ Wl, const int8_t *__restrict__ tag,
    const double *__restrict__ u, const double *__restrict__ v, double rho, double mu,
    const double *__restrict__ x, double *__restrict__ y, double *__restrict__ part) {
  __shared__ double sred[RT / 32];
  double acc = 0.0;
  for (int i = blockIdx.x * RT + threadIdx.x; i < n; i += gridDim.x * RT) {
    double yi = 0.0;
    if (tag[i] == 0) {
      double gx = 0.0, gy = 0.0, gl = 0.0;
      for (int j = 0; j < q; ++j) {
        const int64_t e = (int64_t)j * ldn + i;
        const double xc = x[col[e]];
        gx += Wx[e] * xc;
        gy += Wy[e] * xc;
        gl += Wl[e] * xc;
      }
      yi = rho * (u[i] * gx + v[i] * gy) - mu * gl;
    }
    y[i] = yi;
    acc += yi * yi;
  }
  acc = block_sum<RT>(acc, sred);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// x = y / |y| (every block sums the partials in the same order); block 0
// adds log|y| to *logacc when `count` is set.
__global__ void __launch_bounds__(RT) k_cd_scale(int n, const double *__restrict__ y,
                                                 const double *__restrict__ part, int nb,
                                                 double *__restrict__ x, double *logacc,
                                                 int count) {
  __shared__ double s_norm;
  if (threadIdx.x < 32) {
    const double t = warp_sum_array(part, nb);
    if (threadIdx.x == 0) s_norm = sqrt(t);
  }
  __syncthreads();
  const double nrm = s_norm;
  if (blockIdx.x == 0 && threadIdx.x == 0 && count && nrm > 0.0) *logacc += log(nrm);
  const double r = nrm > 0.0 ? 1.0 / nrm : 0.0;
  for (int i = blockIdx.x * RT + threadIdx.x; i < n; i += gridDim.x * RT) x[i] = y[i] * r;
}

__global__ void k_cd_start(int n, double *__restrict__ x, double *logacc) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) *logacc = 0.0;
  if (i < n) x[i] = 1.0 + 0.5 * (double)((i * 7919) % 13) / 13.0;
}

// Right-hand side e_I (1 at interior rows, 0 elsewhere) and a zero initial
// guess, for the once-per-build solve z = M^{-1} e_I of the compatible p'.
__global__ void k_interior_ones(int n, const int8_t *__restrict__ tag, double *__restrict__ b,
                                double *__restrict__ x) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  b[i] = tag[i] == RBFFD_TAG_INTERIOR ? 1.0 : 0.0;
  x[i] = 0.0;
}

// ------------------------------------------------------------------ host

static inline int grid_of(int n) { return (n + RT - 1) / RT; }

int ops_pack(rbffd_problem *P) {
  k_pack<<<(P->ldn + RT - 1) / RT, RT, 0, P->ctx->stream>>>(
      P->n, P->q, P->ldn, P->pin, P->idx_rm, P->wx_rm, P->wy_rm, P->wl_rm, P->tag, P->nx, P->ny,
      P->col, P->Wx, P->Wy, P->Wl, P->Pp, P->p_dinv);
  return after_launch(P->ctx, "k_pack");
}

int ops_momentum(rbffd_problem *P, const rbffd_step_params *sp) {
  k_momentum<<<grid_of(P->n), RT, 0, P->ctx->stream>>>(
      P->n, P->q, P->ldn, P->col, P->Wx, P->Wy, P->Wl, P->tag, P->u, P->v, P->p, P->un, P->vn,
      P->unm1, P->vnm1, P->ubc, P->vbc, P->nx, P->ny, P->rho, P->mu, sp->dt, sp->alpha[0],
      sp->alpha[1], sp->alpha[2], P->force[0], P->force[1], P->Am, P->m_dinv,
      P->has_sym ? P->Am2 : nullptr,
      P->has_sym ? P->m_dinv2 : nullptr, P->bu, P->bv, P->ut, P->vt);
  return after_launch(P->ctx, "k_momentum");
}

int ops_divergence(rbffd_problem *P, const rbffd_step_params *sp) {
  double coef = P->rho * sp->alpha[0] / sp->dt;
  k_divergence<<<P->rblocks, RT, 0, P->ctx->stream>>>(P->n, P->q, P->ldn, P->col, P->Wx,
                                                      P->Wy, P->tag, P->ut, P->vt, coef, P->bp,
                                                      P->pc, P->rpart);
  RBFFD_TRY(after_launch(P->ctx, "k_divergence"));
  if (!P->compat) return RBFFD_OK;
  k_center<<<P->rblocks, RT, 0, P->ctx->stream>>>(P->n, P->tag, P->bp, P->rec);
  return after_launch(P->ctx, "k_center");
}

int ops_pressure(rbffd_problem *P, const rbffd_step_params *sp) {
  k_pressure<<<grid_of(P->n), RT, 0, P->ctx->stream>>>(
      P->n, P->q, P->ldn, P->col, P->Wx, P->Wy, P->Wl, P->tag, P->nx, P->ny, P->p, P->pc,
      P->compat ? P->zc : nullptr, P->pin < 0 ? 0 : P->pin, P->ut, P->vt, P->un, P->vn,
      P->unm1, P->vnm1, P->rho, P->mu, sp->dt, sp->alpha[0], sp->alpha[1], sp->alpha[2],
      P->force[0], P->force[1], P->p2, P->pcs, P->rec);
  return after_launch(P->ctx, "k_pressure");
}

int ops_correct(rbffd_problem *P, const rbffd_step_params *sp) {
  double c = sp->dt / (P->rho * sp->alpha[0]);
  k_correct<<<P->rblocks, RT, 0, P->ctx->stream>>>(P->n, P->q, P->ldn, P->col, P->Wx, P->Wy,
                                                   P->tag, P->nx, P->ny, P->pcs, P->pc, P->ut,
                                                   P->vt, c, P->u, P->v, P->p2, P->p, P->rpart);
  RBFFD_TRY(after_launch(P->ctx, "k_correct"));
  k_finalize<<<1, 32, 0, P->ctx->stream>>>(P->rpart, P->rblocks, P->n, 0, P->rec);
  return after_launch(P->ctx, "k_finalize");
}

int ops_rotate(rbffd_problem *P) {
  k_rotate<<<P->rblocks, RT, 0, P->ctx->stream>>>(P->n, P->u, P->v, P->un, P->vn, P->unm1,
                                                  P->vnm1, P->rpart);
  RBFFD_TRY(after_launch(P->ctx, "k_rotate"));
  k_finalize<<<1, 32, 0, P->ctx->stream>>>(P->rpart, P->rblocks, P->n, 1, P->rec);
  return after_launch(P->ctx, "k_finalize");
}

int ops_resid(rbffd_problem *P) {
  k_resid<<<P->rblocks, RT, 0, P->ctx->stream>>>(P->n, P->q, P->ldn, P->col, P->Wx, P->Wy,
                                                 P->Wl, P->tag, P->u, P->v, P->p, P->rho, P->mu,
                                                 P->force[0], P->force[1], P->rpart);
  RBFFD_TRY(after_launch(P->ctx, "k_resid"));
  k_finalize<<<1, 32, 0, P->ctx->stream>>>(P->rpart, P->rblocks, P->n, 2, P->rec,
                                            P->compat ? 1 : 0);
  return after_launch(P->ctx, "k_finalize");
}

// Power iteration of the Courant helper (see k_cd_apply): iters steps from
// the fixed start, log|C x_k| summed over the second half into *logacc.
int ops_courant(rbffd_problem *P, int iters, double *logacc) {
  cudaStream_t st = P->ctx->stream;
  double *x = P->kv[0].r, *y = P->kv[0].p;  // Krylov workspace, free between solves
  double *part = P->rpart;
  k_cd_start<<<grid_of(P->n), RT, 0, st>>>(P->n, x, logacc);
  RBFFD_TRY(after_launch(P->ctx, "k_cd_start"));
  for (int k = 0; k < iters; ++k) {
    k_cd_apply<<<P->rblocks, RT, 0, st>>>(P->n, P->q, P->ldn, P->col, P->Wx, P->Wy, P->Wl,
                                          P->tag, P->u, P->v, P->rho, P->mu, x, y, part);
    RBFFD_TRY(after_launch(P->ctx, "k_cd_apply"));
    k_cd_scale<<<P->rblocks, RT, 0, st>>>(P->n, y, part, P->rblocks, x, logacc,
                                          k >= iters / 2);
    RBFFD_TRY(after_launch(P->ctx, "k_cd_scale"));
  }
  return RBFFD_OK;
}

int ops_interior_ones(rbffd_problem *P, double *b, double *x) {
  k_interior_ones<<<grid_of(P->n), RT, 0, P->ctx->stream>>>(P->n, P->tag, b, x);
  return after_launch(P->ctx, "k_interior_ones");
}

int ops_spmv(rbffd_problem *P, const double *val, const double *x, double *y) {
  k_spmv<<<grid_of(P->n), RT, 0, P->ctx->stream>>>(P->n, P->q, P->ldn, P->col, val, x, y);
  return after_launch(P->ctx, "k_spmv");
}

int ops_to_inner(rbffd_problem *P, const double *src, void *dst, int64_t m) {
  int ff = P->inner == INNER_FF;
  k_to_inner<<<(unsigned)((m + RT - 1) / RT), RT, 0, P->ctx->stream>>>(m, src, dst, ff);
  return after_launch(P->ctx, "k_to_inner");
}

int ops_reduce_blocks(rbffd_ctx *ctx, int n) {
  int b = grid_of(n);
  int cap = ctx->num_sms * 4;
  return b < cap ? b : cap;
}

}  // namespace rbffd
