"""Seeded synthetic point clouds and boundary data for the flow problems.

This module only makes INPUTS: coordinates, boundary tags, outward normals,
prescribed boundary velocities and the index of the point where the
pressure correction is pinned.  It holds none of the method's arithmetic
(no stencils, weights, operators or solver steps), so both the CUDA path and
the CPU oracle can be fed from it without sharing any of the method.

Workloads (all synthetic; the paper's own Gmsh point sets are not public
data here, so seeded clouds with the same structure stand in for them):

* ``kovasznay(n_side)``: Kovasznay flow, Re = 40, on [-0.5, 1.5]^2;
  an n_side x n_side Cartesian lattice whose interior points are jittered
  uniformly by +-0.25 h (h = 2/(n_side-1)); boundary points stay on the
  edges.  Velocity is prescribed from the closed form on every boundary
  point.
* ``cavity(n_side)``: lid-driven cavity on the unit square, lid u = 1,
  Re = 1000.  Per axis the lattice is mapped by x = s - sin(2 pi s)/(4 pi),
  which halves the spacing at the walls (2x boundary-layer clustering);
  interior points are jittered by +-0.25 of the local spacing.  Corner
  points belong to the side walls (u = v = 0); the lid velocity is applied
  on the open top edge only.

* ``channel(n_x, n_y)``: plane Poiseuille flow in [0, L] x [0, H] at
  Re = U H / nu: parabolic inlet u = 4 U y (H - y) / H^2 at x = 0, no-slip
  walls, a fixed-pressure outlet (p = 0) at x = L.  With ``symmetry=True``
  only the lower half [0, L] x [0, H/2] is meshed and y = H/2 is a
  symmetry line.  Closed form: u as at the inlet, v = 0,
  p = 8 mu U (L - x) / H^2.  Interior points are jittered by +-0.25 h.

* ``cylinder(n_target)``: flow past a circular cylinder (D = 1 at the
  origin) in the box [-5, 15] x [-5, 5], Re = U D / nu = 100: inlet
  u = 1, v = 0 at x = -5; symmetry lines at y = +-5; a fixed-pressure
  outlet (p = 0, zero normal velocity gradient) at x = 15; no-slip
  cylinder.  Spacing graded with the distance d from the centre,
  h(d) = min(h_max, h_0 + g (d - 0.5)), h_0 = 0.02, h_max = 0.2, with g
  found by bisection so that the point count is within 2 % of n_target.
  Points lie on concentric rings r_{k+1} = r_k + h(r_k) (one ring = the
  cylinder surface), each ring with round(2 pi r / h) points at a seeded
  random phase and a +-0.15 h seeded jitter, clipped to the box half a
  spacing from its edges; the box edges carry points spaced by h(d).
  Points are numbered along a Morton curve (stencil neighbours stay close
  in memory).

* ``periodic_channel(n_x, n_y)``: plane Poiseuille flow in a channel that
  is periodic in x (period L, points at x = i L / n_x, no seam points)
  between no-slip walls at y = 0 and y = H, driven by a body force f (the
  paper's mean pressure gradient of periodic flows): u = f y (H - y) /
  (2 mu), v = 0, p constant.  Interior points jittered by +-0.25 h.
* ``couette(h)``: steady cylindrical Couette flow between r1 = 0.5 (turning
  at omega = 2) and r2 = 1 (at rest), Re = rho r1 omega (2 r1) / mu = 100.
  Concentric rings at a radial spacing of about h, each with
  round(2 pi r / h) points at a seeded phase; interior rings jittered by
  +-0.25 h.  Closed form v_theta(r) = A (r2 / r - r / r2),
  A = omega r1^2 r2 / (r2^2 - r1^2), and p(r) from dp/dr = rho v_theta^2 / r.
* ``decaying(n_side, level)``: the decaying flow in the unit square from
  the stream function sin^2(pi x) sin^2(pi y) / pi, no-slip walls,
  Re = 100.  The clouds of levels 0, 1, 2 are nested: the level-l cloud is
  the points of the finest (n_side^2) jittered lattice whose lattice
  indices are multiples of 2^(2 - l), so coarser clouds are subsets of
  finer ones and fields compare at shared points without interpolation.

Point numbering is lattice row-major (index = j * n_side + i), which keeps
stencil neighbours close in memory.  ``pin`` is the boundary point nearest
the middle of the bottom edge: the pressure correction has only Neumann
boundary rows, and the row of that point fixes its free constant.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

TAG_INTERIOR = 0
TAG_DIRICHLET = 1  # wall / inlet: velocity prescribed, p' homogeneous Neumann
TAG_OUTFLOW = 2    # fixed-pressure outlet: p held, p' = 0, zero normal velocity gradient
TAG_SYMMETRY = 3   # symmetry line: normal velocity prescribed, tangential d/dn = 0


@dataclasses.dataclass
class FlowProblem:
    """Inputs of one flow problem (host arrays, FP64 unless noted)."""

    name: str
    x: np.ndarray
    y: np.ndarray
    tag: np.ndarray  # int8
    nx: np.ndarray
    ny: np.ndarray
    ubc: np.ndarray
    vbc: np.ndarray
    pin: int
    rho: float
    mu: float
    degree: int
    q: int
    dt: float
    exact: dict | None = None  # closed-form fields where one exists
    initial: dict | None = None  # initial fields other than the rest state, if any
    period: tuple = (0.0, 0.0)   # periods of x and y (0: bounded axis)
    force: tuple = (0.0, 0.0)    # body force per unit volume (mean pressure gradient)

    @property
    def n(self) -> int:
        return int(self.x.shape[0])


def num_monomials(degree: int) -> int:
    """m = C(k+2, k) appended monomials in two dimensions."""
    return (degree + 1) * (degree + 2) // 2


def kovasznay_exact(x, y, re=40.0):
    """Closed-form Kovasznay velocity and pressure (pressure up to a constant)."""
    lam = re / 2.0 - math.sqrt(re * re / 4.0 + 4.0 * math.pi * math.pi)
    u = 1.0 - np.exp(lam * x) * np.cos(2.0 * math.pi * y)
    v = lam / (2.0 * math.pi) * np.exp(lam * x) * np.sin(2.0 * math.pi * y)
    p = 0.5 * (1.0 - np.exp(2.0 * lam * x))
    return u, v, p


def _lattice(n_side, lo, hi, mapping=None):
    s = np.linspace(0.0, 1.0, n_side)
    if mapping is None:
        t = s
        dt_ds = np.ones_like(s)
    else:
        t, dt_ds = mapping(s)
    coord = lo + (hi - lo) * t
    spacing = (hi - lo) * dt_ds / (n_side - 1)
    return coord, spacing


def _box_cloud(n_side, lo, hi, seed, mapping=None, jitter=0.25):
    """Row-major lattice on [lo, hi]^2 with interior jitter; returns x, y,
    boundary mask, outward normals."""
    c, h = _lattice(n_side, lo, hi, mapping)
    ii, jj = np.meshgrid(np.arange(n_side), np.arange(n_side), indexing="xy")
    ii = ii.ravel()
    jj = jj.ravel()
    x = c[ii].astype(np.float64)
    y = c[jj].astype(np.float64)
    bnd = (ii == 0) | (ii == n_side - 1) | (jj == 0) | (jj == n_side - 1)
    rng = np.random.Generator(np.random.PCG64(seed))
    jx = rng.uniform(-jitter, jitter, size=x.shape) * h[ii]
    jy = rng.uniform(-jitter, jitter, size=y.shape) * h[jj]
    x = np.where(bnd, x, x + jx)
    y = np.where(bnd, y, y + jy)
    nx = np.zeros_like(x)
    ny = np.zeros_like(y)
    nx[ii == 0] = -1.0
    nx[ii == n_side - 1] = 1.0
    ny[jj == 0] = -1.0
    ny[jj == n_side - 1] = 1.0
    norm = np.hypot(nx, ny)
    nz = norm > 0
    nx[nz] /= norm[nz]
    ny[nz] /= norm[nz]
    return x, y, bnd, nx, ny, ii, jj


def _pin_index(x, y, bnd, cx, cy):
    """The boundary point nearest (cx, cy), lowest index on ties."""
    d2 = (x - cx) ** 2 + (y - cy) ** 2
    d2 = np.where(bnd, d2, np.inf)
    return int(np.argmin(d2))


def kovasznay(n_side=50, seed=1, degree=3, q=20, re=40.0, dt=0.05):
    x, y, bnd, nx, ny, _, _ = _box_cloud(n_side, -0.5, 1.5, seed)
    ue, ve, pe = kovasznay_exact(x, y, re)
    tag = np.where(bnd, TAG_DIRICHLET, TAG_INTERIOR).astype(np.int8)
    ubc = np.where(bnd, ue, 0.0)
    vbc = np.where(bnd, ve, 0.0)
    pin = _pin_index(x, y, bnd, 0.5, -0.5)
    return FlowProblem(
        name=f"kovasznay{n_side}", x=x, y=y, tag=tag, nx=nx, ny=ny, ubc=ubc, vbc=vbc,
        pin=pin, rho=1.0, mu=1.0 / re, degree=degree, q=q, dt=dt,
        exact={"u": ue, "v": ve, "p": pe})


def _cluster2x(s):
    t = s - np.sin(2.0 * math.pi * s) / (4.0 * math.pi)
    dt_ds = 1.0 - 0.5 * np.cos(2.0 * math.pi * s)
    return t, dt_ds


def cavity(n_side=200, seed=2, degree=4, q=30, re=1000.0, dt=None, lid=1.0):
    x, y, bnd, nx, ny, ii, jj = _box_cloud(n_side, 0.0, 1.0, seed, mapping=_cluster2x)
    tag = np.where(bnd, TAG_DIRICHLET, TAG_INTERIOR).astype(np.int8)
    top_open = (jj == n_side - 1) & (ii > 0) & (ii < n_side - 1)
    ubc = np.where(top_open, lid, 0.0)
    vbc = np.zeros_like(x)
    pin = _pin_index(x, y, bnd, 0.5, 0.0)
    if dt is None:
        # Courant ~10 on the mean lattice spacing at unit velocity
        dt = 10.0 * (1.0 / (n_side - 1)) / lid
    return FlowProblem(
        name=f"cavity{n_side}", x=x, y=y, tag=tag, nx=nx, ny=ny, ubc=ubc, vbc=vbc,
        pin=pin, rho=1.0, mu=lid * 1.0 / re, degree=degree, q=q, dt=float(dt))


def _rect_cloud(n_x, n_y, x0, x1, y0, y1, seed, jitter=0.25):
    """Row-major n_x x n_y lattice on [x0, x1] x [y0, y1] with interior
    jitter; returns x, y, lattice indices."""
    cx = np.linspace(x0, x1, n_x)
    cy = np.linspace(y0, y1, n_y)
    hx, hy = (x1 - x0) / (n_x - 1), (y1 - y0) / (n_y - 1)
    ii, jj = np.meshgrid(np.arange(n_x), np.arange(n_y), indexing="xy")
    ii, jj = ii.ravel(), jj.ravel()
    x, y = cx[ii].astype(np.float64), cy[jj].astype(np.float64)
    bnd = (ii == 0) | (ii == n_x - 1) | (jj == 0) | (jj == n_y - 1)
    rng = np.random.Generator(np.random.PCG64(seed))
    jx = rng.uniform(-jitter, jitter, size=x.shape) * hx
    jy = rng.uniform(-jitter, jitter, size=y.shape) * hy
    return np.where(bnd, x, x + jx), np.where(bnd, y, y + jy), ii, jj


def poiseuille_exact(x, y, mu, length=3.0, height=1.0, u_max=1.0):
    """Plane Poiseuille flow with p = 0 at x = length."""
    u = 4.0 * u_max * y * (height - y) / height**2
    return u, np.zeros_like(x), 8.0 * mu * u_max * (length - x) / height**2


def channel(n_x=31, n_y=11, length=3.0, height=1.0, seed=6, degree=3, q=20, re=10.0, dt=0.1,
            symmetry=False):
    """Poiseuille channel with an inlet, walls, an outlet and optionally a
    symmetry line (see the module docstring).  The outlet and the symmetry
    line start at rest; the pressure correction needs no pin (the outlet
    fixes its level)."""
    top = height / 2.0 if symmetry else height
    x, y, ii, jj = _rect_cloud(n_x, n_y, 0.0, length, 0.0, top, seed)
    mu = 1.0 / re
    ue, ve, pe = poiseuille_exact(x, y, mu, length, height)
    n = x.shape[0]
    tag = np.full(n, TAG_INTERIOR, np.int8)
    nx, ny = np.zeros(n), np.zeros(n)
    ubc, vbc = np.zeros(n), np.zeros(n)
    inlet, outlet = ii == 0, ii == n_x - 1
    bottom, upper = jj == 0, jj == n_y - 1
    # walls (and wall corners) first; the inlet edge keeps its own normal
    wall_top = upper & (not symmetry)
    tag[bottom | wall_top] = TAG_DIRICHLET
    ny[bottom] = -1.0
    ny[wall_top] = 1.0
    if symmetry:
        sym = upper & ~inlet & ~outlet
        tag[sym] = TAG_SYMMETRY
        ny[sym] = 1.0
    out = outlet & ~bottom & ~wall_top
    tag[out] = TAG_OUTFLOW
    nx[out], ny[out] = 1.0, 0.0
    tag[inlet] = TAG_DIRICHLET
    nx[inlet], ny[inlet] = -1.0, 0.0
    ubc[inlet] = ue[inlet]
    return FlowProblem(
        name=f"channel{n_x}x{n_y}{'s' if symmetry else ''}", x=x, y=y, tag=tag, nx=nx, ny=ny,
        ubc=ubc, vbc=vbc, pin=-1, rho=1.0, mu=mu, degree=degree, q=q, dt=dt,
        exact={"u": ue, "v": ve, "p": pe})


def _graded_spacing(d, g, h0, hmax):
    return np.minimum(hmax, h0 + g * np.maximum(d - 0.5, 0.0))


def _edge_points(a, b, fixed, axis, g, h0, hmax):
    """Points along one box edge from a to b (inclusive ends) spaced by the
    graded spacing at each point; axis 0: the edge runs along x at y=fixed."""
    pts = [a]
    t = a
    while True:
        x, y = (t, fixed) if axis == 0 else (fixed, t)
        t = t + float(_graded_spacing(math.hypot(x, y), g, h0, hmax))
        if t > b - 0.5 * float(_graded_spacing(math.hypot(*((b, fixed) if axis == 0 else (fixed, b))), g, h0, hmax)):
            break
        pts.append(t)
    pts.append(b)
    return np.asarray(pts)


def _cylinder_cloud(g, seed, h0, hmax, box):
    x0, x1, y0, y1 = box
    rng = np.random.Generator(np.random.PCG64(seed))
    rmax = math.hypot(max(-x0, x1), max(-y0, y1))
    xs, ys, ts, nxs, nys = [], [], [], [], []
    r = 0.5
    ring = 0
    while r < rmax:
        h = float(_graded_spacing(r, g, h0, hmax))
        cnt = max(8, int(round(2.0 * math.pi * r / h)))
        th = 2.0 * math.pi * (np.arange(cnt) + rng.uniform()) / cnt
        if ring == 0:  # the cylinder surface: no jitter, no-slip
            x, y = r * np.cos(th), r * np.sin(th)
            xs.append(x); ys.append(y)
            ts.append(np.full(cnt, TAG_DIRICHLET, np.int8))
            nxs.append(-np.cos(th)); nys.append(-np.sin(th))  # out of the fluid
        else:
            rr = r + rng.uniform(-0.15, 0.15, cnt) * h
            tt = th + rng.uniform(-0.15, 0.15, cnt) * h / r
            x, y = rr * np.cos(tt), rr * np.sin(tt)
            m = ((x > x0 + 0.5 * h) & (x < x1 - 0.5 * h) & (y > y0 + 0.5 * h) &
                 (y < y1 - 0.5 * h))
            xs.append(x[m]); ys.append(y[m])
            ts.append(np.full(int(m.sum()), TAG_INTERIOR, np.int8))
            nxs.append(np.zeros(int(m.sum()))); nys.append(np.zeros(int(m.sum())))
        r = r + h
        ring += 1
    # box edges: inlet (with its corners), outlet, the two symmetry lines
    yi = _edge_points(y0, y1, x0, 1, g, h0, hmax)
    xs.append(np.full(yi.shape, x0)); ys.append(yi)
    ts.append(np.full(yi.shape, TAG_DIRICHLET, np.int8))
    nxs.append(np.full(yi.shape, -1.0)); nys.append(np.zeros(yi.shape))
    yo = _edge_points(y0, y1, x1, 1, g, h0, hmax)
    xs.append(np.full(yo.shape, x1)); ys.append(yo)
    ts.append(np.full(yo.shape, TAG_OUTFLOW, np.int8))
    nxs.append(np.full(yo.shape, 1.0)); nys.append(np.zeros(yo.shape))
    for yline, nyv in ((y0, -1.0), (y1, 1.0)):
        xe = _edge_points(x0, x1, yline, 0, g, h0, hmax)[1:-1]
        xs.append(xe); ys.append(np.full(xe.shape, yline))
        ts.append(np.full(xe.shape, TAG_SYMMETRY, np.int8))
        nxs.append(np.zeros(xe.shape)); nys.append(np.full(xe.shape, nyv))
    return (np.concatenate(xs), np.concatenate(ys), np.concatenate(ts), np.concatenate(nxs),
            np.concatenate(nys))


def _morton_order(x, y):
    """Permutation sorting points along a Morton (Z-order) curve."""
    def spread(v):
        v = v.astype(np.uint64)
        v = (v | (v << np.uint64(16))) & np.uint64(0x0000FFFF0000FFFF)
        v = (v | (v << np.uint64(8))) & np.uint64(0x00FF00FF00FF00FF)
        v = (v | (v << np.uint64(4))) & np.uint64(0x0F0F0F0F0F0F0F0F)
        v = (v | (v << np.uint64(2))) & np.uint64(0x3333333333333333)
        v = (v | (v << np.uint64(1))) & np.uint64(0x5555555555555555)
        return v
    qx = ((x - x.min()) / max(np.ptp(x), 1e-300) * 65535).astype(np.uint64)
    qy = ((y - y.min()) / max(np.ptp(y), 1e-300) * 65535).astype(np.uint64)
    return np.argsort(spread(qx) | (spread(qy) << np.uint64(1)), kind="stable")


def cylinder(n_target=150_000, seed=3, degree=3, q=20, re=100.0, dt=0.2, h0=0.02, hmax=0.2,
             box=(-5.0, 15.0, -5.0, 5.0)):
    """Flow past a cylinder (see the module docstring).  ``initial`` holds the
    paper's start, a uniform stream u = 1 away from the cylinder wall (the
    library itself starts from rest; callers set these fields)."""
    lo, hi = 1e-4, 1.0
    best = None
    for _ in range(60):  # bisection on g: fewer points as g grows
        g = math.sqrt(lo * hi)
        cl = _cylinder_cloud(g, seed, h0, hmax, box)
        n = cl[0].shape[0]
        best = cl
        if abs(n - n_target) <= 0.02 * n_target:
            break
        if n > n_target:
            lo = g
        else:
            hi = g
    x, y, tag, nx, ny = best
    if abs(x.shape[0] - n_target) > 0.02 * n_target:
        raise ValueError(f"cylinder: no grading reaches {n_target} points with h0={h0}, "
                         f"hmax={hmax}")
    order = _morton_order(x, y)
    x, y, tag, nx, ny = x[order], y[order], tag[order], nx[order], ny[order]
    ubc = np.where(tag == TAG_DIRICHLET, 1.0, 0.0)
    ubc[(tag == TAG_DIRICHLET) & (np.hypot(x, y) < 0.75)] = 0.0  # the cylinder
    vbc = np.zeros_like(x)
    u0 = np.where(tag == TAG_DIRICHLET, ubc, 1.0)
    init = {"u": u0, "un": u0, "unm1": u0}
    return FlowProblem(
        name=f"cylinder{x.shape[0]}", x=x, y=y, tag=tag.astype(np.int8), nx=nx, ny=ny,
        ubc=ubc, vbc=vbc, pin=-1, rho=1.0, mu=1.0 / re, degree=degree, q=q, dt=dt,
        initial=init)


def periodic_channel(n_x=24, n_y=13, length=1.0, height=1.0, seed=9, degree=3, q=20, re=10.0,
                     dt=0.1):
    """Force-driven channel, periodic in x (see the module docstring); the
    force makes the centre-line velocity 1, so Re = H / nu."""
    hx, hy = length / n_x, height / (n_y - 1)
    ii, jj = np.meshgrid(np.arange(n_x), np.arange(n_y), indexing="xy")
    ii, jj = ii.ravel(), jj.ravel()
    x, y = ii * hx, jj * hy
    wall = (jj == 0) | (jj == n_y - 1)
    rng = np.random.Generator(np.random.PCG64(seed))
    x = np.where(wall, x, x + rng.uniform(-0.25, 0.25, x.shape) * hx) % length
    y = np.where(wall, y, y + rng.uniform(-0.25, 0.25, y.shape) * hy)
    mu = height / re
    f = 8.0 * mu / height**2
    tag = np.where(wall, TAG_DIRICHLET, TAG_INTERIOR).astype(np.int8)
    ny = np.where(jj == 0, -1.0, np.where(jj == n_y - 1, 1.0, 0.0))
    ue = f * y * (height - y) / (2.0 * mu)
    return FlowProblem(
        name=f"pchannel{n_x}x{n_y}", x=x, y=y, tag=tag, nx=np.zeros_like(x), ny=ny,
        ubc=np.zeros_like(x), vbc=np.zeros_like(x), pin=_pin_index(x, y, wall, 0.5 * length, 0.0),
        rho=1.0, mu=mu, degree=degree, q=q, dt=dt,
        exact={"u": ue, "v": np.zeros_like(x), "p": np.zeros_like(x)},
        period=(length, 0.0), force=(f, 0.0))


def couette_exact(x, y, r1=0.5, r2=1.0, omega=2.0, rho=1.0):
    """Cylindrical Couette flow; pressure zero at r = r2."""
    r = np.hypot(x, y)
    a = omega * r1 * r1 * r2 / (r2 * r2 - r1 * r1)
    vt = a * (r2 / r - r / r2)
    th = np.arctan2(y, x)

    def prim(rr):  # integral of v_theta^2 / r
        return a * a * (-r2 * r2 / (2 * rr * rr) - 2.0 * np.log(rr) + rr * rr / (2 * r2 * r2))
    return -vt * np.sin(th), vt * np.cos(th), rho * (prim(r) - prim(r2))


def couette(h=0.036, r1=0.5, r2=1.0, omega=2.0, re=100.0, seed=7, degree=3, q=None, dt=None):
    rng = np.random.Generator(np.random.PCG64(seed))
    nr = max(2, int(round((r2 - r1) / h)))
    dr = (r2 - r1) / nr
    xs, ys, ts, nxs, nys = [], [], [], [], []
    for k in range(nr + 1):
        r = r1 + k * dr
        cnt = max(8, int(round(2.0 * math.pi * r / h)))
        th = 2.0 * math.pi * (np.arange(cnt) + rng.uniform()) / cnt
        if 0 < k < nr:
            rr = r + rng.uniform(-0.25, 0.25, cnt) * dr
            tt = th + rng.uniform(-0.25, 0.25, cnt) * h / r
            xs.append(rr * np.cos(tt)); ys.append(rr * np.sin(tt))
            ts.append(np.full(cnt, TAG_INTERIOR, np.int8))
            nxs.append(np.zeros(cnt)); nys.append(np.zeros(cnt))
        else:
            xs.append(r * np.cos(th)); ys.append(r * np.sin(th))
            ts.append(np.full(cnt, TAG_DIRICHLET, np.int8))
            sgn = -1.0 if k == 0 else 1.0  # out of the fluid
            nxs.append(sgn * np.cos(th)); nys.append(sgn * np.sin(th))
    x, y = np.concatenate(xs), np.concatenate(ys)
    tag, nx, ny = np.concatenate(ts), np.concatenate(nxs), np.concatenate(nys)
    order = _morton_order(x, y)
    x, y, tag, nx, ny = x[order], y[order], tag[order], nx[order], ny[order]
    ue, ve, pe = couette_exact(x, y, r1, r2, omega)
    bnd = tag != TAG_INTERIOR
    m = num_monomials(degree)
    if q is None:
        q = 2 * m
    if dt is None:
        # Courant ~2 at the wall speed: at ~10 the Jacobi-preconditioned
        # momentum solve of this flow diverges and no steady state is reached
        dt = 2.0 * h / (omega * r1)
    # the pressure-correction pin sits on the turning inner wall: pinned on
    # the outer wall, the outer iteration diverged on the 7.6k-point cloud
    # (Delta growing ~1.4x per iteration from the first time step)
    pin = _pin_index(x, y, bnd, r1, 0.0)
    return FlowProblem(
        name=f"couette{x.shape[0]}", x=x, y=y, tag=tag, nx=nx, ny=ny,
        ubc=np.where(bnd, ue, 0.0), vbc=np.where(bnd, ve, 0.0), pin=pin, rho=1.0,
        mu=omega * r1 * 2 * r1 / re, degree=degree, q=q, dt=float(dt),
        exact={"u": ue, "v": ve, "p": pe})


def decaying(n_side=65, level=2, seed=8, degree=3, q=None, re=100.0, dt=0.01):
    """Nested clouds of the decaying flow (see the module docstring); the
    initial fields are in ``initial``; ``lattice`` holds each point's
    finest-lattice (i, j)."""
    if (n_side - 1) % 4:
        raise ValueError("n_side - 1 must be a multiple of 4")
    x, y, bnd, nx, ny, ii, jj = _box_cloud(n_side, 0.0, 1.0, seed)
    stride = 1 << (2 - level)
    keep = (ii % stride == 0) & (jj % stride == 0)
    x, y, bnd, nx, ny, ii, jj = (a[keep] for a in (x, y, bnd, nx, ny, ii, jj))
    tag = np.where(bnd, TAG_DIRICHLET, TAG_INTERIOR).astype(np.int8)
    s2 = np.sin(math.pi * x) ** 2, np.sin(math.pi * y) ** 2
    u0 = s2[0] * np.sin(2 * math.pi * y)
    v0 = -np.sin(2 * math.pi * x) * s2[1]
    u0[bnd] = 0.0
    v0[bnd] = 0.0
    m = num_monomials(degree)
    fp = FlowProblem(
        name=f"decaying{(n_side - 1) // stride + 1}", x=x, y=y, tag=tag, nx=nx, ny=ny,
        ubc=np.zeros_like(x), vbc=np.zeros_like(x), pin=_pin_index(x, y, bnd, 0.5, 0.0),
        rho=1.0, mu=1.0 / re, degree=degree, q=2 * m if q is None else q, dt=dt,
        initial={"u": u0, "un": u0, "unm1": u0, "v": v0, "vn": v0, "vnm1": v0})
    fp.lattice = (ii, jj)
    return fp


def random_cloud(n, seed, lo=0.0, hi=1.0):
    """Uniform random points (for stencil and weight tests)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(lo, hi, size=n), rng.uniform(lo, hi, size=n)


def jittered_grid(n_side, seed, lo=0.0, hi=1.0, jitter=0.25):
    """Jittered lattice points without boundary data (for weight tests)."""
    x, y, _, _, _, _, _ = _box_cloud(n_side, lo, hi, seed, jitter=jitter)
    return x, y
