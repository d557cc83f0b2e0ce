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


def random_cloud(n, seed, lo=0.0, hi=1.0):
    """Uniform random points (for stencil and weight tests)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(lo, hi, size=n), rng.uniform(lo, hi, size=n)


def jittered_grid(n_side, seed, lo=0.0, hi=1.0, jitter=0.25):
    """Jittered lattice points without boundary data (for weight tests)."""
    x, y, _, _, _, _, _ = _box_cloud(n_side, lo, hi, seed, jitter=jitter)
    return x, y
