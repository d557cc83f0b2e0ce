"""Closed-form flows used to pin the oracle and the CUDA path.

Each is an exact solution of the incompressible Navier-Stokes equations
whose velocity and pressure are polynomials of degree <= 2 in space.  The
PHS-RBF-FD weights reproduce every polynomial up to the appended degree
exactly (the constraint rows of Sec. 2), so for these flows the discrete
operators are exact and the discrete equations are satisfied by the closed
form itself, up to rounding.
"""
import numpy as np

from paper_2106_07616_gb300 import clouds


def _box(n_side, seed, degree=3, q=20, rho=1.0, mu=0.05, dt=0.1, lo=-0.5, hi=1.5):
    fp = clouds.kovasznay(n_side, seed=seed, degree=degree, q=q, dt=dt)
    fp.rho, fp.mu = rho, mu
    fp.x = lo + (fp.x + 0.5) * (hi - lo) / 2.0
    fp.y = lo + (fp.y + 0.5) * (hi - lo) / 2.0
    fp.exact = None
    return fp


def stagnation(n_side=24, seed=11, degree=3, q=20, rho=1.3, mu=0.07, dt=0.1):
    """Steady stagnation-point flow u = x, v = -y, p = -rho (x^2 + y^2) / 2."""
    fp = _box(n_side, seed, degree, q, rho, mu, dt)
    u, v, p = fp.x.copy(), -fp.y.copy(), -rho * (fp.x ** 2 + fp.y ** 2) / 2.0
    bnd = fp.tag != 0
    fp.ubc = np.where(bnd, u, 0.0)
    fp.vbc = np.where(bnd, v, 0.0)
    fp.exact = {"u": u, "v": v, "p": p}
    fp.name = "stagnation"
    return fp


def poiseuille(n_side=24, seed=12, degree=3, q=20, rho=1.0, mu=0.2, dt=0.1):
    """Steady shear flow u = y^2, v = 0, p = 2 mu x (viscous balance)."""
    fp = _box(n_side, seed, degree, q, rho, mu, dt)
    u, v, p = fp.y ** 2, np.zeros_like(fp.x), 2.0 * mu * fp.x
    bnd = fp.tag != 0
    fp.ubc = np.where(bnd, u, 0.0)
    fp.vbc = np.where(bnd, v, 0.0)
    fp.exact = {"u": u, "v": v, "p": p}
    fp.name = "poiseuille"
    return fp


def accelerating(n_side=20, seed=13, degree=3, q=20, rho=0.9, mu=0.03, dt=0.25, a=(0.4, -0.2),
                 b=(0.3, 0.5), c=(0.0, 0.0)):
    """Uniform flow whose velocity is a polynomial of degree <= 2 in time:
    u = a0 + b0 t + c0 t^2, v = a1 + b1 t + c1 t^2, and
    p = -rho ((b0 + 2 c0 t) x + (b1 + 2 c1 t) y).
    BDF2 differentiates such a function of time exactly."""
    fp = _box(n_side, seed, degree, q, rho, mu, dt)

    def at(t):
        u = np.full(fp.n, a[0] + b[0] * t + c[0] * t * t)
        v = np.full(fp.n, a[1] + b[1] * t + c[1] * t * t)
        p = -rho * ((b[0] + 2 * c[0] * t) * fp.x + (b[1] + 2 * c[1] * t) * fp.y)
        return u, v, p

    fp.at = at
    fp.name = "accelerating"
    return fp
