"""Pin of the Courant helper (paper Sec. 3.2: lambda dt / 2 with lambda from
the discrete convection-diffusion operator): its power-iteration lambda
against the spectral radius of the dense operator."""
import numpy as np
import pytest

import oracle
from paper_2106_07616_gb300 import clouds


def dense_operator(O, fp):
    n = fp.n
    u, v = O.get("u"), O.get("v")
    Dx = np.array([O.apply("dx", e) for e in np.eye(n)]).T
    Dy = np.array([O.apply("dy", e) for e in np.eye(n)]).T
    L = np.array([O.apply("lap", e) for e in np.eye(n)]).T
    C = fp.rho * (u[:, None] * Dx + v[:, None] * Dy) - fp.mu * L
    C[fp.tag != 0] = 0.0
    return C


@pytest.mark.parametrize("state", ["rest", "kovasznay"])
def test_courant_lambda_matches_spectral_radius(state):
    fp = clouds.kovasznay(16, dt=0.4)
    O = oracle.Problem(fp)
    if state == "kovasznay":
        O.set("u", fp.exact["u"])
        O.set("v", fp.exact["v"])
    lam, co = O.courant(fp.dt, iters=400)
    rho = np.abs(np.linalg.eigvals(dense_operator(O, fp))).max()
    assert abs(lam - rho) <= 0.05 * rho, (lam, rho)
    assert co == pytest.approx(lam * fp.dt / 2)


def test_courant_scales_with_viscosity_at_rest():
    """At rest only diffusion is left: lambda is proportional to mu."""
    import dataclasses
    fp = clouds.kovasznay(16, dt=0.4)
    l1 = oracle.Problem(fp).courant(fp.dt)[0]
    l2 = oracle.Problem(dataclasses.replace(fp, mu=2 * fp.mu)).courant(fp.dt)[0]
    assert l2 == pytest.approx(2 * l1, rel=1e-12)
