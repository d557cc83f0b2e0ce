"""Direct pins of the oracle's assembled matrices (paper Sec. 3 and 3.1):
the pressure-correction matrix and the two linearised momentum matrices,
row kind by row kind, applied to a quadratic field.  Weights of degree
>= 2 differentiate a quadratic exactly (to roundoff), so every row has a
closed form: the Laplacian inside, the normal derivative on walls, inlets
and (for the tangential component) symmetry lines, the value itself where
the row is an identity."""
import numpy as np
import pytest

import oracle
from paper_2106_07616_gb300 import clouds

TI, TD, TO, TS = (clouds.TAG_INTERIOR, clouds.TAG_DIRICHLET, clouds.TAG_OUTFLOW,
                  clouds.TAG_SYMMETRY)
C0 = (0.3, -0.7, 0.4, 0.9, -0.5, 0.6)  # a + b x + c y + d x^2 + e x y + g y^2


def quad(x, y, c=C0):
    a, b, cc, d, e, g = c
    f = a + b * x + cc * y + d * x * x + e * x * y + g * y * y
    fx = b + 2 * d * x + e * y
    fy = cc + e * x + 2 * g * y
    lap = np.full_like(x, 2 * d + 2 * g)
    return f, fx, fy, lap


CASES = {"cavity": lambda: clouds.cavity(24, dt=0.05),
         "channel_sym": lambda: clouds.channel(symmetry=True)}


@pytest.mark.parametrize("case", list(CASES))
def test_pressure_correction_rows(case):
    """Laplacian rows inside; n . grad at walls, inlets and symmetry lines
    (homogeneous Neumann p'); identity at outlets (p' = 0) and at the pin."""
    fp = CASES[case]()
    O = oracle.Problem(fp)
    f, fx, fy, lap = quad(fp.x, fp.y)
    got = O.apply("pp", f)
    want = np.where(fp.tag == TI, lap, fp.nx * fx + fp.ny * fy)
    ident = fp.tag == TO
    if fp.pin >= 0:
        ident[fp.pin] = True
    want[ident] = f[ident]
    scale = np.abs(want).max()
    assert np.abs(got - want).max() <= 1e-8 * scale * (1 + np.abs(fp.x).max()) ** 2
    assert ident.any() and (fp.tag != TI).any()


@pytest.mark.parametrize("case", list(CASES))
def test_momentum_rows(case):
    """Eqs. u~ and v~ linearised about the iterate u^r: inside,
    rho a1 / dt f + rho (u^r f_x + v^r f_y) - mu lap f; outlets and the
    tangential component on symmetry lines, n . grad f; identity where the
    component is prescribed (walls, inlets, the normal component on
    symmetry lines).  The matrix of an outer iteration is built from the
    iterate it starts from, which is set here."""
    fp = CASES[case]()
    O = oracle.Problem(fp)
    rng = np.random.Generator(np.random.PCG64(5))
    ur, vr = rng.uniform(-1, 1, fp.n), rng.uniform(-1, 1, fp.n)
    O.set("u", ur)
    O.set("v", vr)
    dt, a1 = 0.07, 1.5
    O.simple_iterate(dt)
    f, fx, fy, lap = quad(fp.x, fp.y)
    inner = fp.rho * a1 / dt * f + fp.rho * (ur * fx + vr * fy) - fp.mu * lap
    neu = fp.nx * fx + fp.ny * fy
    normal_is_x = np.abs(fp.nx) > np.abs(fp.ny)
    for which, comp_is_x in (("mom", True), ("momv", False)):
        got = O.apply(which, f)
        want = np.where(fp.tag == TI, inner, f)
        want = np.where(fp.tag == TO, neu, want)
        sym_tangential = (fp.tag == TS) & (normal_is_x != comp_is_x)
        want = np.where(sym_tangential, neu, want)
        scale = np.abs(want).max()
        assert np.abs(got - want).max() <= 1e-8 * scale * (1 + np.abs(fp.x).max()) ** 2, which
