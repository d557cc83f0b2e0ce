"""The oracle against values the paper prints (fixtures in tests/golden/,
each citing its passage)."""
import os
from math import comb

import numpy as np

import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_monomial_order_of_the_worked_example():
    """Sec. 2, Eq. RBF_interp_poly: d = 2, k = 2 gives the six terms
    1, x, y, x^2, xy, y^2 as the columns of P, in that order."""
    want = np.loadtxt(os.path.join(GOLDEN, "monomials_d2_k2.txt"), dtype=np.int32)
    ax, ay = oracle.monomial_exponents(2)
    assert len(want) == comb(2 + 2, 2) == 6
    assert np.array_equal(np.stack([ax, ay], 1), want)


def test_monomial_order_is_graded_for_every_degree():
    """The same rule for the degrees the configurations use (2..6): every
    term of total degree <= k once, by total degree, the x power
    descending within a degree -- which for k = 2 is the printed order."""
    for k in range(7):
        ax, ay = oracle.monomial_exponents(k)
        assert len(ax) == comb(k + 2, k)
        terms = list(zip(ax.tolist(), ay.tolist()))
        assert len(set(terms)) == len(terms)
        assert all(a + b <= k for a, b in terms)
        assert terms == sorted(terms, key=lambda t: (t[0] + t[1], -t[0]))


def bdf2():
    return np.loadtxt(os.path.join(GOLDEN, "bdf2_coefficients.txt"))


def test_printed_bdf2_coefficients_are_second_order():
    """The printed alphas differentiate 1, (t - t1) and (t - t1)^2 exactly
    at t1 = t_{n+1} -- the three conditions that define BDF2."""
    a1, a2, a3 = bdf2()
    for f, df in ((lambda s: 1.0, 0.0), (lambda s: s, 1.0), (lambda s: s * s, 0.0)):
        # nodes at s = 0, -1, -2 (units of dt) relative to t_{n+1}
        assert a1 * f(0.0) + a2 * f(-1.0) + a3 * f(-2.0) == df


def test_oracle_time_step_uses_the_printed_bdf2():
    """A uniform flow quadratic in time is, with its exact history, a fixed
    point of the discrete step at t + dt only for these three alphas
    (linear-in-time flows pin two of the conditions, this one the third):
    a time step started on the closed form at t + dt stays there."""
    import flows
    fp = flows.accelerating(c=(0.7, -0.4))
    P = oracle.Problem(fp, krylov_tol=1e-13)
    t0 = 1.0
    u1, v1, _ = fp.at(t0 - fp.dt)
    u0, v0, _ = fp.at(t0)
    u2, v2, p2 = fp.at(t0 + fp.dt)
    for k, a in (("unm1", u1), ("vnm1", v1), ("un", u0), ("vn", v0), ("u", u2), ("v", v2),
                 ("p", p2), ("ubc", u2), ("vbc", v2)):
        P.set(k, a)
    it, _, _ = P.time_step(fp.dt, 1e-10, max_outer=10)
    assert it <= 2, it
    assert np.abs(P.get("un") - u2).max() < 1e-10
    assert np.abs(P.get("vn") - v2).max() < 1e-10
    assert np.abs(P.get("p") - p2).max() < 1e-9
    # the defaults of the oracle's outer iteration are the printed values
    import inspect
    assert inspect.signature(oracle.Problem.simple_iterate).parameters["alpha"].default == \
        tuple(bdf2())
