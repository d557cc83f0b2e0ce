"""Pins for the oracle's outer iteration (Sec. 3 steps 2-7), time step
(Sec. 3.2) and steady residual, against closed-form Navier-Stokes flows."""
import numpy as np
import pytest

import flows
import oracle
from paper_2106_07616_gb300 import clouds


def set_state(P, u, v, p):
    for k, a in (("u", u), ("un", u), ("unm1", u), ("v", v), ("vn", v), ("vnm1", v), ("p", p)):
        P.set(k, a)


@pytest.mark.parametrize("make", [flows.stagnation, flows.poiseuille])
def test_closed_form_is_a_fixed_point(make):
    """A steady flow that the weights differentiate exactly satisfies every
    discrete equation: one outer iteration must leave it unchanged."""
    fp = make()
    P = oracle.Problem(fp, krylov_tol=1e-13)
    ex = fp.exact
    set_state(P, ex["u"], ex["v"], ex["p"])
    d, st = P.simple_iterate(fp.dt)
    assert d < 1e-10, d
    for k in ("u", "v", "p"):
        ref = ex[k]
        assert np.abs(P.get(k) - ref).max() <= 1e-9 * max(1.0, np.abs(ref).max()), k
    assert np.abs(P.get("pc")).max() < 1e-9
    R = P.steady_residual()
    assert R.max() < 1e-10, R


def test_fixed_point_detects_a_wrong_pressure():
    """The same check fails when the pressure is off by a non-constant
    field: the outer iteration must move the state."""
    fp = flows.stagnation()
    P = oracle.Problem(fp, krylov_tol=1e-13)
    ex = fp.exact
    set_state(P, ex["u"], ex["v"], ex["p"] + 0.01 * fp.x)
    d, _ = P.simple_iterate(fp.dt)
    assert d > 1e-6


def test_bdf2_accelerating_flow_exact():
    """u, v linear in time and uniform in space, p = -rho (b . x): BDF2 and
    the operators are exact, so one time step lands on the closed form at
    t + dt (the time term of Eqs. u:tilde and normal momentum is exercised
    through the moving boundary values)."""
    fp = flows.accelerating()
    P = oracle.Problem(fp, krylov_tol=1e-13)
    t0 = 1.0
    u1, v1, p1 = fp.at(t0 - fp.dt)
    u0, v0, p0 = fp.at(t0)
    u2, v2, p2 = fp.at(t0 + fp.dt)
    for k, a in (("unm1", u1), ("vnm1", v1), ("un", u0), ("vn", v0), ("u", u0), ("v", v0),
                 ("p", p0), ("ubc", u2), ("vbc", v2)):
        P.set(k, a)
    it, change, last = P.time_step(fp.dt, 1e-12, max_outer=10)
    assert it <= 3, it
    assert np.abs(P.get("un") - u2).max() < 1e-10
    assert np.abs(P.get("vn") - v2).max() < 1e-10
    assert np.abs(P.get("unm1") - u0).max() < 1e-12
    assert np.abs(P.get("p") - p2).max() < 1e-9


def test_steady_residual_truncation_order():
    """R evaluated on the exact Kovasznay fields is the truncation error of
    the discrete steady equations: it must fall under refinement."""
    Rs = []
    for ns in (20, 40):
        fp = clouds.kovasznay(ns)
        P = oracle.Problem(fp)
        ex = fp.exact
        set_state(P, ex["u"], ex["v"], ex["p"])
        Rs.append(P.steady_residual()[2])
    assert Rs[1] < Rs[0] / 4, Rs


def test_krylov_tolerance_path_independence():
    """The outer iterate depends on the Krylov solves only through their
    residual: tolerances 1e-10 and 1e-13 give the same step to ~1e-7."""
    fp = clouds.kovasznay(24, dt=0.4)
    out = []
    for tol in (1e-10, 1e-13):
        P = oracle.Problem(fp, krylov_tol=tol)
        for _ in range(3):
            P.simple_iterate(fp.dt)
        out.append([P.get(k) for k in ("u", "v", "p")])
    for a, b in zip(*out):
        assert np.linalg.norm(a - b) <= 1e-6 * np.linalg.norm(b)


def test_kovasznay_marches_toward_closed_form():
    """Pseudo-time marching from rest reduces the steady residual and the
    distance to the closed form (coarse cloud, bounded work)."""
    fp = clouds.kovasznay(30, dt=0.4)
    P = oracle.Problem(fp, krylov_tol=1e-10)
    rc, info = P.solve_steady(fp.dt, resid_tol=5e-3, max_steps=400, max_outer=20)
    assert rc == 0, info
    err = np.abs(P.get("u") - fp.exact["u"]).max()
    assert err < 0.06, err


def test_steady_error_criterion_matches_manual_march():
    """The paper's steady-state test (Sec. 4.1): stop once the mean change
    of u and v between consecutive steps, divided by dt, is below the
    tolerance.  A march driven one time step at a time, with the outer
    tolerance rule of Sec. 3.2 and that stopping test, takes the same number
    of steps and lands on the same fields."""
    fp = clouds.kovasznay(30, dt=0.4)
    tol = 2e-3
    A = oracle.Problem(fp, krylov_tol=1e-10)
    rc, info = A.solve_steady(fp.dt, resid_tol=tol, max_steps=400, max_outer=20, criterion=1)
    assert rc == 0, info
    assert info["change"] / fp.dt <= tol
    B = oracle.Problem(fp, krylov_tol=1e-10)
    tol_outer, steps = 1e-4, 0
    while True:
        _, change, _ = B.time_step(fp.dt, tol_outer, 20)
        steps += 1
        tol_outer = min(1e-4, change)
        if change / fp.dt <= tol:
            break
        assert steps < 400
    assert steps == info["steps"]
    for k in ("u", "v", "p"):
        np.testing.assert_array_equal(A.get(k), B.get(k))


def test_unsteady_driver_follows_the_outer_tolerance_rule():
    """The unsteady driver marches n steps with the outer tolerance of
    Sec. 3 (1e-4 on the first step, then min(1e-4, dt eps_s) with dt eps_s
    the mean change of u and v over the last step): a march driven one time
    step at a time with that rule takes the same outer iterations and lands
    on the same fields, bit for bit.  A small step (2e-4) keeps the change
    per step near 1e-4, so the rule's minimum is taken on some steps."""
    fp = clouds.decaying(33, 2, degree=3, dt=2e-4)
    A = oracle.Problem(fp, krylov_tol=1e-12)
    B = oracle.Problem(fp, krylov_tol=1e-12)
    for X in (A, B):
        for k, a in fp.initial.items():
            X.set(k, a)
    n = 12
    rc, info = A.solve_unsteady(fp.dt, n, max_outer=20)
    assert rc == 0 and info["steps"] == n
    tol_outer, outer, tols = 1e-4, 0, []
    for _ in range(n):
        it, change, _ = B.time_step(fp.dt, tol_outer, 20)
        outer += it
        tols.append(tol_outer)
        tol_outer = min(1e-4, change)
    assert outer == info["outer"] and change == info["change"]
    assert min(tols) < 1e-4  # the rule took the measured change on some steps
    for k in ("u", "v", "p", "un", "unm1"):
        np.testing.assert_array_equal(A.get(k), B.get(k))


def test_oracle_does_not_depend_on_the_thread_count():
    """The oracle's OpenMP loops run over points and rows and its dot
    products are serial in index order, so clouds, weights and outer
    iterates are bit-identical on one thread and on four."""
    fp = clouds.kovasznay(20, dt=0.4)
    before = oracle.set_threads(0)  # 0 leaves the count as it is
    out = []
    try:
        for t in (1, 4):
            oracle.set_threads(t)
            O = oracle.Problem(fp, krylov_tol=1e-12)
            for _ in range(3):
                O.simple_iterate(fp.dt)
            out.append([O.get(k) for k in ("u", "v", "p")] + list(O.operators().values()))
    finally:
        oracle.set_threads(before)
    for a, b in zip(*out):
        np.testing.assert_array_equal(a, b)
