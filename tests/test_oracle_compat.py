"""Pins for the compatible pressure-correction equation of the oracle.

With Neumann rows only (Sec. 3.1: homogeneous Neumann p' at walls and
inlets; no outlet), the discrete p' operator L_N maps constants to zero and
is solvable only for a right-hand side orthogonal to its left null vector
psi.  The oracle makes the source (rho a1/dt) div u~ compatible by taking
away a multiple of e_I (1 at interior rows) and fixes the free constant with
the pin.  These tests check the definition itself (psi, the full Neumann
system including the pin's own row), that the steady march then reaches the
metric's residual, and that the plain pin (planted by switching the
compatibility off) violates the dropped row and stalls.
"""
import numpy as np
import pytest

import oracle
from paper_2106_07616_gb300 import clouds


def neumann_operator(fp, ops):
    """Dense L_N: Laplacian rows inside, n.grad rows on the boundary."""
    n, q = ops["idx"].shape
    L = np.zeros((n, n))
    for i in range(n):
        w = ops["wl"][i] if fp.tag[i] == 0 else fp.nx[i] * ops["wx"][i] + fp.ny[i] * ops["wy"][i]
        np.add.at(L[i], ops["idx"][i], w)
    return L


def apply(ops, w, f):
    return (w * f[ops["idx"]]).sum(axis=1)


def test_psi_is_the_left_null_vector():
    fp = clouds.kovasznay(14, dt=0.1)
    O = oracle.Problem(fp, krylov_tol=1e-13)
    ops = O.operators()
    L = neumann_operator(fp, ops)
    psi = O.compat()
    assert abs(psi[fp.pin] - 1.0) < 1e-9
    # constants are in the right null space (row sums zero), psi in the left
    assert np.abs(L @ np.ones(fp.n)).max() < 1e-9 * np.abs(L).max()
    assert np.abs(psi @ L).max() < 1e-9 * np.abs(psi).max() * np.abs(L).max()
    # an independent left null vector (SVD) is parallel to psi
    _, sv, vt = np.linalg.svd(L.T)
    ref = vt[-1] / vt[-1][fp.pin]
    assert sv[-1] < 1e-10 * sv[0]
    assert np.abs(ref - psi).max() < 1e-7 * np.abs(psi).max()
    assert abs(psi[fp.tag == 0].sum()) > 1e-3 * np.abs(psi).sum()


def _one_iteration(compat):
    fp = clouds.kovasznay(20, dt=0.1)
    O = oracle.Problem(fp, krylov_tol=1e-13)
    if not compat:
        O.set_compat(False)
    O.simple_iterate(fp.dt)
    ops = O.operators()
    ut, vt, pc = O.get("ut"), O.get("vt"), O.get("pc")
    b = np.where(fp.tag == 0, 1.5 / fp.dt * (apply(ops, ops["wx"], ut) + apply(ops, ops["wy"], vt)),
                 0.0)
    L = neumann_operator(fp, ops)
    res = L @ pc - b
    return fp, res, b


def test_compatible_pprime_solves_the_whole_neumann_system():
    """Every Neumann row holds, the pin's included, and the interior rows
    differ from the source by one constant (the removed incompatible part)."""
    fp, res, b = _one_iteration(True)
    scale = np.abs(b).max()
    inner = res[fp.tag == 0]
    assert np.abs(res[fp.tag != 0]).max() < 1e-9 * scale  # pin row too
    assert np.abs(inner - inner.mean()).max() < 1e-9 * scale
    assert abs(inner.mean()) > 1e-6 * scale  # this source was not compatible


def test_plain_pin_violates_the_dropped_row():
    """Planted: the compatibility switched off, the pin's own Neumann row is
    no longer satisfied (the incompatible part is pushed into it)."""
    fp, res, b = _one_iteration(False)
    scale = np.abs(b).max()
    assert abs(res[fp.pin]) > 1e-6 * scale
    others = np.ones(fp.n, bool)
    others[fp.pin] = False
    assert np.abs(res[others]).max() < 1e-9 * scale


def test_steady_march_reaches_the_metric_residual():
    """Kovasznay 20^2: the compatible march reaches R <= 1e-8 (continuity
    taken up to its constant lambda); with the plain pin (planted) the
    residual stalls far above it over the same number of steps."""
    fp = clouds.kovasznay(20, dt=0.05)
    O = oracle.Problem(fp, krylov_tol=1e-12)
    rc, st = O.solve_steady(fp.dt, resid_tol=1e-8, max_steps=3000)
    assert rc == 0, st
    R = O.steady_residual()
    assert R[2] <= 1e-8
    lam = R[3]
    # lambda is the uniform part of the divergence: the divergence minus
    # lambda is what R_c measures
    ops = O.operators()
    d = (apply(ops, ops["wx"], O.get("u")) + apply(ops, ops["wy"], O.get("v")))[fp.tag == 0]
    assert abs(d.mean() - lam) <= 1e-12 + 1e-9 * abs(lam)
    P = oracle.Problem(fp, krylov_tol=1e-12)
    P.set_compat(False)
    rc2, st2 = P.solve_steady(fp.dt, resid_tol=1e-8, max_steps=st["steps"])
    assert rc2 != 0 and st2["R"] > 1e-6, st2


def test_kovasznay_error_decays_under_refinement():
    """Closed-form Kovasznay flow (Re 40), degree 3, marched to R <= 1e-8 on
    13^2, 19^2 and 25^2 clouds: the L1 error of u and v falls at a slope
    between k - 1.5 and k + 1 (Sec. 4.1: the Navier-Stokes error converges
    between the Laplacian's k - 1 and the interpolant's k + 1 orders; the
    coarsest cloud is still pre-asymptotic), and the continuity constant
    lambda shrinks."""
    hs, eu, ev, lams = [], [], [], []
    for ns, dt in ((13, 0.1), (19, 0.07), (25, 0.05)):
        fp = clouds.kovasznay(ns, dt=dt)
        O = oracle.Problem(fp, krylov_tol=1e-12)
        rc, st = O.solve_steady(dt, resid_tol=1e-8, max_steps=20000)
        assert rc == 0, (ns, st)
        inner = fp.tag == 0
        eu.append(np.abs(O.get("u") - fp.exact["u"])[inner].mean())
        ev.append(np.abs(O.get("v") - fp.exact["v"])[inner].mean())
        lams.append(abs(O.steady_residual()[3]))
        hs.append(2.0 / (ns - 1))
    for e in (eu, ev):
        slope = np.polyfit(np.log(hs), np.log(e), 1)[0]
        assert 1.5 <= slope <= 4.0, (slope, e)
        assert e[0] > e[1] > e[2]
    assert lams[2] < lams[0], lams
