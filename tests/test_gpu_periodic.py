"""Periodic boundaries and the body force on the GPU (paper Sec. 3.1:
clouds wrap around a periodic boundary; a mean pressure gradient drives the
flow), against the oracle."""
import numpy as np
import pytest

import oracle
from gpu_util import ctx, rel_l2
from paper_2106_07616_gb300 import clouds, rbffd

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape", [(24, 13), (150, 40)])
def test_periodic_clouds_bit_exact_and_weights(shape):
    fp = clouds.periodic_channel(*shape)
    P = rbffd.Problem(ctx(), fp)
    O = oracle.Problem(fp)
    g, o = P.operators(), O.operators()
    assert np.array_equal(g["idx"], o["idx"])
    for k in ("wx", "wy", "wl"):
        scale = np.abs(o[k]).max(axis=1, keepdims=True)
        assert (np.abs(g[k] - o[k]) / scale).max() <= 1e-10, k


def test_periodic_outer_iterations_match_oracle():
    fp = clouds.periodic_channel()
    P = rbffd.Problem(ctx(), fp)
    O = oracle.Problem(fp, krylov_tol=1e-12)
    for r in range(3):
        dg, _ = P.simple_iterate(fp.dt, krylov_tol=1e-12)
        do, _ = O.simple_iterate(fp.dt)
        assert abs(dg - do) <= 1e-8 * abs(do)
    for k in ("u", "v", "p"):
        assert rel_l2(P.get(k), O.get(k)) <= 1e-8, k
    rg, ro = P.steady_residual(), O.steady_residual()
    assert np.allclose(rg, ro, rtol=1e-7, atol=0)


def test_force_driven_channel_fixed_point_gpu():
    fp = clouds.periodic_channel()
    P = rbffd.Problem(ctx(), fp, precond=rbffd.PRECOND_AMG)
    for k, f in (("u", "u"), ("un", "u"), ("unm1", "u"), ("v", "v"), ("vn", "v"),
                 ("vnm1", "v"), ("p", "p")):
        P.set(k, fp.exact[f])
    d, _ = P.simple_iterate(fp.dt, krylov_tol=1e-13)
    assert d < 1e-12
    assert np.abs(P.get("u") - fp.exact["u"]).max() < 1e-12
    assert P.steady_residual()[2] < 1e-10


def test_force_driven_channel_from_rest_gpu():
    fp = clouds.periodic_channel()
    P = rbffd.Problem(ctx(), fp, precond=rbffd.PRECOND_AMG)
    rc, st = P.solve_steady(fp.dt, resid_tol=1e-6, max_steps=3000, criterion=1)
    assert np.abs(P.get("u") - fp.exact["u"]).max() < 2e-3


@pytest.mark.parametrize("state", ["rest", "moving"])
def test_courant_helper_matches_oracle(state):
    """The Courant helper's power iteration on the GPU and in the oracle."""
    fp = clouds.kovasznay(30, dt=0.4)
    P = rbffd.Problem(ctx(), fp)
    O = oracle.Problem(fp)
    if state == "moving":
        for X in (P, O):
            X.set("u", fp.exact["u"])
            X.set("v", fp.exact["v"])
    lg, cg = P.courant(fp.dt)
    lo, co = O.courant(fp.dt)
    assert abs(lg - lo) <= 1e-8 * lo
    assert abs(cg - co) <= 1e-8 * co
