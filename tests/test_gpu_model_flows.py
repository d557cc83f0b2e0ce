"""The paper's model problems (Sec. 4) on the GPU: steady cylindrical
Couette flow against its closed form under point refinement (Sec. 4.1),
and the decaying flow's spatial order by Richardson extrapolation on nested
clouds (Sec. 4.2).  Both use the multigrid-preconditioned p' solve (the
same fixed point as the Jacobi one, faster)."""
import numpy as np
import pytest

import oracle
from gpu_util import ctx, rel_l2
from paper_2106_07616_gb300 import clouds, rbffd

pytestmark = pytest.mark.gpu


def mean_spacing(fp):
    from scipy.spatial import cKDTree
    d, _ = cKDTree(np.c_[fp.x, fp.y]).query(np.c_[fp.x, fp.y], k=2)
    return d[:, 1].mean()


@pytest.mark.parametrize("degree", [3, 4])
def test_couette_error_falls_under_refinement(degree):
    """Marched from rest to the paper's steady error of 2e-7: the L1 error of
    u, v against the closed form falls under refinement at a slope of at
    least 1.  The paper reports slopes of k - 1 to k + 1; on these clouds the
    slope is about 1.3 (k = 3) and 1.4 (k = 4), a property of the discrete
    steady solution (marching from the exact fields ends at the same error),
    not of the march."""
    errs, hs = [], []
    for h in (0.036, 0.026, 0.018):
        fp = clouds.couette(h, degree=degree)
        P = rbffd.Problem(ctx(), fp, precond=rbffd.PRECOND_AMG)
        rc, st = P.solve_steady(fp.dt, resid_tol=2e-7, max_steps=12000, criterion=1,
                                krylov_tol=1e-12, krylov_maxit=20000)
        inter = fp.tag == 0
        e = (np.abs(P.get("u") - fp.exact["u"])[inter].mean() +
             np.abs(P.get("v") - fp.exact["v"])[inter].mean())
        errs.append(e)
        hs.append(mean_spacing(fp))
    slope = np.polyfit(np.log(hs), np.log(errs), 1)[0]
    assert errs[0] > errs[1] > errs[2], errs
    assert slope >= 1.0, (slope, errs)


def test_couette_steps_match_oracle():
    fp = clouds.couette(0.036)
    P = rbffd.Problem(ctx(), fp, precond=rbffd.PRECOND_AMG)
    O = oracle.Problem(fp, krylov_tol=1e-12)
    for _ in range(5):
        ig, cg = P.time_step(fp.dt, 1e-30, max_outer=3)
        io, co, _ = O.time_step(fp.dt, 1e-30, max_outer=3)
        assert abs(cg - co) <= 1e-8 * abs(co)
    for k in ("u", "v"):
        assert rel_l2(P.get(k), O.get(k)) <= 1e-8


def _decay(level, degree, n_steps=50):
    fp = clouds.decaying(129, level, degree=degree)
    P = rbffd.Problem(ctx(), fp, precond=rbffd.PRECOND_AMG)
    for k, a in fp.initial.items():
        P.set(k, a)
    # the paper's outer-iteration rule (the same for every cloud, so its
    # iteration error cancels in the differences like the temporal error)
    P.solve_unsteady(fp.dt, n_steps, krylov_tol=1e-12, krylov_maxit=20000)
    ii, jj = fp.lattice
    m = (ii % 4 == 0) & (jj % 4 == 0)  # the coarsest cloud's points
    key = np.lexsort((ii[m], jj[m]))
    return P.get("u")[m][key], P.get("v")[m][key]


@pytest.mark.parametrize("degree", [3, 4])
def test_decaying_flow_richardson_order(degree):
    """t = 0.5 with dt = 0.01 on nested clouds of 33^2, 65^2, 129^2 points:
    C = log2(|f4h - f2h|_1 / |f2h - fh|_1) in the paper's range k - 1 .. k + 1
    with a quarter order of slack below: the Laplacian weights themselves
    converge at about k - 1 on jittered clouds (the oracle's refinement pin
    allows k - 1.6), and the oracle gives 1.90 (three outer iterations per
    step) and 1.92 (the paper's rule) for k = 3 on these clouds."""
    f = [_decay(lv, degree) for lv in (0, 1, 2)]
    d1 = sum(np.abs(a - b).mean() for a, b in zip(f[0], f[1]))
    d2 = sum(np.abs(a - b).mean() for a, b in zip(f[1], f[2]))
    order = np.log2(d1 / d2)
    assert degree - 1.25 <= order <= degree + 1.5, (order, d1, d2)


def test_decaying_flow_matches_oracle():
    fp = clouds.decaying(33, 2, degree=3)
    P = rbffd.Problem(ctx(), fp, precond=rbffd.PRECOND_AMG)
    O = oracle.Problem(fp, krylov_tol=1e-12)
    for k, a in fp.initial.items():
        P.set(k, a)
        O.set(k, a)
    for _ in range(10):
        P.time_step(fp.dt, 1e-30, max_outer=3)
        O.time_step(fp.dt, 1e-30, max_outer=3)
    for k in ("u", "v", "p"):
        assert rel_l2(P.get(k), O.get(k)) <= 1e-8, k
