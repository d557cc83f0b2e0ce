"""Flow past a cylinder (paper Sec. 5.1) on the GPU: the outlet, symmetry
and no-slip rows together, against the oracle on a small graded cloud, and
spot checks of the full 150 000-point cloud."""
import numpy as np
import pytest

import oracle
from gpu_util import ctx, rel_l2
from paper_2106_07616_gb300 import clouds, rbffd

pytestmark = pytest.mark.gpu


def _start(X, fp):
    for k, a in fp.initial.items():
        X.set(k, a)


@pytest.mark.parametrize("prec, steps", [(rbffd.PREC_FP64, 20), (rbffd.PREC_MIXED_FF, 3)])
def test_small_cylinder_steps_match_oracle(prec, steps):
    """The first time steps from the paper's uniform start, three outer
    iterations each."""
    fp = clouds.cylinder(5000, h0=0.1, hmax=0.5)
    P = rbffd.Problem(ctx(), fp, prec)
    O = oracle.Problem(fp, krylov_tol=1e-12)
    _start(P, fp)
    _start(O, fp)
    for s in range(steps):
        ig, cg = P.time_step(fp.dt, 1e-30, max_outer=3)
        io, co, _ = O.time_step(fp.dt, 1e-30, max_outer=3)
        assert ig == io == 3
        assert abs(cg - co) <= 1e-7 * abs(co), (s, cg, co)
    vel = lambda X: np.concatenate([X.get("u"), X.get("v")])
    assert rel_l2(vel(P), vel(O)) <= 1e-8
    assert rel_l2(P.get("p"), O.get("p")) <= 1e-8


def test_full_cylinder_spot_checks():
    """150 000 points: sampled clouds bit-exact and weights within 1e-10 of
    the oracle's for the same clouds; one outer iteration from the uniform
    start converges with a finite Delta."""
    fp = clouds.cylinder()
    P = rbffd.Problem(ctx(), fp)
    g = P.operators()
    rows = np.random.Generator(np.random.PCG64(11)).choice(fp.n, 256, replace=False)
    rows = np.concatenate([rows, np.where(fp.tag != 0)[0][::97]]).astype(np.int32)
    idx = oracle.knn_rows(fp.x, fp.y, fp.q, rows, fp.tag)
    assert np.array_equal(g["idx"][rows], idx)
    w = oracle.weights_rows(fp.x, fp.y, idx, rows, fp.degree)
    for name, o in zip(("wx", "wy", "wl"), w):
        scale = np.abs(o).max(axis=1, keepdims=True)
        assert (np.abs(g[name][rows] - o) / scale).max() <= 1e-10, name
    _start(P, fp)
    d, st = P.simple_iterate(fp.dt, krylov_tol=1e-10, krylov_maxit=100000)
    assert np.isfinite(d) and d > 0
    assert max(st["relres"]) <= 1e-10
