"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Stencils: bit-exact.  Weights: 1e-10 relative per cloud.  Fields after
outer iterations and time steps: 1e-8 relative L2 (FP64 path)."""
import numpy as np
import pytest
import torch

import flows
import oracle
from gpu_util import ctx, dev, rel_l2
from paper_2106_07616_gb300 import clouds, rbffd

pytestmark = pytest.mark.gpu


def gpu_knn(x, y, q, tag=None):
    n = x.size
    idx = torch.zeros(n * q, dtype=torch.int32, device="cuda:0")
    rbffd.rbffd_build_stencils(ctx(), dev(x), dev(y), None if tag is None else dev(tag), q, idx)
    return idx.cpu().numpy().reshape(n, q)


def gpu_weights(x, y, idx, degree):
    n, q = idx.shape
    w = [torch.zeros(n * q, dtype=torch.float64, device="cuda:0") for _ in range(3)]
    fs = rbffd.rbffd_weights(ctx(), dev(x), dev(y), q, dev(idx.ravel()), degree, *w)
    return fs, [a.cpu().numpy().reshape(n, q) for a in w]


@pytest.mark.parametrize("n,q,seed", [(1, 1, 0), (33, 7, 1), (3000, 20, 2), (5000, 42, 3)])
def test_stencils_random_bit_exact(n, q, seed):
    x, y = clouds.random_cloud(n, seed)
    assert np.array_equal(gpu_knn(x, y, q), oracle.knn(x, y, q))


def test_stencils_lattice_ties_bit_exact():
    s = np.arange(40, dtype=np.float64)
    x, y = np.meshgrid(s, s)
    x, y = x.ravel().copy(), y.ravel().copy()
    assert np.array_equal(gpu_knn(x, y, 21), oracle.knn(x, y, 21))


@pytest.mark.parametrize("make", [lambda: clouds.kovasznay(50), lambda: clouds.cavity(64)])
def test_stencils_with_boundaries_bit_exact(make):
    fp = make()
    assert np.array_equal(gpu_knn(fp.x, fp.y, fp.q, fp.tag), oracle.knn(fp.x, fp.y, fp.q, fp.tag))


@pytest.mark.parametrize("degree,q", [(1, 6), (2, 12), (3, 20), (4, 30), (5, 42), (6, 56)])
def test_weights_parity(degree, q):
    x, y = clouds.jittered_grid(30, seed=degree)
    idx = oracle.knn(x, y, q)
    fs, (gx, gy, gl) = gpu_weights(x, y, idx, degree)
    assert fs == -1
    ox, oy, ol = oracle.weights(x, y, idx, degree)
    for g, o in ((gx, ox), (gy, oy), (gl, ol)):
        scale = np.abs(o).max(axis=1, keepdims=True)
        err = (np.abs(g - o) / scale).max()
        assert err <= 1e-10, err


def test_weights_singular_reported():
    x, y = clouds.random_cloud(200, seed=4)
    x[17], y[17] = x[50], y[50]
    idx = oracle.knn(x, y, 12)
    fs, _ = gpu_weights(x, y, idx, 2)
    assert fs >= 0


def _pair(fp, tol=1e-12, precision=rbffd.PREC_FP64):
    P = rbffd.Problem(ctx(), fp, precision)
    O = oracle.Problem(fp, krylov_tol=tol)
    return P, O


def test_problem_operators_match_oracle():
    fp = clouds.kovasznay(30, dt=0.4)
    P, O = _pair(fp)
    g, o = P.operators(), O.operators()
    assert np.array_equal(g["idx"], o["idx"])
    for k in ("wx", "wy", "wl", "pval"):
        scale = np.abs(o[k]).max(axis=1, keepdims=True)
        assert (np.abs(g[k] - o[k]) / scale).max() <= 1e-10, k


def test_closed_form_fixed_point_gpu():
    fp = flows.stagnation()
    P = rbffd.Problem(ctx(), fp)
    ex = fp.exact
    for k, a in (("u", ex["u"]), ("un", ex["u"]), ("unm1", ex["u"]), ("v", ex["v"]),
                 ("vn", ex["v"]), ("vnm1", ex["v"]), ("p", ex["p"])):
        P.set(k, a)
    d, st = P.simple_iterate(fp.dt, krylov_tol=1e-13)
    assert d < 1e-10
    for k in ("u", "v", "p"):
        assert np.abs(P.get(k) - ex[k]).max() <= 1e-9 * max(1.0, np.abs(ex[k]).max())
    assert P.steady_residual()[2] < 1e-10


@pytest.mark.parametrize("kind", ["kovasznay", "cavity"])
def test_outer_iterations_match_oracle(kind):
    fp = clouds.kovasznay(30, dt=0.4) if kind == "kovasznay" else clouds.cavity(40, dt=0.05)
    P, O = _pair(fp)
    for r in range(3):
        dg, sg = P.simple_iterate(fp.dt, krylov_tol=1e-12)
        do, so = O.simple_iterate(fp.dt)
        assert abs(dg - do) <= 1e-8 * abs(do), (r, dg, do)
        for k in ("ut", "vt", "pc", "u", "v", "p"):
            e = rel_l2(P.get(k), O.get(k))
            assert e <= 1e-8, (r, k, e)


def test_time_steps_and_residual_match_oracle():
    fp = clouds.kovasznay(30, dt=0.4)
    P, O = _pair(fp)
    for s in range(3):
        ig, cg = P.time_step(fp.dt, 1e-30, max_outer=3)
        io, co, _ = O.time_step(fp.dt, 1e-30, max_outer=3)
        assert ig == io == 3
        assert abs(cg - co) <= 1e-8 * abs(co)
    for k in ("u", "v", "p", "un", "vn", "unm1", "vnm1"):
        assert rel_l2(P.get(k), O.get(k)) <= 1e-8, k
    rg, ro = P.steady_residual(), O.steady_residual()
    assert np.allclose(rg, ro, rtol=1e-7, atol=0)


def test_bdf2_accelerating_flow_gpu():
    fp = flows.accelerating()
    P = rbffd.Problem(ctx(), fp)
    t0 = 1.0
    u1, v1, _ = fp.at(t0 - fp.dt)
    u0, v0, p0 = fp.at(t0)
    u2, v2, p2 = fp.at(t0 + fp.dt)
    for k, a in (("unm1", u1), ("vnm1", v1), ("un", u0), ("vn", v0), ("u", u0), ("v", v0),
                 ("p", p0), ("ubc", u2), ("vbc", v2)):
        P.set(k, a)
    it, ch = P.time_step(fp.dt, 1e-12, max_outer=10, krylov_tol=1e-13)
    assert it <= 3
    assert np.abs(P.get("un") - u2).max() < 1e-10
    assert np.abs(P.get("p") - p2).max() < 1e-9


def test_bdf2_quadratic_in_time_fixed_point_gpu():
    """The paper's BDF2 coefficients (Sec. 3) make a uniform flow quadratic
    in time, with its exact history, a fixed point of the step at t + dt:
    the GPU step started there stays there."""
    fp = flows.accelerating(c=(0.7, -0.4))
    P = rbffd.Problem(ctx(), fp)
    t0 = 1.0
    u1, v1, _ = fp.at(t0 - fp.dt)
    u0, v0, _ = fp.at(t0)
    u2, v2, p2 = fp.at(t0 + fp.dt)
    for k, a in (("unm1", u1), ("vnm1", v1), ("un", u0), ("vn", v0), ("u", u2), ("v", v2),
                 ("p", p2), ("ubc", u2), ("vbc", v2)):
        P.set(k, a)
    it, ch = P.time_step(fp.dt, 1e-10, max_outer=10, krylov_tol=1e-13)
    assert it <= 2
    assert np.abs(P.get("un") - u2).max() < 1e-10
    assert np.abs(P.get("vn") - v2).max() < 1e-10
    assert np.abs(P.get("p") - p2).max() < 1e-9


def test_solve_steady_reaches_tolerance_like_oracle():
    fp = clouds.kovasznay(30, dt=0.4)
    P, O = _pair(fp, tol=1e-10)
    rc, sg = P.solve_steady(fp.dt, resid_tol=5e-3, max_steps=400, krylov_tol=1e-10)
    rco, so = O.solve_steady(fp.dt, resid_tol=5e-3, max_steps=400)
    assert rco == 0
    assert sg["resid"][2] <= 5e-3
    # the march is path-dependent only through rounding: same step count
    # within one, and the same state to the residual tolerance
    assert abs(sg["steps"] - so["steps"]) <= 1
    assert rel_l2(P.get("u"), O.get("u")) < 1e-3


def test_solve_steady_paper_criterion_like_oracle():
    """Stopping on the paper's steady error (change / dt, Sec. 4.1) gives the
    oracle's step count within one and the same state."""
    fp = clouds.kovasznay(30, dt=0.4)
    P, O = _pair(fp, tol=1e-10)
    rc, sg = P.solve_steady(fp.dt, resid_tol=2e-3, max_steps=400, krylov_tol=1e-10,
                            criterion=1)
    rco, so = O.solve_steady(fp.dt, resid_tol=2e-3, max_steps=400, criterion=1)
    assert rco == 0
    assert sg["change"] / fp.dt <= 2e-3
    assert abs(sg["steps"] - so["steps"]) <= 1
    assert rel_l2(P.get("u"), O.get("u")) < 1e-3


def test_reload_resets_and_matches_fresh():
    fp = clouds.kovasznay(30, dt=0.4)
    P = rbffd.Problem(ctx(), fp)
    P.simple_iterate(fp.dt)
    fp2 = clouds.kovasznay(30, seed=9, dt=0.4)
    P.reload(fp2)
    Q = rbffd.Problem(ctx(), fp2)
    d1, _ = P.simple_iterate(fp.dt)
    d2, _ = Q.simple_iterate(fp.dt)
    assert d1 == d2
    assert np.array_equal(P.get("u"), Q.get("u"))


def test_bad_arguments_rejected():
    fp = clouds.kovasznay(12)
    fp.q = 5  # q < m = 10
    with pytest.raises(rbffd.RbffdError) as e:
        rbffd.Problem(ctx(), fp)
    assert e.value.code == rbffd.EINVAL
    fp = clouds.kovasznay(12)
    fp.pin = 70  # an interior point
    with pytest.raises(rbffd.RbffdError):
        rbffd.Problem(ctx(), fp)


@pytest.mark.parametrize("prec", [rbffd.PREC_MIXED, rbffd.PREC_MIXED_FF])
@pytest.mark.parametrize("kind", ["kovasznay", "cavity"])
def test_mixed_precision_outer_iterations_match_oracle(kind, prec):
    """FP32 or float-float BiCGSTAB inside FP64 defect correction stops on
    the same FP64 relative residual as the FP64 solver, so the outer iterates
    agree with the FP64 oracle to the same tolerance."""
    fp = clouds.kovasznay(30, dt=0.4) if kind == "kovasznay" else clouds.cavity(40, dt=0.05)
    P = rbffd.Problem(ctx(), fp, prec)
    O = oracle.Problem(fp, krylov_tol=1e-12)
    for r in range(3):
        dg, sg = P.simple_iterate(fp.dt, krylov_tol=1e-12)
        do, so = O.simple_iterate(fp.dt)
        assert max(sg["relres"]) <= 1e-12
        assert sg["sweeps"][2] >= 1
        assert abs(dg - do) <= 1e-8 * abs(do), (r, dg, do)
        for k in ("u", "v", "p"):
            e = rel_l2(P.get(k), O.get(k))
            assert e <= 1e-8, (r, k, e)


@pytest.mark.parametrize("prec", [rbffd.PREC_MIXED, rbffd.PREC_MIXED_FF])
def test_mixed_and_fp64_paths_agree_on_steps(prec):
    fp = clouds.kovasznay(30, dt=0.4)
    A = rbffd.Problem(ctx(), fp, rbffd.PREC_FP64)
    B = rbffd.Problem(ctx(), fp, prec)
    for _ in range(2):
        A.time_step(fp.dt, 1e-4, max_outer=3)
        B.time_step(fp.dt, 1e-4, max_outer=3)
    for k in ("u", "v", "p"):
        assert rel_l2(B.get(k), A.get(k)) <= 1e-8


def test_float_float_path_on_full_cavity_matches_fp64_path():
    """The 200 x 200 cavity (N = 40 000): the FP32 inner solve cannot reach
    it (cond * eps_fp32 ~ 1), float-float can; both stop on the same FP64
    residual as the FP64 path, so the outer iterates agree."""
    fp = clouds.cavity(200)
    A = rbffd.Problem(ctx(), fp, rbffd.PREC_FP64)
    B = rbffd.Problem(ctx(), fp, rbffd.PREC_MIXED_FF)
    for _ in range(2):
        da, _ = A.simple_iterate(fp.dt, krylov_tol=1e-12, krylov_maxit=100000)
        db, sb = B.simple_iterate(fp.dt, krylov_tol=1e-12, krylov_maxit=100000)
        assert max(sb["relres"]) <= 1e-12
        assert abs(da - db) <= 1e-8 * abs(da)
    for k in ("u", "v", "p"):
        assert rel_l2(B.get(k), A.get(k)) <= 1e-8, k
