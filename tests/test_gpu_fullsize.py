"""Full-size parity with the oracle on the workloads the benchmark and the
scope name: the 200 x 200 lid-driven cavity (Re 1000, degree 4, q 30; the
benchmark step), Kovasznay flow on 50 x 50 points (Re 40, degree 3, q 20)
and the 150 000-point cylinder (Re 100, degree 3, q 20).  u, v and p are
compared with oracle.Problem at 1e-8 relative L2 after the same outer
iterations, on the default path (flexible GMRES with an FP32 Arnoldi
process and V-cycle for p', FP32 BiCGSTAB inside FP64 refinement for
momentum) and on the plain FP64 Jacobi path.  These sizes span hundreds of
CTAs per solve, so a fault in row partitioning or threads per row that a
small case would not show is caught here."""
import numpy as np
import pytest

import oracle
from gpu_util import ctx, rel_l2
from paper_2106_07616_gb300 import clouds, rbffd

pytestmark = pytest.mark.gpu

PATHS = {"default": (rbffd.PREC_MIXED, rbffd.PRECOND_AMG_FGMRES),
         "fp64_jacobi": (rbffd.PREC_FP64, rbffd.PRECOND_JACOBI)}


def _fields_match(P, O, tol=1e-8):
    for k in ("u", "v", "p"):
        e = rel_l2(P.get(k), O.get(k))
        assert e <= tol, (k, e)


@pytest.fixture(scope="module")
def cavity_oracle():
    """One BDF2 time step of three outer iterations from rest (the oracle
    needs about a minute on the host cores for this)."""
    fp = clouds.cavity(200)
    O = oracle.Problem(fp, krylov_tol=1e-12, krylov_maxit=100000)
    it, change, _ = O.time_step(fp.dt, 1e-30, max_outer=3)
    assert it == 3
    return fp, O, change


@pytest.mark.parametrize("path", list(PATHS))
def test_cavity200_time_step_matches_oracle(cavity_oracle, path):
    fp, O, change = cavity_oracle
    prec, pc = PATHS[path]
    P = rbffd.Problem(ctx(), fp, prec, precond=pc)
    it, cg = P.time_step(fp.dt, 1e-30, max_outer=3, krylov_tol=1e-12, krylov_maxit=100000)
    assert it == 3
    assert abs(cg - change) <= 1e-8 * abs(change), (cg, change)
    _fields_match(P, O)
    P.close()


@pytest.mark.parametrize("path", list(PATHS))
def test_kovasznay50_outer_iterations_match_oracle(path):
    fp = clouds.kovasznay(50, dt=0.4)
    prec, pc = PATHS[path]
    P = rbffd.Problem(ctx(), fp, prec, precond=pc)
    O = oracle.Problem(fp, krylov_tol=1e-12, krylov_maxit=100000)
    for r in range(3):
        dg, sg = P.simple_iterate(fp.dt, krylov_tol=1e-12, krylov_maxit=100000)
        do, so = O.simple_iterate(fp.dt)
        assert max(sg["relres"]) <= 1e-12
        assert abs(dg - do) <= 1e-8 * abs(do), (r, dg, do)
    _fields_match(P, O)
    P.close()


def test_cylinder150k_time_step_matches_oracle():
    """One time step of three outer iterations from the paper's uniform
    stream (outlet, symmetry lines, no-slip cylinder: no pin), default path."""
    fp = clouds.cylinder()
    prec, pc = PATHS["default"]
    P = rbffd.Problem(ctx(), fp, prec, precond=pc)
    O = oracle.Problem(fp, krylov_tol=1e-12, krylov_maxit=100000)
    for k, a in fp.initial.items():
        P.set(k, a)
        O.set(k, a)
    ig, cg = P.time_step(fp.dt, 1e-30, max_outer=3, krylov_tol=1e-12, krylov_maxit=100000)
    io, co, _ = O.time_step(fp.dt, 1e-30, max_outer=3)
    assert ig == io == 3
    assert abs(cg - co) <= 1e-8 * abs(co), (cg, co)
    _fields_match(P, O)
    P.close()
