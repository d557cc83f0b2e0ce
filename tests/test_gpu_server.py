"""The continuous-batching request server: requests of different sizes,
geometries and time steps share the device; each result matches the same
steady solve run alone (to the requested steady tolerance)."""
import numpy as np
import pytest

from gpu_util import rel_l2
from paper_2106_07616_gb300 import _build, clouds, rbffd

pytestmark = pytest.mark.gpu

TOL = 5e-3


def requests():
    return [clouds.kovasznay(30, dt=0.4), clouds.kovasznay(26, seed=4, dt=0.4),
            clouds.kovasznay(34, seed=6, dt=0.4), clouds.cavity(30, seed=9, dt=0.2)]


def solve_alone(ctx, fp):
    P = rbffd.Problem(ctx, fp)
    rc, st = P.solve_steady(fp.dt, resid_tol=TOL, max_steps=3000, check=False)
    return rc, st, P


def test_server_results_match_solves_alone():
    _build.build()
    ctx = rbffd.Context(0)
    S = rbffd.Server(ctx)
    fps = requests()
    tickets = [S.submit(fp, resid_tol=TOL, max_steps=3000) for fp in fps]
    S.drain()
    solo_ctx = rbffd.Context(0)
    for fp, t in zip(fps, tickets):
        r = S.poll(t, fields=True)
        assert r["state"] == 2
        rc, st, P = solve_alone(solo_ctx, fp)
        # a request that fails alone fails in the mix too; which error ends
        # it (steps exhausted, divergence) depends on rounding
        assert (r["status"] == 0) == (rc == 0), (r["status"], rc)
        if rc != 0:
            continue
        assert r["resid"][2] <= TOL and st["resid"][2] <= TOL
        for k in ("u", "v"):
            assert rel_l2(r[k], P.get(k)) <= 20 * TOL, (fp.name, k)
        P.close()
    S.close()


def test_server_mixes_pressure_solvers():
    """Requests with flexible GMRES, multigrid BiCGSTAB and Jacobi p' solvers,
    one with mixed-precision momentum, run in the same batched iterations;
    each result matches the request solved alone with its own solvers."""
    ctx = rbffd.Context(0)
    S = rbffd.Server(ctx)
    fps = requests()
    cfg = [(rbffd.PREC_MIXED, rbffd.PRECOND_AMG_FGMRES), (rbffd.PREC_FP64, rbffd.PRECOND_AMG),
           (rbffd.PREC_FP64, rbffd.PRECOND_AMG_FGMRES), (rbffd.PREC_FP64, rbffd.PRECOND_JACOBI)]
    tickets = [S.submit(fp, resid_tol=TOL, max_steps=3000, precond=pc, precision=pr)
               for fp, (pr, pc) in zip(fps, cfg)]
    S.drain()
    solo_ctx = rbffd.Context(0)
    for fp, (pr, pc), t in zip(fps, cfg, tickets):
        r = S.poll(t, fields=True)
        assert r["state"] == 2
        P = rbffd.Problem(solo_ctx, fp, pr, precond=pc)
        rc, st = P.solve_steady(fp.dt, resid_tol=TOL, max_steps=3000, check=False)
        assert (r["status"] == 0) == (rc == 0), (r["status"], rc)
        if rc == 0:
            assert r["resid"][2] <= TOL and st["resid"][2] <= TOL
            for k in ("u", "v"):
                assert rel_l2(r[k], P.get(k)) <= 20 * TOL, (fp.name, pr, pc, k)
        P.close()
    S.close()


def test_server_admits_by_budget_and_reports_bad_requests():
    ctx = rbffd.Context(0)
    fp = clouds.kovasznay(30, dt=0.4)
    one = rbffd.Problem(ctx, fp).nbytes
    # room for about two problems: the rest must wait in the queue
    S = rbffd.Server(ctx, hbm_budget=int(2.5 * one) + (8 << 20))
    bad = clouds.kovasznay(20)
    bad.q = 5  # fewer cloud points than monomials
    tb = S.submit(bad)
    # identical requests (a cloud known to march to the tolerance)
    ts = [S.submit(clouds.kovasznay(30, dt=0.4), resid_tol=TOL) for i in range(4)]
    S.drain()
    rb = S.poll(tb)
    assert rb["state"] == 2 and rb["status"] == rbffd.EINVAL
    res = [S.poll(t) for t in ts]
    assert all(r["status"] == 0 for r in res), res
    assert max(r["queue_s"] for r in res) > 0.0
    S.close()
