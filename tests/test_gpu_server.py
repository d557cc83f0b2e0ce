"""The continuous-batching request server: requests of different sizes,
geometries and time steps share the device.  With a fixed number of time
steps per request (criterion 2: no steady test, so the march a request
makes does not depend on when it stops) every result must equal the same
march run alone, to the 1e-8 relative L2 the fields are held to, and the
requests must really have overlapped on the device."""
import time

import numpy as np
import pytest

from gpu_util import rel_l2
from paper_2106_07616_gb300 import _build, clouds, rbffd

pytestmark = pytest.mark.gpu

TOL = 5e-3
FIELD_TOL = 1e-8


def requests():
    return [clouds.kovasznay(30, dt=0.1), clouds.kovasznay(26, seed=4, dt=0.1),
            clouds.kovasznay(34, seed=6, dt=0.1), clouds.cavity(30, seed=9, dt=0.05)]


STEPS = [60, 45, 80, 50]


def overlapped(res):
    """Pairs of requests whose admission-to-completion intervals intersect."""
    pairs = 0
    for i in range(len(res)):
        for j in range(i + 1, len(res)):
            a, b = res[i], res[j]
            if a["admit_s"] < b["done_s"] and b["admit_s"] < a["done_s"]:
                pairs += 1
    return pairs


def run_staggered(S, fps, cfg):
    """Submit half the requests, wait until the first one runs, then submit
    the rest while those are on the device."""
    tickets = []
    half = len(fps) // 2
    for k, (fp, (pr, pc)) in enumerate(zip(fps, cfg)):
        if k == half:
            t0 = time.time()
            while S.poll(tickets[0])["state"] < 1 and time.time() - t0 < 60:
                time.sleep(0.005)
            time.sleep(0.02)
        tickets.append(S.submit(fp, resid_tol=0.0, max_steps=STEPS[k], criterion=2,
                                precond=pc, precision=pr))
    S.drain()
    return tickets


def check_against_alone(S, fps, cfg, tickets):
    solo_ctx = rbffd.Context(0)
    res = []
    for k, (fp, (pr, pc), t) in enumerate(zip(fps, cfg, tickets)):
        r = S.poll(t, fields=True)
        assert r["state"] == 2 and r["status"] == 0, (fp.name, r)
        assert r["steps"] == STEPS[k]
        P = rbffd.Problem(solo_ctx, fp, pr, precond=pc)
        rc, st = P.solve_steady(fp.dt, resid_tol=0.0, max_steps=STEPS[k], criterion=2)
        assert st["steps"] == STEPS[k]
        assert r["outer"] == st["outer"], (fp.name, r["outer"], st["outer"])
        for key in ("u", "v", "p"):
            assert rel_l2(r[key], P.get(key)) <= FIELD_TOL, (fp.name, pr, pc, key,
                                                              rel_l2(r[key], P.get(key)))
        P.close()
        res.append(r)
    solo_ctx.close()
    return res


def test_server_results_match_solves_alone():
    _build.build()
    ctx = rbffd.Context(0)
    S = rbffd.Server(ctx)
    fps = requests()
    cfg = [(rbffd.PREC_FP64, rbffd.PRECOND_AMG)] * len(fps)
    tickets = run_staggered(S, fps, cfg)
    res = check_against_alone(S, fps, cfg, tickets)
    # the later half arrived while the first request was running, and the
    # requests' device work overlapped
    assert res[2]["arrive_s"] > res[0]["admit_s"]
    assert overlapped(res) >= 2, [(r["admit_s"], r["done_s"]) for r in res]
    S.close()


def test_server_mixes_pressure_solvers():
    """Requests with flexible GMRES, multigrid BiCGSTAB and Jacobi p' solvers,
    one with mixed-precision momentum, run in the same batched iterations;
    each result equals the request marched alone with its own solvers."""
    ctx = rbffd.Context(0)
    S = rbffd.Server(ctx)
    fps = requests()
    cfg = [(rbffd.PREC_MIXED, rbffd.PRECOND_AMG_FGMRES), (rbffd.PREC_FP64, rbffd.PRECOND_AMG),
           (rbffd.PREC_FP64, rbffd.PRECOND_AMG_FGMRES), (rbffd.PREC_FP64, rbffd.PRECOND_JACOBI)]
    tickets = run_staggered(S, fps, cfg)
    res = check_against_alone(S, fps, cfg, tickets)
    assert overlapped(res) >= 2
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


def test_admission_retries_only_the_hierarchy_upload():
    """A request whose problem fits the budget but whose multigrid hierarchy
    does not (while another request runs) keeps its built problem: only the
    upload is retried until the running request frees its memory, and the
    clouds, weights and operators are built once."""
    probe = rbffd.Context(0)
    small = clouds.kovasznay(50, dt=0.4)
    big = clouds.kovasznay(125, dt=0.4)  # 15 625 rows: the hierarchy is built on the host
    A = rbffd.Problem(probe, small, precond=rbffd.PRECOND_AMG)
    A.amg_info()  # uploads the hierarchy
    full_a = A.nbytes
    B = rbffd.Problem(probe, big, precond=rbffd.PRECOND_AMG)
    base_b = B.nbytes  # before the upload
    B.amg_info()
    hier_b = B.nbytes - base_b
    print("bytes: small", full_a, "big", base_b, "+ hierarchy", hier_b)
    # the big request fits whole once the small one is gone, with half the
    # small one's size to spare for the batch's tables; while the small one
    # runs only the big problem fits, not its hierarchy as well
    assert hier_b > full_a // 2 + (2 << 20), (hier_b, full_a)
    A.close()
    B.close()
    probe.close()
    ctx = rbffd.Context(0)
    S = rbffd.Server(ctx, hbm_budget=base_b + hier_b + full_a // 2)
    ta = S.submit(small, resid_tol=0.0, max_steps=300, criterion=2, precond=rbffd.PRECOND_AMG)
    t0 = time.time()
    while S.poll(ta)["state"] < 1 and time.time() - t0 < 60:
        time.sleep(0.002)
    tb = S.submit(big, resid_tol=0.0, max_steps=3, criterion=2, precond=rbffd.PRECOND_AMG)
    S.drain()
    ra, rb = S.poll(ta), S.poll(tb)
    assert ra["status"] == 0 and rb["status"] == 0, (ra, rb)
    assert ra["builds"] == 1 and rb["builds"] == 1, (ra, rb)
    assert rb["admit_attempts"] >= 2, rb  # the upload waited for the small request
    assert rb["admit_s"] >= ra["done_s"] - 1e-3, (ra, rb)
    S.close()
    ctx.close()
