"""Batched outer iterations: many problems, one Krylov launch per solve.
Each member must give the same result in the mix as alone (to the Krylov
tolerance: only the order of the partial sums differs)."""
import numpy as np
import pytest

import oracle
from gpu_util import ctx, rel_l2
from paper_2106_07616_gb300 import clouds, rbffd

pytestmark = pytest.mark.gpu


def members():
    return [clouds.kovasznay(30, dt=0.4), clouds.cavity(40, dt=0.05),
            clouds.kovasznay(30, seed=7, dt=0.4), clouds.cavity(24, seed=3, dt=0.05)]


def test_batch_matches_members_solved_alone():
    fps = members()
    alone = [rbffd.Problem(ctx(), fp) for fp in fps]
    for fp, P in zip(fps, alone):
        for r in range(3):
            P.simple_iterate(fp.dt)
    # all members in one batch, each with its own dt, three outer iterations
    B = rbffd.Batch(ctx(), [rbffd.Problem(ctx(), fp) for fp in fps])
    B.set_autotune(False)  # its iterations run directly: the graph counts below assume none
    for r in range(3):
        d, its, status = B.iterate([fp.dt for fp in fps])
        assert np.all(status == 0)
    for i in range(len(fps)):
        for k in ("u", "v", "p"):
            e = rel_l2(B.problems[i].get(k), alone[i].get(k))
            assert e <= 1e-8, (i, k, e)
    # the first iteration ran directly, the second was captured as a graph,
    # the third replayed it
    captures, replays, kernels = B.graph_stats()
    assert (captures, replays) == (1, 1), (captures, replays)
    assert kernels >= 4 * len(fps) + 2
    B.close()


def test_batch_graph_captured_again_after_a_reload():
    """A reload rebuilds a member (new weights, hierarchy, fields): the next
    batched iteration must not replay the old graph."""
    fps = [clouds.kovasznay(30, dt=0.4), clouds.cavity(24, seed=3, dt=0.05)]
    alone = [rbffd.Problem(ctx(), fp, precond=rbffd.PRECOND_AMG) for fp in fps]
    B = rbffd.Batch(ctx(), [rbffd.Problem(ctx(), fp, precond=rbffd.PRECOND_AMG) for fp in fps])
    B.set_autotune(False)
    dts = [fp.dt for fp in fps]
    for _ in range(2):
        B.iterate(dts)
    for fp, P in zip(fps, alone):
        for _ in range(2):
            P.simple_iterate(fp.dt)
    B.problems[0].reload(fps[0], precond=rbffd.PRECOND_AMG)
    alone[0].reload(fps[0], precond=rbffd.PRECOND_AMG)
    d, its, status = B.iterate(dts)
    assert np.all(status == 0)
    for fp, P in zip(fps, alone):
        P.simple_iterate(fp.dt)
    # iterations 1, 2: direct, captured; after the reload: direct again
    assert B.graph_stats()[:2] == (1, 0)
    d, its, status = B.iterate(dts)
    for fp, P in zip(fps, alone):
        P.simple_iterate(fp.dt)
    assert B.graph_stats()[:2] == (2, 0)
    d, its, status = B.iterate(dts)
    for fp, P in zip(fps, alone):
        P.simple_iterate(fp.dt)
    assert B.graph_stats()[:2] == (2, 1)
    for i in range(len(fps)):
        for k in ("u", "v", "p"):
            e = rel_l2(B.problems[i].get(k), alone[i].get(k))
            assert e <= 1e-8, (i, k, e)
    B.close()


def test_batch_autotuner_keeps_results_and_then_captures():
    """The first nine iterations (one untimed, then four team sizes per launch
    slot, each twice, mirrored order; all run directly) tune the work lists;
    each slot keeps its cheapest.  Results stay those of the
    members solved alone; the iterations after tuning are captured and
    replayed as before."""
    fps = members()
    alone = [rbffd.Problem(ctx(), fp) for fp in fps]
    B = rbffd.Batch(ctx(), [rbffd.Problem(ctx(), fp) for fp in fps])
    for r in range(12):
        d, its, status = B.iterate([fp.dt for fp in fps])
        assert np.all(status == 0)
        for fp, P in zip(fps, alone):
            P.simple_iterate(fp.dt)
        tuned, scales, cost = B.tuning()
        assert tuned == (r >= 8), (r, tuned)
    for i in range(len(fps)):
        for k in ("u", "v", "p"):
            e = rel_l2(B.problems[i].get(k), alone[i].get(k))
            assert e <= 1e-8, (i, k, e)
    # slots 0 (momentum, two right-hand sides) and 2 (p' Jacobi BiCGSTAB)
    # ran: every candidate has a cost, the kept scale is the cheapest
    cand = [1.0, 2.0, 0.5, 4.0]
    for k in (0, 2):
        assert np.all(cost[k] > 0), (k, cost[k])
        assert scales[k] == cand[int(np.argmin(cost[k]))], (k, scales[k], cost[k])
    assert all(s in cand for s in scales)
    # iterations 10 (first of this set), 11 (captured), 12 (replayed)
    assert B.graph_stats()[:2] == (1, 1)
    B.set_autotune(False)
    assert B.tuning()[0] is False and B.tuning()[1] == [1.0] * 9
    B.close()


def test_batch_member_matches_oracle():
    fps = [clouds.kovasznay(30, dt=0.4), clouds.kovasznay(30, seed=5, dt=0.4)]
    B = rbffd.Batch(ctx(), [rbffd.Problem(ctx(), fp) for fp in fps])
    O = [oracle.Problem(fp, krylov_tol=1e-12) for fp in fps]
    for r in range(2):
        d, its, status = B.iterate(0.4)
        for i, o in enumerate(O):
            do, _ = o.simple_iterate(0.4)
            assert abs(d[i] - do) <= 1e-8 * abs(do)
    for i, o in enumerate(O):
        for k in ("u", "v", "p"):
            assert rel_l2(B.problems[i].get(k), o.get(k)) <= 1e-8
    B.close()


def test_batch_active_mask_leaves_others_untouched():
    fps = [clouds.kovasznay(30, dt=0.4), clouds.kovasznay(30, seed=8, dt=0.4)]
    B = rbffd.Batch(ctx(), [rbffd.Problem(ctx(), fp) for fp in fps])
    before = B.problems[1].get("u").copy()
    d, its, status = B.iterate(0.4, active=[1, 0])
    assert np.array_equal(B.problems[1].get("u"), before)
    assert d[0] > 0
    B.close()


def test_batch_many_small_members():
    """More members than SMs: every member gets at least one CTA."""
    fps = [clouds.kovasznay(12 + (i % 5), seed=100 + i, dt=0.05) for i in range(200)]
    probs = [rbffd.Problem(ctx(), fp) for fp in fps]
    B = rbffd.Batch(ctx(), probs)
    d, its, status = B.iterate(0.05)
    assert np.all(status == 0)
    # spot-check a few members against a solo solve
    for i in (0, 57, 199):
        solo = rbffd.Problem(ctx(), fps[i])
        ds, _ = solo.simple_iterate(0.05)
        assert abs(ds - d[i]) <= 1e-8 * abs(ds)
        assert rel_l2(probs[i].get("p"), solo.get("p")) <= 1e-8
    B.close()
