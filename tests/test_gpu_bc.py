"""Outlet and symmetry-line boundary rows on the GPU (paper Sec. 3.1)
against the oracle, on the Poiseuille channel."""
import dataclasses

import numpy as np
import pytest

import oracle
from gpu_util import ctx, rel_l2
from paper_2106_07616_gb300 import clouds, rbffd

pytestmark = pytest.mark.gpu


def _vel_err(P, O):
    a = np.concatenate([P.get("u"), P.get("v")])
    b = np.concatenate([O.get("u"), O.get("v")])
    return rel_l2(a, b)


@pytest.mark.parametrize("prec", [rbffd.PREC_FP64, rbffd.PREC_MIXED_FF])
@pytest.mark.parametrize("symmetry", [False, True])
def test_channel_outer_iterations_match_oracle(symmetry, prec):
    fp = clouds.channel(symmetry=symmetry)
    P = rbffd.Problem(ctx(), fp, prec)
    O = oracle.Problem(fp, krylov_tol=1e-12)
    for r in range(3):
        dg, sg = P.simple_iterate(fp.dt, krylov_tol=1e-12)
        do, _ = O.simple_iterate(fp.dt)
        assert max(sg["relres"]) <= 1e-12
        assert abs(dg - do) <= 1e-8 * abs(do), (r, dg, do)
        assert _vel_err(P, O) <= 1e-8
        assert rel_l2(P.get("p"), O.get("p")) <= 1e-8


@pytest.mark.parametrize("symmetry", [False, True])
def test_channel_momentum_rows_match_oracle(symmetry):
    """u~ and v~ matrices (they differ on symmetry lines) applied to a
    random vector after one outer iteration."""
    fp = clouds.channel(symmetry=symmetry)
    P = rbffd.Problem(ctx(), fp)
    O = oracle.Problem(fp, krylov_tol=1e-12)
    P.simple_iterate(fp.dt)
    O.simple_iterate(fp.dt)
    x = np.random.Generator(np.random.PCG64(3)).standard_normal(fp.n)
    for op, name in ((rbffd.OP_MOMENTUM, "mom"), (rbffd.OP_MOMENTUM_V, "momv"),
                     (rbffd.OP_PCORR, "pp")):
        y = np.zeros(fp.n)
        P.apply(op, x, y)
        assert rel_l2(y, O.apply(name, x)) <= 1e-12, name


@pytest.mark.parametrize("symmetry", [False, True])
def test_channel_poiseuille_fixed_point_gpu(symmetry):
    fp = clouds.channel(symmetry=symmetry)
    P = rbffd.Problem(ctx(), fp)
    ex = fp.exact
    for k, a in (("u", ex["u"]), ("un", ex["u"]), ("unm1", ex["u"]), ("v", ex["v"]),
                 ("vn", ex["v"]), ("vnm1", ex["v"]), ("p", ex["p"])):
        P.set(k, a)
    d, _ = P.simple_iterate(fp.dt, krylov_tol=1e-13)
    assert d < 1e-12
    assert np.abs(P.get("u") - ex["u"]).max() < 1e-12
    assert np.abs(P.get("v")).max() < 1e-12
    assert np.abs(P.get("p") - ex["p"]).max() < 1e-10


def test_channel_march_like_oracle():
    """March from rest on the paper's steady error (1e-6): same step count
    as the oracle within one, and the closed form within a few 1e-4."""
    fp = clouds.channel(symmetry=True)
    P = rbffd.Problem(ctx(), fp)
    O = oracle.Problem(fp, krylov_tol=1e-12)
    rc, sg = P.solve_steady(fp.dt, resid_tol=1e-6, max_steps=2000, criterion=1)
    rco, so = O.solve_steady(fp.dt, resid_tol=1e-6, max_steps=2000, criterion=1)
    assert rco == 0
    assert abs(sg["steps"] - so["steps"]) <= 1
    assert _vel_err(P, O) <= 1e-5
    assert np.abs(P.get("u") - fp.exact["u"]).max() < 5e-4
    assert np.abs(P.get("p") - fp.exact["p"]).max() < 3e-3


def test_batch_with_symmetry_member_matches_alone():
    """A member with symmetry lines solves u~ and v~ as two single-RHS
    systems inside the batched launches; results equal the member alone."""
    fps = [clouds.channel(symmetry=True), clouds.kovasznay(30, dt=0.4),
           clouds.channel(symmetry=False, seed=9)]
    alone = [rbffd.Problem(ctx(), fp) for fp in fps]
    for fp, P in zip(fps, alone):
        for _ in range(3):
            P.simple_iterate(fp.dt)
    B = rbffd.Batch(ctx(), [rbffd.Problem(ctx(), fp) for fp in fps])
    for _ in range(3):
        d, its, status = B.iterate([fp.dt for fp in fps])
        assert np.all(status == 0)
    for i in range(len(fps)):
        for k in ("u", "v", "p"):
            e = rel_l2(B.problems[i].get(k), alone[i].get(k))
            assert e <= 1e-8, (i, k, e)
    B.close()


def test_bad_boundary_descriptions_rejected_gpu():
    fp = clouds.channel(symmetry=True)
    tag = fp.tag.copy()
    tag[tag == clouds.TAG_OUTFLOW] = clouds.TAG_DIRICHLET
    bad = [dataclasses.replace(fp, tag=tag)]                     # no level: pin -1, no outlet
    nx = fp.nx.copy()
    nx[np.where(fp.tag == clouds.TAG_SYMMETRY)[0][0]] = 0.5
    bad.append(dataclasses.replace(fp, nx=nx))                  # oblique symmetry normal
    tag = fp.tag.copy()
    tag[0] = 7
    bad.append(dataclasses.replace(fp, tag=tag))                # unknown tag
    bad.append(dataclasses.replace(
        fp, pin=int(np.where(fp.tag == clouds.TAG_OUTFLOW)[0][0])))  # pin at an outlet
    for b in bad:
        with pytest.raises(rbffd.RbffdError) as e:
            rbffd.Problem(ctx(), b)
        assert e.value.code == rbffd.EINVAL
