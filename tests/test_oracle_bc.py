"""Oracle pins for the outlet and symmetry boundary rows (paper Sec. 3.1).

Plane Poiseuille flow is reproduced exactly by weights of degree >= 2
(quadratic velocity, linear pressure), so it is a discrete fixed point of
the outer iteration to roundoff, and marching from rest must approach it.
A wrong outlet or symmetry row (identity instead of zero normal derivative,
pressure not held at the outlet, normal component left free) either breaks
the fixed point, shifts the pressure level or breaks one of the prescribed
values checked below.
"""
import numpy as np
import pytest

import oracle
from paper_2106_07616_gb300 import clouds


def _exact_start(O, fp):
    O.set("u", fp.exact["u"])
    O.set("v", fp.exact["v"])
    O.set("p", fp.exact["p"])
    for k in ("un", "unm1"):
        O.set(k, fp.exact["u"])
    for k in ("vn", "vnm1"):
        O.set(k, fp.exact["v"])


@pytest.mark.parametrize("symmetry", [False, True])
def test_poiseuille_is_a_fixed_point(symmetry):
    fp = clouds.channel(symmetry=symmetry)
    O = oracle.Problem(fp, krylov_tol=1e-12)
    _exact_start(O, fp)
    delta, _ = O.simple_iterate(fp.dt)
    assert delta < 1e-12
    assert np.abs(O.get("u") - fp.exact["u"]).max() < 1e-12
    assert np.abs(O.get("v")).max() < 1e-12
    assert np.abs(O.get("p") - fp.exact["p"]).max() < 1e-10


@pytest.mark.parametrize("symmetry", [False, True])
def test_march_from_rest_reaches_poiseuille(symmetry):
    """Stopping on the paper's steady error (Sec. 4.1) at 1e-6 leaves the
    fields within a few 1e-4 of the closed form, with the pressure level
    set by the outlet (no pin)."""
    fp = clouds.channel(symmetry=symmetry)
    assert fp.pin == -1
    O = oracle.Problem(fp, krylov_tol=1e-12)
    rc, info = O.solve_steady(fp.dt, resid_tol=1e-6, max_steps=2000, criterion=1)
    assert rc == 0, info
    assert np.abs(O.get("u") - fp.exact["u"]).max() < 5e-4
    assert np.abs(O.get("v")).max() < 5e-4
    assert np.abs(O.get("p") - fp.exact["p"]).max() < 3e-3
    assert info["R"] < 1e-4


def test_prescribed_values_hold_during_the_march():
    """Walls and inlet keep u, v; a symmetry line keeps its normal
    component; an outlet keeps its pressure -- after every iteration."""
    fp = clouds.channel(symmetry=True)
    O = oracle.Problem(fp, krylov_tol=1e-12)
    dir_ = fp.tag == clouds.TAG_DIRICHLET
    sym = fp.tag == clouds.TAG_SYMMETRY
    out = fp.tag == clouds.TAG_OUTFLOW
    tol = 1e-4
    for _ in range(5):
        _, change, _ = O.time_step(fp.dt, tol, 20)
        tol = min(1e-4, change)
        u, v, p = O.get("u"), O.get("v"), O.get("p")
        assert np.array_equal(u[dir_], fp.ubc[dir_])
        assert np.array_equal(v[dir_], fp.vbc[dir_])
        assert np.array_equal(v[sym], fp.vbc[sym])
        assert np.array_equal(p[out], np.zeros(out.sum()))
        # the tangential component on the symmetry line and both components
        # at the outlet are free and move off their rest values
        assert np.abs(u[sym]).min() > 0
        assert np.abs(u[out]).min() > 0


def test_bad_boundary_descriptions_rejected():
    fp = clouds.channel(symmetry=True)
    # no outlet and no pin: the pressure level is undefined
    tag = fp.tag.copy()
    tag[tag == clouds.TAG_OUTFLOW] = clouds.TAG_DIRICHLET
    with pytest.raises(ValueError):
        oracle.Problem(_with(fp, tag=tag))
    # a symmetry point with an oblique normal
    nx = fp.nx.copy()
    nx[np.where(fp.tag == clouds.TAG_SYMMETRY)[0][0]] = 0.5
    with pytest.raises(ValueError):
        oracle.Problem(_with(fp, nx=nx))
    # an unknown tag
    tag = fp.tag.copy()
    tag[0] = 7
    with pytest.raises(ValueError):
        oracle.Problem(_with(fp, tag=tag))


def _with(fp, **kw):
    import dataclasses
    return dataclasses.replace(fp, **kw)
