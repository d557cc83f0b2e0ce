"""Oracle pins for periodic boundaries and the body force (paper Sec. 3.1:
clouds wrap around a periodic boundary; a mean pressure gradient drives
periodic flows)."""
import numpy as np

import oracle
from paper_2106_07616_gb300 import clouds


def test_clouds_wrap_and_derivatives_hold_across_the_seam():
    fp = clouds.periodic_channel()
    O = oracle.Problem(fp)
    ops = O.operators()
    seam = np.where((fp.x < 0.05) & (fp.tag == 0))[0]
    # clouds of points next to x = 0 reach points next to x = L
    assert all((fp.x[ops["idx"][i]] > 0.9).any() for i in seam)
    # d/dx of a periodic function is as accurate next to the seam as
    # anywhere else inside (the wall points' one-sided clouds are coarser)
    k = 2 * np.pi
    f = np.sin(k * fp.x) * (1 + fp.y)
    err = np.abs(O.apply("dx", f) - k * np.cos(k * fp.x) * (1 + fp.y))
    inter = fp.tag == 0
    far = inter & (fp.x > 0.2) & (fp.x < 0.8)
    assert err[inter].max() < 0.01 * k
    assert err[seam].max() < 2 * err[far].max()


def test_force_driven_channel_is_a_fixed_point():
    fp = clouds.periodic_channel()
    O = oracle.Problem(fp, krylov_tol=1e-12)
    for k, f in (("u", "u"), ("un", "u"), ("unm1", "u"), ("v", "v"), ("vn", "v"),
                 ("vnm1", "v"), ("p", "p")):
        O.set(k, fp.exact[f])
    d, _ = O.simple_iterate(fp.dt)
    assert d < 1e-12
    assert np.abs(O.get("u") - fp.exact["u"]).max() < 1e-12
    assert O.steady_residual()[2] < 1e-10


def test_force_driven_channel_from_rest():
    fp = clouds.periodic_channel()
    O = oracle.Problem(fp, krylov_tol=1e-12)
    rc, info = O.solve_steady(fp.dt, resid_tol=1e-6, max_steps=3000, criterion=1)
    assert rc == 0, info
    assert np.abs(O.get("u") - fp.exact["u"]).max() < 2e-3
    assert np.abs(O.get("v")).max() < 2e-3


def test_without_the_force_the_fluid_stays_at_rest():
    import dataclasses
    fp = dataclasses.replace(clouds.periodic_channel(), force=(0.0, 0.0))
    O = oracle.Problem(fp, krylov_tol=1e-12)
    for _ in range(3):
        O.time_step(fp.dt, 1e-4, 20)
    assert np.abs(O.get("u")).max() < 1e-12
