"""The seeded cylinder cloud (flow past a cylinder, paper Sec. 5.1): point
count, boundary tagging, normals and spacing grading."""
import numpy as np
import pytest

from paper_2106_07616_gb300 import clouds


@pytest.fixture(scope="module")
def cyl():
    return clouds.cylinder()


def test_count_and_grading(cyl):
    assert abs(cyl.n - 150_000) <= 3000
    from scipy.spatial import cKDTree
    d, _ = cKDTree(np.c_[cyl.x, cyl.y]).query(np.c_[cyl.x, cyl.y], k=2)
    nn = d[:, 1]
    r = np.hypot(cyl.x, cyl.y)
    assert nn.min() > 0.5 * 0.02  # no near-duplicates
    near, far = np.median(nn[r < 0.7]), np.median(nn[r > 12])
    assert 0.015 < near < 0.025 and far > 2.5 * near


def test_boundary_tags_values_and_normals(cyl):
    x, y, t = cyl.x, cyl.y, cyl.tag
    r = np.hypot(x, y)
    wall = (t == clouds.TAG_DIRICHLET) & (r < 0.75)
    inlet = (t == clouds.TAG_DIRICHLET) & (r >= 0.75)
    assert np.allclose(r[wall], 0.5) and wall.sum() == round(2 * np.pi * 0.5 / 0.02)
    assert np.all(x[inlet] == -5.0)
    assert np.all(cyl.ubc[inlet] == 1.0) and np.all(cyl.ubc[wall] == 0.0)
    assert np.all(cyl.vbc == 0.0)
    assert np.all(x[t == clouds.TAG_OUTFLOW] == 15.0)
    assert np.all(np.abs(y[t == clouds.TAG_SYMMETRY]) == 5.0)
    # outward normals: unit, out of the fluid (into the cylinder on its wall)
    bnd = t != clouds.TAG_INTERIOR
    assert np.allclose(np.hypot(cyl.nx[bnd], cyl.ny[bnd]), 1.0)
    assert np.allclose(cyl.nx[wall], -x[wall] / 0.5) and np.allclose(cyl.ny[wall], -y[wall] / 0.5)
    sym = t == clouds.TAG_SYMMETRY
    assert np.all(cyl.ny[sym] == np.sign(y[sym])) and np.all(cyl.nx[sym] == 0.0)
    # interior points strictly inside the box and outside the cylinder
    i = t == clouds.TAG_INTERIOR
    assert np.all((x[i] > -5) & (x[i] < 15) & (np.abs(y[i]) < 5) & (r[i] > 0.5))
    assert cyl.pin == -1


def test_seeded_and_small_variant():
    a = clouds.cylinder(5000, h0=0.1, hmax=0.5)
    b = clouds.cylinder(5000, h0=0.1, hmax=0.5)
    assert np.array_equal(a.x, b.x) and abs(a.n - 5000) <= 100
    with pytest.raises(ValueError):
        clouds.cylinder(5000)  # h0 = 0.02 cannot be graded down to 5000 points
