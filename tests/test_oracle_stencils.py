"""Pins for the oracle's cloud selection (Sec. 2 clouds; one-sided boundary
clouds, Sec. 3.1) against an independent brute force built on numpy's sort."""
import numpy as np
import pytest

import oracle
from paper_2106_07616_gb300 import clouds


def brute(x, y, q, tag=None):
    n = x.size
    out = np.zeros((n, q), np.int32)
    j = np.arange(n)
    for i in range(n):
        dx = x - x[i]
        dy = y - y[i]
        d2 = dx * dx + dy * dy
        ok = j != i
        if tag is not None and tag[i] != 0:
            ok &= tag == 0
        cand = j[ok]
        order = np.lexsort((cand, d2[ok]))  # primary d2, then index
        out[i, 0] = i
        out[i, 1:] = cand[order[: q - 1]]
    return out


@pytest.mark.parametrize("n,q,seed", [(1, 1, 0), (7, 7, 1), (200, 12, 2), (500, 30, 3)])
def test_knn_random_matches_sort(n, q, seed):
    x, y = clouds.random_cloud(n, seed)
    assert np.array_equal(oracle.knn(x, y, q), brute(x, y, q))


def test_knn_ties_broken_by_index():
    # an unjittered lattice has many exactly equal distances
    s = np.arange(6, dtype=np.float64)
    x, y = np.meshgrid(s, s)
    x, y = x.ravel(), y.ravel()
    idx = oracle.knn(x, y, 9)
    assert np.array_equal(idx, brute(x, y, 9))
    # the centre of a 3x3 block: self, then the 4 axis neighbours by index,
    # then the 4 diagonal neighbours by index
    i = 2 * 6 + 2
    assert list(idx[i]) == [i, i - 6, i - 1, i + 1, i + 6, i - 7, i - 5, i + 5, i + 7]


def test_knn_boundary_clouds_one_sided():
    fp = clouds.kovasznay(12, seed=5)
    idx = oracle.knn(fp.x, fp.y, 20, fp.tag)
    assert np.array_equal(idx, brute(fp.x, fp.y, 20, fp.tag))
    bnd = np.where(fp.tag != 0)[0]
    assert np.all(fp.tag[idx[bnd, 1:]] == 0)
    assert np.all(idx[:, 0] == np.arange(fp.n))


def test_knn_golden_five_points():
    # hand-worked: points on a line at 0, 1, 3, 4, 10 (y = 0)
    x = np.array([0.0, 1.0, 3.0, 4.0, 10.0])
    y = np.zeros(5)
    idx = oracle.knn(x, y, 3)
    # point 2 (x=3): d2 to 1 is 4, to 3 is 1  -> [2, 3, 1]
    # point 1 (x=1): d2 to 0 is 1, to 2 is 4  -> [1, 0, 2]
    # point 4 (x=10): d2 36 (pt 3), 49 (pt 2) -> [4, 3, 2]
    assert idx[2].tolist() == [2, 3, 1]
    assert idx[1].tolist() == [1, 0, 2]
    assert idx[4].tolist() == [4, 3, 2]


def test_knn_rejects_bad_sizes():
    x, y = clouds.random_cloud(5, 0)
    with pytest.raises(ValueError):
        oracle.knn(x, y, 6)


def test_row_subset_matches_full_build():
    """knn_rows / weights_rows (spot checks of large problems) give the rows
    of the full build exactly."""
    fp = clouds.kovasznay(20)
    full = oracle.knn(fp.x, fp.y, 20, fp.tag)
    rows = np.array([0, 5, 77, 212, 399, 19], np.int32)
    sub = oracle.knn_rows(fp.x, fp.y, 20, rows, fp.tag)
    assert np.array_equal(sub, full[rows])
    wf = oracle.weights(fp.x, fp.y, full, 3)
    ws = oracle.weights_rows(fp.x, fp.y, sub, rows, 3)
    for a, b in zip(ws, wf):
        assert np.array_equal(a, b[rows])
