"""Pins for the oracle's PHS r^3 + polynomial operator weights (Sec. 2,
Eqs. RBF_interp .. RBF_interp_mat_vec_L_solve)."""
import math

import numpy as np
import pytest

import oracle
from paper_2106_07616_gb300 import clouds


def monomials(x, y, degree):
    """Columns x^a y^b in graded order, x power descending inside a degree."""
    cols, dcols, ecols, lcols = [], [], [], []
    for d in range(degree + 1):
        for a in range(d, -1, -1):
            b = d - a
            cols.append((a, b))
    return cols


def eval_mono(a, b, x, y):
    return x ** a * y ** b


def lop(a, b, x, y, op):
    if op == "x":
        return a * x ** max(a - 1, 0) * y ** b if a > 0 else 0.0 * x
    if op == "y":
        return b * x ** a * y ** max(b - 1, 0) if b > 0 else 0.0 * x
    t = 0.0 * x
    if a >= 2:
        t = t + a * (a - 1) * x ** (a - 2) * y ** b
    if b >= 2:
        t = t + b * (b - 1) * x ** a * y ** (b - 2)
    return t


@pytest.mark.parametrize("degree,q", [(1, 6), (2, 12), (3, 20), (4, 30), (5, 42), (6, 56)])
def test_polynomial_reproduction(degree, q):
    """sum_j w_j P(x_j) = L P(x_c) for every appended monomial: the
    constraint rows of Eq. (RBF_interp_mat_vec) make this exact."""
    x, y = clouds.jittered_grid(14, seed=degree)
    idx = oracle.knn(x, y, q)
    wx, wy, wl = oracle.weights(x, y, idx, degree)
    h = 1.0 / 13
    for (a, b) in monomials(x, y, degree):
        # shift to the centre so the monomials stay O(h^d) in each cloud
        for i in range(0, x.size, 7):
            xc, yc = x[i], y[i]
            xs, ys = x[idx[i]] - xc, y[idx[i]] - yc
            pv = eval_mono(a, b, xs, ys)
            scale = h ** (a + b)
            for w, op, s in ((wx[i], "x", h), (wy[i], "y", h), (wl[i], "l", h * h)):
                want = float(lop(a, b, np.zeros(1), np.zeros(1), op)[0])
                got = float(w @ pv)
                assert abs(got - want) <= 1e-8 * scale / s + 1e-9, (a, b, op, i, got, want)


def test_row_sums_vanish():
    x, y = clouds.jittered_grid(12, seed=3)
    idx = oracle.knn(x, y, 20)
    wx, wy, wl = oracle.weights(x, y, idx, 3)
    h = 1.0 / 11
    assert np.abs(wx.sum(1)).max() < 1e-9 / h
    assert np.abs(wy.sum(1)).max() < 1e-9 / h
    assert np.abs(wl.sum(1)).max() < 1e-8 / h ** 2


@pytest.mark.parametrize("degree", [1, 2, 3])
def test_q_equals_m_is_polynomial_differentiation(degree):
    """With q = m the constraints P^T lambda = 0 force lambda = 0 (P square
    and invertible), so the weights solve P^T w = L P(x_c) alone."""
    m = (degree + 1) * (degree + 2) // 2
    x, y = clouds.random_cloud(60, seed=10 + degree)
    idx = oracle.knn(x, y, m)
    wx, wy, wl = oracle.weights(x, y, idx, degree)
    cols = monomials(x, y, degree)
    for i in range(0, 60, 5):
        xs, ys = x[idx[i]] - x[i], y[idx[i]] - y[i]
        Pm = np.stack([eval_mono(a, b, xs, ys) for (a, b) in cols], axis=1)  # q x m
        for w, op in ((wx[i], "x"), (wy[i], "y"), (wl[i], "l")):
            rhs = np.array([float(lop(a, b, np.zeros(1), np.zeros(1), op)[0]) for (a, b) in cols])
            ref = np.linalg.solve(Pm.T, rhs)
            assert np.allclose(w, ref, rtol=1e-7, atol=1e-8 * max(1.0, np.abs(ref).max()))


def _smooth(x, y):
    f = np.sin(1.7 * x + 0.3) * np.cos(1.3 * y - 0.2)
    fx = 1.7 * np.cos(1.7 * x + 0.3) * np.cos(1.3 * y - 0.2)
    fy = -1.3 * np.sin(1.7 * x + 0.3) * np.sin(1.3 * y - 0.2)
    fl = -(1.7 ** 2 + 1.3 ** 2) * f
    return f, fx, fy, fl


@pytest.mark.parametrize("degree,q", [(2, 12), (3, 20), (4, 30)])
def test_refinement_orders(degree, q):
    """Errors of d/dx and the Laplacian fall as h^k and h^(k-1) (the orders
    the paper quotes for a polynomial degree k)."""
    ex, el, hs = [], [], []
    for ns in (16, 32, 64):
        x, y = clouds.jittered_grid(ns, seed=7)
        idx = oracle.knn(x, y, q)
        wx, wy, wl = oracle.weights(x, y, idx, degree)
        f, fx, fy, fl = _smooth(x, y)
        inner = (x > 0.25) & (x < 0.75) & (y > 0.25) & (y < 0.75)
        ex.append(np.abs((wx * f[idx]).sum(1) - fx)[inner].max())
        el.append(np.abs((wl * f[idx]).sum(1) - fl)[inner].max())
        hs.append(1.0 / (ns - 1))
    sx = np.polyfit(np.log(hs), np.log(ex), 1)[0]
    sl = np.polyfit(np.log(hs), np.log(el), 1)[0]
    assert sx > degree - 0.6, (sx, ex)
    assert sl > degree - 1 - 0.6, (sl, el)


def test_singular_cloud_reported():
    x, y = clouds.random_cloud(40, seed=1)
    x[5], y[5] = x[9], y[9]  # duplicate point -> zero pivot
    idx = oracle.knn(x, y, 12)
    with pytest.raises(ValueError, match="first singular"):
        oracle.weights(x, y, idx, 2)


def test_lu_matches_numpy_and_pivots():
    rng = np.random.default_rng(0)
    for n in (1, 2, 5, 30, 63):
        A = rng.standard_normal((n, n)) + n * np.eye(n) * 0.1
        B = rng.standard_normal((n, 3))
        X = oracle.lu_solve(A, B)
        assert np.allclose(X, np.linalg.solve(A, B), rtol=1e-9, atol=1e-10)
    # a zero leading entry needs a row swap
    A = np.array([[0.0, 1.0], [2.0, 3.0]])
    assert np.allclose(oracle.lu_solve(A, np.array([1.0, 8.0])).ravel(), [2.5, 1.0])
    with pytest.raises(ValueError):
        oracle.lu_solve(np.array([[1.0, 2.0], [2.0, 4.0]]), np.array([1.0, 1.0]))
