"""Pins for the oracle's right-Jacobi BiCGSTAB (used by the paper for the
momentum and pressure-correction systems, Sec. 3) against a dense solve."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle


def random_system(n, seed, nnz_row=9):
    rng = np.random.default_rng(seed)
    rows = []
    for i in range(n):
        cols = np.unique(np.concatenate([[i], rng.integers(0, n, nnz_row - 1)]))
        vals = rng.standard_normal(cols.size)
        vals[cols == i] = np.abs(vals).sum() + 1.0
        rows.append((cols, vals))
    rowptr = np.zeros(n + 1, np.int64)
    rowptr[1:] = np.cumsum([c.size for c, _ in rows])
    col = np.concatenate([c for c, _ in rows]).astype(np.int32)
    val = np.concatenate([v for _, v in rows])
    return rowptr, col, val


@pytest.mark.parametrize("n,seed", [(1, 0), (10, 1), (200, 2), (500, 3)])
def test_bicgstab_matches_dense(n, seed):
    rowptr, col, val = random_system(n, seed)
    A = sp.csr_matrix((val, col, rowptr), shape=(n, n)).toarray()
    b = np.random.default_rng(seed + 100).standard_normal(n)
    rc, x, it, rr = oracle.bicgstab_csr(rowptr, col, val, b, tol=1e-13)
    assert rc == 0
    ref = np.linalg.solve(A, b)
    assert np.linalg.norm(x - ref) <= 1e-11 * np.linalg.norm(ref)
    assert np.linalg.norm(A @ x - b) <= 1e-12 * np.linalg.norm(b) * 10


def test_bicgstab_zero_rhs_and_exact_guess():
    rowptr, col, val = random_system(50, 4)
    rc, x, it, rr = oracle.bicgstab_csr(rowptr, col, val, np.zeros(50), x0=np.ones(50))
    assert rc == 0 and it == 0 and np.all(x == 0)
    A = sp.csr_matrix((val, col, rowptr), shape=(50, 50))
    xs = np.random.default_rng(5).standard_normal(50)
    rc, x, it, rr = oracle.bicgstab_csr(rowptr, col, val, A @ xs, x0=xs, tol=1e-12)
    assert rc == 0 and it == 0


def test_bicgstab_reports_no_convergence():
    rowptr, col, val = random_system(300, 6)
    b = np.ones(300)
    rc, x, it, rr = oracle.bicgstab_csr(rowptr, col, val, b, tol=1e-14, maxit=2)
    assert rc == oracle.ENOCONV and it == 2
