"""Host part of the multigrid preconditioner (rbffd_amg_analyze): the
hierarchy build runs on the CPU, no GPU needed.  Its operators are checked
on the GPU by the preconditioned solves (tests/test_gpu_amg.py); here the
structure: coarsening, determinism, argument checks."""
import numpy as np
import pytest

import oracle
from paper_2106_07616_gb300 import _build, clouds, rbffd


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()


def poisson5(m):
    """5-point Laplacian on an m x m grid with identity rows on the edge."""
    n = m * m
    rows, cols, vals = [], [], []
    for j in range(m):
        for i in range(m):
            r = j * m + i
            if i in (0, m - 1) or j in (0, m - 1):
                rows.append(r); cols.append(r); vals.append(1.0)
                continue
            for di, dj, v in ((0, 0, -4.0), (1, 0, 1.0), (-1, 0, 1.0), (0, 1, 1.0), (0, -1, 1.0)):
                rows.append(r); cols.append((j + dj) * m + i + di); vals.append(v)
    order = np.lexsort((np.arange(len(rows)), rows))
    rows, cols, vals = np.array(rows)[order], np.array(cols)[order], np.array(vals)[order]
    rowptr = np.searchsorted(rows, np.arange(n + 1))
    return rowptr, cols, vals


def test_poisson_hierarchy_coarsens_to_a_dense_level():
    levels, ms = rbffd.amg_analyze(*poisson5(64))
    sizes = [n for n, _ in levels]
    assert sizes[0] == 64 * 64
    assert all(b < a / 3 for a, b in zip(sizes, sizes[1:]))  # aggregates of >3 points
    assert sizes[-1] <= 200 and len(sizes) >= 3
    assert ms >= 0.0


def test_hierarchy_is_deterministic_on_a_p_prime_matrix():
    fp = clouds.cavity(60, dt=0.05)
    O = oracle.Problem(fp)
    ops = O.operators()
    pv, idx = ops["pval"], ops["idx"]
    keep = (pv != 0) | (idx == np.arange(fp.n)[:, None])
    rowptr = np.concatenate([[0], np.cumsum(keep.sum(1))])
    a = rbffd.amg_analyze(rowptr, idx[keep], pv[keep])[0]
    b = rbffd.amg_analyze(rowptr, idx[keep], pv[keep])[0]
    assert a == b and len(a) >= 2 and a[-1][0] <= 600


def test_bad_csr_rejected():
    rowptr, cols, vals = poisson5(8)
    bad = cols.copy()
    bad[3] = 10_000
    with pytest.raises(rbffd.RbffdError) as e:
        rbffd.amg_analyze(rowptr, bad, vals)
    assert e.value.code == rbffd.EINVAL


def test_hierarchy_does_not_depend_on_the_thread_count(tmp_path):
    """Loops run in parallel only above a work threshold and with row chunks
    sized to the thread count; the hierarchy is the same on one thread and
    on four.  The 80 x 80 cavity's p' matrix (192 000 entries) crosses the
    threshold on level 0 and not on the coarse levels."""
    import json
    import os
    import subprocess
    import sys
    fp = clouds.cavity(80, dt=0.05)
    ops = oracle.Problem(fp).operators()
    pv, idx = ops["pval"], ops["idx"]
    keep = (pv != 0) | (idx == np.arange(fp.n)[:, None])
    rowptr = np.concatenate([[0], np.cumsum(keep.sum(1))])
    path = tmp_path / "pp.npz"
    np.savez(path, rowptr=rowptr, col=idx[keep], val=pv[keep])
    code = ("import json, sys, numpy as np\n"
            "from paper_2106_07616_gb300 import rbffd\n"
            "d = np.load(sys.argv[1])\n"
            "print(json.dumps(rbffd.amg_analyze(d['rowptr'], d['col'], d['val'])[0]))\n")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = []
    for threads in ("1", "4"):
        env = dict(os.environ, OMP_NUM_THREADS=threads)
        r = subprocess.run([sys.executable, "-c", code, str(path)], env=env, cwd=root,
                           capture_output=True, text=True, timeout=300)
        assert r.returncode == 0, r.stderr
        out.append(json.loads(r.stdout.strip().splitlines()[-1]))
    assert out[0] == out[1] and len(out[0]) >= 2 and out[0][0][1] > (1 << 17)


def p_prime_csr(m):
    fp = clouds.cavity(m, dt=0.05)
    ops = oracle.Problem(fp).operators()
    pv, idx = ops["pval"], ops["idx"]
    keep = (pv != 0) | (idx == np.arange(fp.n)[:, None])
    rowptr = np.concatenate([[0], np.cumsum(keep.sum(1))])
    return rowptr, idx[keep], pv[keep]


@pytest.mark.parametrize("which", ["cavity120", "poisson64"])
def test_composed_cycle_equals_the_level_by_level_cycle(which):
    """The folded V-cycle regrouped into three phases (restriction straight
    from level 0 to every coarse level, all corrections prolonged to level 1
    together) is the same linear map: both forms, applied on the host in
    FP64 to random right-hand sides, agree to rounding."""
    A = p_prime_csr(120) if which == "cavity120" else poisson5(64)
    n = A[0].size - 1
    levels = rbffd.amg_analyze(*A)[0]
    assert len(levels) >= 3
    rng = np.random.default_rng(5)
    for _ in range(3):
        b = rng.standard_normal(n)
        yl, yc, nc, chunks = rbffd.amg_cycle_host(*A, b)
        assert nc == sum(r for r, _ in levels[2:])  # levels 2 .. L-1 stacked
        assert chunks >= nc
        assert np.linalg.norm(yl) > 0
        assert np.linalg.norm(yc - yl) <= 1e-12 * np.linalg.norm(yl)
    # linear: the cycle of a combination is the combination of the cycles
    b1, b2 = rng.standard_normal(n), rng.standard_normal(n)
    y1 = rbffd.amg_cycle_host(*A, b1)[1]
    y2 = rbffd.amg_cycle_host(*A, b2)[1]
    y12 = rbffd.amg_cycle_host(*A, 2.0 * b1 - 3.0 * b2)[1]
    assert np.linalg.norm(y12 - (2.0 * y1 - 3.0 * y2)) <= 1e-12 * np.linalg.norm(y12)


def test_composed_cycle_not_built_for_two_levels_or_fewer():
    A = poisson5(8)  # 64 rows: the coarsest level at once
    assert len(rbffd.amg_analyze(*A)[0]) == 1
    b = np.random.default_rng(1).standard_normal(64)
    yl, yc, nc, chunks = rbffd.amg_cycle_host(*A, b)
    assert nc == 0 and chunks == 0 and not yc.any()
    # one level: the cycle is the dense inverse
    rowptr, col, val = A
    M = np.zeros((64, 64))
    for i in range(64):
        M[i, col[rowptr[i]:rowptr[i + 1]]] += val[rowptr[i]:rowptr[i + 1]]
    assert np.allclose(yl, np.linalg.solve(M, b), rtol=1e-10, atol=1e-12)
