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


def _fmix32(h):
    """MurmurHash3's 32-bit finaliser (Appleby), written out."""
    h ^= h >> 16
    h = (h * 0x85EBCA6B) & 0xFFFFFFFF
    h ^= h >> 13
    h = (h * 0xC2B2AE35) & 0xFFFFFFFF
    h ^= h >> 16
    return h


def _mis2_aggregates(rowptr, col, val, theta=0.08):
    """Level-0 aggregation from its definition, plain Python: the symmetric
    strength graph; rounds in which every undecided point whose priority is
    the largest among undecided points within distance 2 becomes a root and
    the undecided points within distance 2 of a new root drop out; then
    aggregates numbered by root index, points next to roots joining the root
    of largest priority, the rest the first-pass neighbour of largest
    priority, isolated points as singletons after the roots."""
    n = len(rowptr) - 1
    nb = [set() for _ in range(n)]
    for i in range(n):
        cs, vs = col[rowptr[i]:rowptr[i + 1]], val[rowptr[i]:rowptr[i + 1]]
        off = [abs(v) for c, v in zip(cs, vs) if c != i]
        mx = max(off) if off else 0.0
        for c, v in zip(cs, vs):
            if c != i and mx > 0.0 and abs(v) >= theta * mx:
                nb[i].add(int(c))
                nb[int(c)].add(i)
    key = [((_fmix32(i) << 32) | i) + 1 for i in range(n)]
    state = ["iso" if not nb[i] else "und" for i in range(n)]
    while "und" in state:
        m1 = [max([key[j] for j in nb[i] | {i} if state[j] == "und"], default=0) for i in range(n)]
        m2 = [max(m1[j] for j in nb[i] | {i}) for i in range(n)]
        new = {i for i in range(n) if state[i] == "und" and m2[i] == key[i]}
        near = new | {i for i in range(n) if nb[i] & new}
        near2 = near | {i for i in range(n) if nb[i] & near}
        for i in range(n):
            if i in new:
                state[i] = "root"
            elif state[i] == "und" and i in near2:
                state[i] = "out"
    roots = [i for i in range(n) if state[i] == "root"]
    num = {r: k for k, r in enumerate(roots)}
    first = [num.get(i, -1) for i in range(n)]
    for i in range(n):
        if state[i] == "out":
            rs = [j for j in nb[i] if state[j] == "root"]
            if rs:
                first[i] = num[max(rs, key=lambda j: key[j])]
    agg = list(first)
    for i in range(n):
        if first[i] < 0 and state[i] != "iso":
            cand = [j for j in nb[i] if first[j] >= 0]
            if cand:
                agg[i] = first[max(cand, key=lambda j: key[j])]
    na = len(roots)
    for i in range(n):
        if agg[i] < 0:
            agg[i] = na
            na += 1
    return np.array(agg), na


def test_level0_aggregation_follows_its_definition():
    """The host's level-0 aggregation (the device build gives the same) is
    the MIS(2) aggregation written out above, exactly, on a Laplacian grid
    and on a p' matrix; the aggregates are connected in the strength graph,
    and the priority hash is MurmurHash3's finaliser."""
    assert _fmix32(0) == 0 and _fmix32(1) == 0x514E28B7
    for A in (poisson5(24), p_prime_csr(30)):
        agg, na = rbffd.amg_aggregates_host(*A)
        ref, nr = _mis2_aggregates(*A)
        assert na == nr and np.array_equal(agg, ref), (na, nr)
        assert agg.min() == 0 and agg.max() == na - 1
        # every aggregate is connected in the (symmetric) strength graph
        rowptr, col, val = A
        n = len(rowptr) - 1
        nb = [set() for _ in range(n)]
        for i in range(n):
            cs, vs = col[rowptr[i]:rowptr[i + 1]], val[rowptr[i]:rowptr[i + 1]]
            off = [abs(v) for c, v in zip(cs, vs) if c != i]
            mx = max(off) if off else 0.0
            for c, v in zip(cs, vs):
                if c != i and mx > 0 and abs(v) >= 0.08 * mx:
                    nb[i].add(int(c)); nb[int(c)].add(i)
        for a in range(na):
            mem = set(np.nonzero(agg == a)[0].tolist())
            seen, stack = set(), [next(iter(mem))]
            while stack:
                i = stack.pop()
                if i in seen:
                    continue
                seen.add(i)
                stack.extend(j for j in nb[i] if j in mem)
            assert seen == mem, a
