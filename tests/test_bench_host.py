"""Host logic of bench.py (no GPU): the ncu traffic figure is reported only
while the kernel sources hash to the profiled revision, and the roofline
peak falls back to the documented figure without a measured-peaks file."""
import json
import os
import shutil

import pytest

import bench


def _tree(tmp_path):
    """A copy of the profile summaries and kernel sources bench reads."""
    root = tmp_path / "repo"
    shutil.copytree(os.path.join(bench.ROOT, "profiles"), root / "profiles")
    shutil.copytree(os.path.join(bench.ROOT, "paper_2106_07616_gb300", "csrc"),
                    root / "paper_2106_07616_gb300" / "csrc")
    return root


@pytest.mark.parametrize("precond,precision", [("fgmres", "mixed"), ("amg", "fp64"),
                                               ("jacobi", "fp64")])
def test_traffic_follows_the_profiled_sources(tmp_path, monkeypatch, precond, precision):
    root = _tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    name, files = bench.KRYLOV_PROFILES[precond]
    fields = dict(l.split(":", 1) for l in open(root / "profiles" / name)
                  if l.startswith("traffic_bytes_per_launch"))
    got = bench.krylov_traffic(precision, "cavity200", precond)
    # while the sources are the profiled ones, the summary's figure; the
    # sources may have moved on, and then nothing is reported
    assert got is None or got == float(fields["traffic_bytes_per_launch"])
    # any change to a listed source withdraws the figure
    src = root / "paper_2106_07616_gb300" / "csrc" / files[-1]
    src.write_bytes(src.read_bytes() + b"\n// changed\n")
    assert bench.krylov_traffic(precision, "cavity200", precond) is None
    # other workloads have no captured summary
    assert bench.krylov_traffic(precision, "cylinder150k", precond) is None


def test_peak_is_measured_when_present_else_the_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.read_peaks() == (bench.FALLBACK_HBM_GBS, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6792.7}))
    assert bench.read_peaks() == (6792.7, "measured")


def test_batched_workload_follows_its_recipe():
    """The batched workload: Kovasznay and cavity instances on square
    lattices of 1k to 64k points, degree 2..5, q = 2m (m = (k+1)(k+2)/2
    appended monomials), seeded per instance, the same on every call."""
    a = bench.batch_instances(12)
    b = bench.batch_instances(12)
    assert [fp.n for fp in a] == [fp.n for fp in b]
    assert all(np_equal(x.x, y.x) for x, y in zip(a, b))
    kinds = set()
    for fp in a:
        k = fp.degree
        assert 2 <= k <= 5 and fp.q == (k + 1) * (k + 2)
        side = round(fp.n ** 0.5)
        assert side * side == fp.n and 31 * 31 <= fp.n <= 253 * 253, fp.n
        kinds.add(fp.name.rstrip("0123456789"))
    assert len(kinds) == 2, kinds


def np_equal(x, y):
    import numpy as np
    return np.array_equal(x, y)
