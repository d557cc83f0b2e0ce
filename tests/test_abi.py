"""The C-ABI library builds, loads and exports every entry point that
include/rbffd.h declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "rbffd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while", "sizeof")))


@pytest.fixture(scope="module")
def lib():
    from paper_2106_07616_gb300 import _build
    path = _build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for must in ("rbffd_build_stencils", "rbffd_weights", "simple_iterate", "solve_steady",
                 "solve_unsteady", "rbffd_problem_create", "rbffd_ctx_create"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_header():
    from paper_2106_07616_gb300 import rbffd
    L = rbffd.load()
    for n in declared_symbols():
        assert getattr(L, n).argtypes is not None, n


def test_host_memory_exhaustion_is_a_status_not_an_exception(tmp_path):
    """No C++ exception crosses the C ABI: with the address space capped
    just above what the process holds, a host-only entry point whose first
    allocation (the 200 MB row-pointer copy of a 50M-row matrix) cannot be
    had returns RBFFD_ENOMEM with its text, and the process lives on.  Runs
    in a child process on one OpenMP thread (no thread is started under the
    cap); no device work."""
    import subprocess
    import sys
    code = r'''
import ctypes as C, resource, sys
import numpy as np
from paper_2106_07616_gb300 import rbffd
L = rbffd.load()
n = 50_000_000
rowptr = np.zeros(n + 1, np.int32)
col = np.zeros(1, np.int32)
val = np.zeros(1)
lv = C.c_int32(0)
rows = (C.c_int32 * rbffd.AMG_MAX_LEVELS)()
nnz = (C.c_int64 * rbffd.AMG_MAX_LEVELS)()
ms = C.c_double(0)
with open("/proc/self/statm") as f:
    held = int(f.read().split()[0]) * resource.getpagesize()
resource.setrlimit(resource.RLIMIT_AS, (held + (96 << 20), resource.RLIM_INFINITY))
rc = L.rbffd_amg_analyze(n, rowptr.ctypes.data, col.ctypes.data, val.ctypes.data,
                         C.byref(lv), rows, nnz, C.byref(ms))
print(rc, L.rbffd_last_error().decode())
'''
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], env=env, cwd=ROOT, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    rc, _, text = r.stdout.strip().splitlines()[-1].partition(" ")
    assert int(rc) == -2 and "host resources exhausted" in text, r.stdout
