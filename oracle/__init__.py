"""CPU oracle for the semi-implicit PHS-RBF-FD method (TEST INFRASTRUCTURE).

A plain, slow FP64 C implementation (``rbffd_oracle.c``) loaded through
ctypes.  Only the tests, the smoke check and the benchmark's CPU-baseline
leg may import this package; the product library never does.  It shares no
code with the CUDA path.

Parity pins: every function here is checked in ``tests/test_oracle_*.py``
against closed forms, invariants and brute force, never against itself.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rbffd_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

FIELDS = {"u": 0, "v": 1, "p": 2, "un": 3, "vn": 4, "unm1": 5, "vnm1": 6, "ut": 7, "vt": 8,
          "pc": 9, "ubc": 10, "vbc": 11}
OK, EINVAL, ENOMEM, ESINGULAR, ENOCONV, EDIVERGED = 0, -1, -2, -3, -4, -5


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no contraction, OpenMP over points)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
           "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_lp = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_bp = np.ctypeslib.ndpointer(dtype=np.int8, flags="C_CONTIGUOUS")


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        L.orc_knn.argtypes = [C.c_int, _dp, _dp, C.c_void_p, C.c_int, _ip]
        L.orc_weights.argtypes = [C.c_int, _dp, _dp, C.c_int, _ip, C.c_int, _dp, _dp, _dp,
                                  C.POINTER(C.c_int32)]
        L.orc_knn_rows.argtypes = [C.c_int, _dp, _dp, C.c_void_p, C.c_int, C.c_int, _ip, _ip]
        L.orc_weights_rows.argtypes = [C.c_int, _dp, _dp, C.c_int, C.c_int, _ip, _ip, C.c_int,
                                       _dp, _dp, _dp, C.POINTER(C.c_int32)]
        L.orc_lu_solve.argtypes = [C.c_int, C.c_int, _dp, C.c_int, _dp]
        L.orc_bicgstab_csr.argtypes = [C.c_int, _lp, _ip, _dp, _dp, _dp, C.c_double, C.c_int,
                                       C.POINTER(C.c_int32), C.POINTER(C.c_double)]
        L.orc_problem_create.argtypes = [C.c_int, C.c_int, C.c_int, _dp, _dp, _bp, _dp, _dp, _dp,
                                         _dp, C.c_int, C.c_double, C.c_double,
                                         C.POINTER(C.c_void_p), C.POINTER(C.c_int32)]
        L.orc_problem_create2.argtypes = [C.c_int, C.c_int, C.c_int, _dp, _dp, _bp, _dp, _dp,
                                          _dp, _dp, C.c_int, C.c_double, C.c_double, _dp, _dp,
                                          C.POINTER(C.c_void_p), C.POINTER(C.c_int32)]
        L.orc_problem_destroy.argtypes = [C.c_void_p]
        L.orc_courant.argtypes = [C.c_void_p, C.c_double, C.c_int, _dp]
        L.orc_get_field.argtypes = [C.c_void_p, C.c_int, _dp]
        L.orc_set_field.argtypes = [C.c_void_p, C.c_int, _dp]
        L.orc_get_operators.argtypes = [C.c_void_p, _ip, _dp, _dp, _dp, _dp]
        L.orc_set_krylov.argtypes = [C.c_void_p, C.c_double, C.c_int]
        L.orc_simple_iterate.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_double,
                                         C.c_double, C.POINTER(C.c_double), _dp]
        L.orc_time_step.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_int,
                                    C.POINTER(C.c_int32), C.POINTER(C.c_double),
                                    C.POINTER(C.c_double)]
        L.orc_steady_residual.argtypes = [C.c_void_p, _dp]
        L.orc_solve_steady.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_int, C.c_int,
                                       _dp]
        L.orc_solve_steady_c.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_int, C.c_int,
                                         C.c_int, _dp]
        L.orc_solve_unsteady.argtypes = [C.c_void_p, C.c_double, C.c_int, C.c_int, _dp]
        L.orc_apply.argtypes = [C.c_void_p, C.c_int, _dp, _dp]
        L.orc_get_compat.argtypes = [C.c_void_p, _dp]
        L.orc_set_compat.argtypes = [C.c_void_p, C.c_int]
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_set_threads.restype = C.c_int
        L.orc_monomial_exponents.argtypes = [C.c_int, _ip, _ip]
        _lib = L
    return _lib


def set_threads(n: int) -> int:
    """Host threads for the per-point loops; returns the count in use."""
    return lib().orc_set_threads(int(n))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def monomial_exponents(degree):
    m = (degree + 1) * (degree + 2) // 2
    ax = np.zeros(m, np.int32)
    ay = np.zeros(m, np.int32)
    lib().orc_monomial_exponents(degree, ax, ay)
    return ax, ay


def knn(x, y, q, tag=None):
    """Stencils: (n, q) int32, self first, then (d^2, index) ascending;
    boundary points (tag != 0) draw their other members from interior points."""
    x, y = _f64(x), _f64(y)
    idx = np.zeros((x.size, q), np.int32)
    tg = None if tag is None else np.ascontiguousarray(tag, np.int8)
    rc = lib().orc_knn(x.size, x, y, None if tg is None else tg.ctypes.data, q, idx)
    if rc:
        raise ValueError(f"orc_knn failed: {rc}")
    return idx


def knn_rows(x, y, q, rows, tag=None):
    """Stencils of the points `rows` only: (len(rows), q), as knn()."""
    x, y = _f64(x), _f64(y)
    rows = np.ascontiguousarray(rows, np.int32)
    idx = np.zeros((rows.size, q), np.int32)
    tg = None if tag is None else np.ascontiguousarray(tag, np.int8)
    rc = lib().orc_knn_rows(x.size, x, y, None if tg is None else tg.ctypes.data, q, rows.size,
                            rows, idx)
    if rc:
        raise ValueError(f"orc_knn_rows failed: {rc}")
    return idx


def weights_rows(x, y, idx, rows, degree):
    """Weights of the clouds idx (len(rows), q) centred at the points rows."""
    x, y = _f64(x), _f64(y)
    idx = np.ascontiguousarray(idx, np.int32)
    rows = np.ascontiguousarray(rows, np.int32)
    k, q = idx.shape
    wx, wy, wl = np.zeros((k, q)), np.zeros((k, q)), np.zeros((k, q))
    fs = C.c_int32(-1)
    rc = lib().orc_weights_rows(x.size, x, y, q, k, rows, idx, degree, wx, wy, wl, C.byref(fs))
    if rc:
        raise ValueError(f"orc_weights_rows failed: {rc} (first singular {fs.value})")
    return wx, wy, wl


def weights(x, y, idx, degree):
    """Operator weights (wx, wy, wl), each (n, q); raises on a singular cloud."""
    x, y = _f64(x), _f64(y)
    idx = np.ascontiguousarray(idx, np.int32)
    n, q = idx.shape
    wx = np.zeros((n, q))
    wy = np.zeros((n, q))
    wl = np.zeros((n, q))
    fs = C.c_int32(-1)
    rc = lib().orc_weights(n, x, y, q, idx, degree, wx, wy, wl, C.byref(fs))
    if rc:
        raise ValueError(f"orc_weights failed: {rc} (first singular {fs.value})")
    return wx, wy, wl


def lu_solve(A, B):
    """Solve A X = B with the oracle's LU (A n x n, B n x nr)."""
    A = np.asarray(A, np.float64)
    B = np.asarray(B, np.float64).reshape(A.shape[0], -1)
    n, nr = B.shape
    M = np.ascontiguousarray(np.hstack([A, B]))
    sol = np.zeros(n * nr)
    rc = lib().orc_lu_solve(n, nr, M, n + nr, sol)
    if rc:
        raise ValueError("singular")
    return sol.reshape(nr, n).T


def bicgstab_csr(rowptr, col, val, b, x0=None, tol=1e-12, maxit=10000):
    b = _f64(b)
    x = np.zeros_like(b) if x0 is None else _f64(x0).copy()
    it = C.c_int32(0)
    rr = C.c_double(0)
    rc = lib().orc_bicgstab_csr(b.size, np.ascontiguousarray(rowptr, np.int64),
                                np.ascontiguousarray(col, np.int32), _f64(val), b, x, tol, maxit,
                                C.byref(it), C.byref(rr))
    return rc, x, it.value, rr.value


class Problem:
    """The oracle's flow problem: stencils, weights, operators and fields."""

    def __init__(self, fp, krylov_tol=1e-12, krylov_maxit=10000):
        self.n, self.q = fp.n, fp.q
        self.fp = fp
        h = C.c_void_p()
        fs = C.c_int32(-1)
        per = np.array(getattr(fp, "period", (0.0, 0.0)), np.float64)
        force = np.array(getattr(fp, "force", (0.0, 0.0)), np.float64)
        rc = lib().orc_problem_create2(
            fp.n, fp.q, fp.degree, _f64(fp.x), _f64(fp.y),
            np.ascontiguousarray(fp.tag, np.int8), _f64(fp.nx), _f64(fp.ny), _f64(fp.ubc),
            _f64(fp.vbc), int(fp.pin), float(fp.rho), float(fp.mu), per, force, C.byref(h),
            C.byref(fs))
        if rc:
            raise ValueError(f"orc_problem_create failed: {rc} (first singular {fs.value})")
        self.h = h
        lib().orc_set_krylov(h, krylov_tol, krylov_maxit)

    def __del__(self):
        if getattr(self, "h", None) is not None and _lib is not None:
            _lib.orc_problem_destroy(self.h)
            self.h = None

    def get(self, name):
        out = np.zeros(self.n)
        lib().orc_get_field(self.h, FIELDS[name], out)
        return out

    def set(self, name, arr):
        lib().orc_set_field(self.h, FIELDS[name], _f64(arr))

    def operators(self):
        n, q = self.n, self.q
        idx = np.zeros((n, q), np.int32)
        wx, wy, wl, pv = (np.zeros((n, q)) for _ in range(4))
        lib().orc_get_operators(self.h, idx, wx, wy, wl, pv)
        return {"idx": idx, "wx": wx, "wy": wy, "wl": wl, "pval": pv}

    def apply(self, which, x):
        y = np.zeros(self.n)
        lib().orc_apply(self.h, {"dx": 0, "dy": 1, "lap": 2, "pp": 3, "mom": 4, "momv": 5}[which], _f64(x), y)
        return y

    def simple_iterate(self, dt, alpha=(1.5, -2.0, 0.5)):
        d = C.c_double(0)
        st = np.zeros(6)
        rc = lib().orc_simple_iterate(self.h, dt, *alpha, C.byref(d), st)
        if rc:
            raise RuntimeError(f"orc_simple_iterate failed: {rc}")
        return d.value, st

    def time_step(self, dt, tol_outer, max_outer=20):
        it = C.c_int32(0)
        ch = C.c_double(0)
        last = C.c_double(0)
        rc = lib().orc_time_step(self.h, dt, tol_outer, max_outer, C.byref(it), C.byref(ch),
                                 C.byref(last))
        if rc:
            raise RuntimeError(f"orc_time_step failed: {rc}")
        return it.value, ch.value, last.value

    def courant(self, dt, iters=200):
        """(lambda, lambda dt / 2) of the convection-diffusion operator."""
        out = np.zeros(2)
        rc = lib().orc_courant(self.h, dt, iters, out)
        if rc:
            raise RuntimeError(f"orc_courant failed: {rc}")
        return out[0], out[1]

    def steady_residual(self):
        """(R_m, R_c, R, lambda): lambda is the mean interior divergence, the
        constant that the compatible p' equation leaves in continuity."""
        r = np.zeros(4)
        lib().orc_steady_residual(self.h, r)
        return r

    def set_compat(self, on):
        """Switch the compatible p' source on or off (off plants the plain pin)."""
        rc = lib().orc_set_compat(self.h, int(bool(on)))
        if rc:
            raise ValueError("no compatibility on a problem with an outlet")

    def compat(self):
        """The left null vector psi of the pure-Neumann p' operator (None
        when an outlet fixes the pressure level)."""
        out = np.zeros(self.n)
        rc = lib().orc_get_compat(self.h, out)
        return None if rc else out

    def solve_steady(self, dt, resid_tol=1e-8, max_steps=10000, max_outer=20, criterion=0):
        out = np.zeros(4)
        rc = lib().orc_solve_steady_c(self.h, dt, resid_tol, max_steps, max_outer, criterion, out)
        return rc, {"steps": int(out[0]), "outer": int(out[1]), "R": out[2], "change": out[3]}

    def solve_unsteady(self, dt, n_steps, max_outer=20):
        out = np.zeros(4)
        rc = lib().orc_solve_unsteady(self.h, dt, n_steps, max_outer, out)
        return rc, {"steps": int(out[0]), "outer": int(out[1]), "change": out[3]}
