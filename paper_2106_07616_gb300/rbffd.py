"""Thin ctypes binding of ``librbffd.so`` (argument marshalling only).

Every step of the method runs in the library's CUDA kernels; this module
only converts Python arguments into the pointers and sizes of the C ABI
declared in ``include/rbffd.h`` and raises ``RbffdError`` on a non-zero
status.  Device buffers are torch CUDA tensors (PyTorch supplies device
memory and streams); host buffers are numpy arrays.  There is no CPU
fallback: if the library is missing or was not built, loading fails.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librbffd.so")

OK, EINVAL, ENOMEM, ESINGULAR, ENOCONV, EDIVERGED, ETIMEOUT, ECUDA, ENOTIMPL = (
    0, -1, -2, -3, -4, -5, -6, -7, -8)
OP_DX, OP_DY, OP_LAP, OP_PCORR, OP_MOMENTUM, OP_MOMENTUM_V = 0, 1, 2, 3, 4, 5
TAG_INTERIOR, TAG_DIRICHLET, TAG_OUTFLOW, TAG_SYMMETRY = 0, 1, 2, 3
FIELDS = {"u": 0, "v": 1, "p": 2, "un": 3, "vn": 4, "unm1": 5, "vnm1": 6, "ut": 7, "vt": 8,
          "pc": 9, "ubc": 10, "vbc": 11}
PREC_FP64, PREC_MIXED, PREC_MIXED_FF = 0, 1, 2
PRECOND_JACOBI, PRECOND_AMG, PRECOND_AMG_FGMRES = 0, 1, 2
AMG_MAX_LEVELS = 10


class RbffdError(RuntimeError):
    def __init__(self, code, where, detail):
        super().__init__(f"{where} failed with status {code}: {detail}")
        self.code = code


class ProblemDesc(C.Structure):
    _fields_ = [("n", C.c_int32), ("q", C.c_int32), ("degree", C.c_int32), ("pin", C.c_int32),
                ("rho", C.c_double), ("mu", C.c_double), ("precision", C.c_int32),
                ("x", C.c_void_p), ("y", C.c_void_p), ("tag", C.c_void_p), ("nx", C.c_void_p),
                ("ny", C.c_void_p), ("ubc", C.c_void_p), ("vbc", C.c_void_p),
                ("precond", C.c_int32), ("period", C.c_double * 2), ("force", C.c_double * 2)]


class StepParams(C.Structure):
    _fields_ = [("dt", C.c_double), ("alpha", C.c_double * 3), ("krylov_tol", C.c_double),
                ("krylov_maxit", C.c_int32), ("inner_tol", C.c_double),
                ("inner_maxit", C.c_int32)]


class IterStats(C.Structure):
    _fields_ = [("iters", C.c_int32 * 3), ("relres", C.c_double * 3),
                ("sweeps", C.c_int32 * 3)]


class SolveParams(C.Structure):
    _fields_ = [("dt", C.c_double), ("resid_tol", C.c_double), ("max_steps", C.c_int32),
                ("max_outer", C.c_int32), ("krylov_tol", C.c_double),
                ("krylov_maxit", C.c_int32), ("inner_tol", C.c_double),
                ("inner_maxit", C.c_int32), ("criterion", C.c_int32)]


class SolveStats(C.Structure):
    _fields_ = [("steps", C.c_int32), ("outer_iters", C.c_int64),
                ("krylov_iters", C.c_int64 * 3), ("resid", C.c_double * 4),
                ("change", C.c_double)]


class KernelStat(C.Structure):
    _fields_ = [("launches", C.c_int64), ("ms", C.c_double), ("units", C.c_double),
                ("bytes", C.c_double)]


KSTAT = {"krylov_p": 0, "krylov_mom": 1, "weights": 2, "knn": 3, "outer": 4}

class ServerParams(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_size_t), ("max_active", C.c_int32)]


class Result(C.Structure):
    _fields_ = [("state", C.c_int32), ("status", C.c_int32), ("queue_s", C.c_double),
                ("latency_s", C.c_double), ("steps", C.c_int32), ("outer_iters", C.c_int64),
                ("resid", C.c_double * 4), ("admit_attempts", C.c_int32),
                ("arrive_s", C.c_double), ("admit_s", C.c_double), ("done_s", C.c_double),
                ("builds", C.c_int32)]


STEP_CB = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_int32, C.c_double)

_lib = None


def load(path: str = LIB_PATH):
    """Load the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build()")
    L = C.CDLL(path)
    vp, i32, i64, dbl, sz = C.c_void_p, C.c_int32, C.c_int64, C.c_double, C.c_size_t
    sig = {
        "rbffd_ctx_create": (C.c_int, [C.POINTER(vp), C.c_int, sz, vp]),
        "rbffd_ctx_destroy": (None, [vp]),
        "rbffd_last_error": (C.c_char_p, []),
        "rbffd_ctx_launch_count": (i64, [vp]),
        "rbffd_ctx_profile": (C.c_int, [vp, C.c_int]),
        "rbffd_ctx_kernel_stat": (C.c_int, [vp, i32, C.POINTER(KernelStat)]),
        "rbffd_build_stencils": (C.c_int, [vp, i32, vp, vp, vp, i32, vp]),
        "rbffd_build_stencils_static": (C.c_int, [vp, i32, vp, vp, vp, i32, vp]),
        "rbffd_weights": (C.c_int, [vp, i32, vp, vp, i32, vp, i32, vp, vp, vp,
                                    C.POINTER(i32)]),
        "rbffd_problem_create": (C.c_int, [vp, C.POINTER(ProblemDesc), C.POINTER(vp)]),
        "rbffd_problem_reload": (C.c_int, [vp, C.POINTER(ProblemDesc)]),
        "rbffd_problem_destroy": (None, [vp]),
        "rbffd_problem_bytes": (sz, [vp]),
        "rbffd_courant": (C.c_int, [vp, dbl, i32, C.POINTER(dbl), C.POINTER(dbl)]),
        "rbffd_problem_amg_info": (C.c_int, [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i64),
                                             C.POINTER(dbl)]),
        "rbffd_amg_analyze": (C.c_int, [i32, vp, vp, vp, C.POINTER(i32), C.POINTER(i32),
                                        C.POINTER(i64), C.POINTER(dbl)]),
        "simple_iterate": (C.c_int, [vp, C.POINTER(StepParams), C.POINTER(dbl),
                                     C.POINTER(IterStats)]),
        "rbffd_time_step": (C.c_int, [vp, C.POINTER(SolveParams), dbl, C.POINTER(i32),
                                      C.POINTER(dbl)]),
        "solve_steady": (C.c_int, [vp, C.POINTER(SolveParams), C.POINTER(SolveStats)]),
        "solve_unsteady": (C.c_int, [vp, C.POINTER(SolveParams), i32, STEP_CB, vp,
                                     C.POINTER(SolveStats)]),
        "rbffd_steady_residual": (C.c_int, [vp, C.POINTER(dbl)]),
        "rbffd_ctx_set_wait_limit": (C.c_int, [vp, i32]),
        "rbffd_ctx_set_amg_compose": (C.c_int, [vp, C.c_int]),
        "rbffd_problem_amg_cycle": (C.c_int, [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i64),
                                              C.POINTER(i64), C.POINTER(i32)]),
        "rbffd_ctx_set_amg_device_setup": (C.c_int, [vp, C.c_int]),
        "rbffd_ctx_set_fgmres_reorth": (C.c_int, [vp, C.c_int]),
        "rbffd_amg_cycle_host": (C.c_int, [i32, vp, vp, vp, vp, vp, vp, C.POINTER(i32),
                                           C.POINTER(i32)]),
        "rbffd_amg_aggregates_host": (C.c_int, [i32, vp, vp, vp, vp, C.POINTER(i32)]),
        "rbffd_get_field": (C.c_int, [vp, i32, vp]),
        "rbffd_set_field": (C.c_int, [vp, i32, vp]),
        "rbffd_get_operators": (C.c_int, [vp, vp, vp, vp, vp, vp]),
        "rbffd_apply": (C.c_int, [vp, i32, vp, vp]),
        "rbffd_batch_create": (C.c_int, [vp, i32, C.POINTER(vp), C.POINTER(vp)]),
        "rbffd_batch_destroy": (None, [vp]),
        "rbffd_batch_iterate": (C.c_int, [vp, C.POINTER(StepParams), vp, vp, vp, vp, vp]),
        "rbffd_batch_graph_stats": (C.c_int, [vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64)]),
        "rbffd_batch_tuning": (C.c_int, [vp, C.POINTER(i32), C.POINTER(dbl), C.POINTER(dbl)]),
        "rbffd_batch_set_autotune": (C.c_int, [vp, C.c_int]),
        "rbffd_plan_work_lists": (C.c_int, [i32, vp, vp, vp, i32, dbl, C.POINTER(i32),
                                            C.POINTER(i32), C.POINTER(i32), vp]),
        "rbffd_server_create": (C.c_int, [vp, C.POINTER(ServerParams), C.POINTER(vp)]),
        "rbffd_server_submit": (C.c_int, [vp, C.POINTER(ProblemDesc), C.POINTER(SolveParams),
                                          C.POINTER(C.c_uint64)]),
        "rbffd_server_poll": (C.c_int, [vp, C.c_uint64, C.POINTER(Result), vp, vp, vp]),
        "rbffd_server_drain": (C.c_int, [vp]),
        "rbffd_server_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(rc, where):
    if rc != OK:
        raise RbffdError(rc, where, load().rbffd_last_error().decode(errors="replace"))


def ptr(a):
    """Raw address of a torch tensor or numpy array (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    raise TypeError(f"cannot take the address of {type(a)}")


class Context:
    """A device context: device, HBM budget and the stream work goes to."""

    def __init__(self, device: int = 0, hbm_budget: int = 0, stream=None):
        L = load()
        h = C.c_void_p()
        s = None if stream is None else C.c_void_p(stream)
        _check(L.rbffd_ctx_create(C.byref(h), device, hbm_budget, s), "rbffd_ctx_create")
        self.h = h
        self.device = device

    def set_wait_limit(self, log2_cycles: int):
        """Bound of the device-side waits of later launches: 2^log2_cycles
        cycles, 0 for the default (rbffd_ctx_set_wait_limit)."""
        _check(load().rbffd_ctx_set_wait_limit(self.h, int(log2_cycles)),
               "rbffd_ctx_set_wait_limit")

    def set_fgmres_reorth(self, mode):
        """Flexible GMRES's Gram-Schmidt (rbffd_ctx_set_fgmres_reorth): 0 one
        pass, 1 (True) two passes a step, 2 two passes with the second
        delayed (one reduction a step)."""
        _check(load().rbffd_ctx_set_fgmres_reorth(self.h, int(mode)),
               "rbffd_ctx_set_fgmres_reorth")

    def set_amg_device_setup(self, on: bool):
        """Whether level 0 of multigrid hierarchies built from now on is built
        on the device (large p' matrices; rbffd_ctx_set_amg_device_setup)."""
        _check(load().rbffd_ctx_set_amg_device_setup(self.h, 1 if on else 0),
               "rbffd_ctx_set_amg_device_setup")

    def set_amg_compose(self, on: bool):
        """Whether multigrid hierarchies built from now on get the composed
        (three-phase) cycle when it pays (rbffd_ctx_set_amg_compose)."""
        _check(load().rbffd_ctx_set_amg_compose(self.h, 1 if on else 0),
               "rbffd_ctx_set_amg_compose")

    def close(self):
        if getattr(self, "h", None) is not None:
            load().rbffd_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def launches(self) -> int:
        return int(load().rbffd_ctx_launch_count(self.h))

    def profile(self, enable: bool = True):
        _check(load().rbffd_ctx_profile(self.h, int(enable)), "rbffd_ctx_profile")

    def kernel_stat(self, name: str) -> dict:
        st = KernelStat()
        _check(load().rbffd_ctx_kernel_stat(self.h, KSTAT[name], C.byref(st)),
               "rbffd_ctx_kernel_stat")
        return {"launches": st.launches, "ms": st.ms, "units": st.units, "bytes": st.bytes}


def rbffd_build_stencils(ctx, x, y, tag, q, idx):
    n = int(x.shape[0])
    _check(load().rbffd_build_stencils(ctx.h, n, ptr(x), ptr(y), ptr(tag), int(q), ptr(idx)),
           "rbffd_build_stencils")


STATIC_MAX_POINTS = 262144


def rbffd_build_stencils_static(ctx, x, y, tag, q, idx):
    """rbffd_build_stencils without any device allocation (fixed workspace
    inside the library; n <= STATIC_MAX_POINTS; overlapping calls race)."""
    n = int(x.shape[0])
    _check(load().rbffd_build_stencils_static(ctx.h, n, ptr(x), ptr(y), ptr(tag), int(q),
                                              ptr(idx)), "rbffd_build_stencils_static")


def rbffd_weights(ctx, x, y, q, idx, degree, wx, wy, wl):
    n = int(x.shape[0])
    fs = C.c_int32(-1)
    rc = load().rbffd_weights(ctx.h, n, ptr(x), ptr(y), int(q), ptr(idx), int(degree), ptr(wx),
                              ptr(wy), ptr(wl), C.byref(fs))
    if rc == ESINGULAR:
        return fs.value
    _check(rc, "rbffd_weights")
    return -1


def make_desc(fp, precision=PREC_FP64, keep=None, precond=PRECOND_JACOBI):
    """ProblemDesc for a FlowProblem (host numpy arrays, copied by the
    library at create/reload).  `keep` receives the arrays to keep alive."""
    arrs = {
        "x": np.ascontiguousarray(fp.x, np.float64), "y": np.ascontiguousarray(fp.y, np.float64),
        "tag": np.ascontiguousarray(fp.tag, np.int8),
        "nx": np.ascontiguousarray(fp.nx, np.float64),
        "ny": np.ascontiguousarray(fp.ny, np.float64),
        "ubc": np.ascontiguousarray(fp.ubc, np.float64),
        "vbc": np.ascontiguousarray(fp.vbc, np.float64)}
    if keep is not None:
        keep.update(arrs)
    d = ProblemDesc()
    d.n, d.q, d.degree, d.pin = fp.n, fp.q, fp.degree, int(fp.pin)
    d.rho, d.mu, d.precision = float(fp.rho), float(fp.mu), int(precision)
    d.precond = int(precond)
    d.period[0], d.period[1] = (float(v) for v in getattr(fp, "period", (0.0, 0.0)))
    d.force[0], d.force[1] = (float(v) for v in getattr(fp, "force", (0.0, 0.0)))
    for k, a in arrs.items():
        setattr(d, k, a.ctypes.data)
    return d


def desc_from_pointers(n, q, degree, pin, rho, mu, precision, x, y, tag, nx, ny, ubc, vbc,
                       precond=PRECOND_JACOBI, period=(0.0, 0.0), force=(0.0, 0.0)):
    """ProblemDesc from raw host or device buffers (tensors or arrays)."""
    d = ProblemDesc()
    d.n, d.q, d.degree, d.pin = int(n), int(q), int(degree), int(pin)
    d.rho, d.mu, d.precision = float(rho), float(mu), int(precision)
    d.precond = int(precond)
    d.period[0], d.period[1] = float(period[0]), float(period[1])
    d.force[0], d.force[1] = float(force[0]), float(force[1])
    for k, a in (("x", x), ("y", y), ("tag", tag), ("nx", nx), ("ny", ny), ("ubc", ubc),
                 ("vbc", vbc)):
        setattr(d, k, ptr(a))
    return d


class Problem:
    """A device-resident flow problem (clouds, weights, operators, fields)."""

    def __init__(self, ctx, fp=None, precision=PREC_FP64, desc=None, precond=PRECOND_JACOBI):
        self.ctx = ctx
        keep = {}
        d = desc if desc is not None else make_desc(fp, precision, keep, precond)
        h = C.c_void_p()
        _check(load().rbffd_problem_create(ctx.h, C.byref(d), C.byref(h)), "rbffd_problem_create")
        self.h = h
        self.n, self.q = int(d.n), int(d.q)

    def reload(self, fp=None, precision=PREC_FP64, desc=None, precond=PRECOND_JACOBI):
        keep = {}
        d = desc if desc is not None else make_desc(fp, precision, keep, precond)
        _check(load().rbffd_problem_reload(self.h, C.byref(d)), "rbffd_problem_reload")

    def close(self):
        if getattr(self, "h", None) is not None:
            load().rbffd_problem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def nbytes(self) -> int:
        return int(load().rbffd_problem_bytes(self.h))

    def courant(self, dt, iters=200):
        """(lambda, lambda dt / 2) of the convection-diffusion operator."""
        lam = C.c_double(0)
        co = C.c_double(0)
        _check(load().rbffd_courant(self.h, float(dt), int(iters), C.byref(lam), C.byref(co)),
               "rbffd_courant")
        return lam.value, co.value

    def amg_info(self, with_time=False):
        """Rows and nonzeros per level of the p' multigrid hierarchy ([] with
        Jacobi); with_time: also the host build time in ms."""
        lv = C.c_int32(0)
        rows = (C.c_int32 * AMG_MAX_LEVELS)()
        nnz = (C.c_int64 * AMG_MAX_LEVELS)()
        ms = C.c_double(0)
        _check(load().rbffd_problem_amg_info(self.h, C.byref(lv), rows, nnz, C.byref(ms)),
               "rbffd_problem_amg_info")
        levels = [(int(rows[i]), int(nnz[i])) for i in range(lv.value)]
        return (levels, ms.value) if with_time else levels

    def amg_cycle(self):
        """The composed multigrid cycle: dict of coarse entries (0: not
        built), chunks, restriction and Q nonzeros (rbffd_problem_amg_cycle)."""
        nc, ch, dl = C.c_int32(0), C.c_int32(0), C.c_int32(0)
        nr, nq = C.c_int64(0), C.c_int64(0)
        _check(load().rbffd_problem_amg_cycle(self.h, C.byref(nc), C.byref(ch), C.byref(nr),
                                              C.byref(nq), C.byref(dl)), "rbffd_problem_amg_cycle")
        return {"coarse_entries": nc.value, "chunks": ch.value, "restrict_nnz": nr.value,
                "q_nnz": nq.value, "device_level0": bool(dl.value)}

    def get(self, name, out=None):
        out = np.zeros(self.n) if out is None else out
        _check(load().rbffd_get_field(self.h, FIELDS[name], ptr(out)), "rbffd_get_field")
        return out

    def set(self, name, arr):
        if isinstance(arr, np.ndarray):
            arr = np.ascontiguousarray(arr, np.float64)
        _check(load().rbffd_set_field(self.h, FIELDS[name], ptr(arr)), "rbffd_set_field")

    def operators(self):
        n, q = self.n, self.q
        idx = np.zeros((n, q), np.int32)
        wx, wy, wl, pc = (np.zeros((n, q)) for _ in range(4))
        _check(load().rbffd_get_operators(self.h, ptr(idx), ptr(wx), ptr(wy), ptr(wl), ptr(pc)),
               "rbffd_get_operators")
        return {"idx": idx, "wx": wx, "wy": wy, "wl": wl, "pval": pc}

    def apply(self, which, x, y):
        _check(load().rbffd_apply(self.h, int(which), ptr(x), ptr(y)), "rbffd_apply")

    def simple_iterate(self, dt, alpha=(1.5, -2.0, 0.5), krylov_tol=1e-12, krylov_maxit=10000,
                       inner_tol=0.0, inner_maxit=0):
        sp = StepParams(dt, (C.c_double * 3)(*alpha), krylov_tol, krylov_maxit, inner_tol,
                        inner_maxit)
        d = C.c_double(0)
        st = IterStats()
        _check(load().simple_iterate(self.h, C.byref(sp), C.byref(d), C.byref(st)),
               "simple_iterate")
        return d.value, {"iters": list(st.iters), "relres": list(st.relres),
                         "sweeps": list(st.sweeps)}

    def time_step(self, dt, tol_outer, max_outer=20, krylov_tol=1e-12, krylov_maxit=10000,
                  inner_tol=0.0, inner_maxit=0):
        sp = SolveParams(dt, 0.0, 1, max_outer, krylov_tol, krylov_maxit, inner_tol, inner_maxit,
                         0)
        it = C.c_int32(0)
        ch = C.c_double(0)
        _check(load().rbffd_time_step(self.h, C.byref(sp), tol_outer, C.byref(it), C.byref(ch)),
               "rbffd_time_step")
        return it.value, ch.value

    def steady_residual(self):
        """(R_m, R_c, R, lambda); see rbffd_steady_residual."""
        r = (C.c_double * 4)()
        _check(load().rbffd_steady_residual(self.h, r), "rbffd_steady_residual")
        return np.array(list(r))

    def solve_steady(self, dt, resid_tol=1e-8, max_steps=10000, max_outer=20, krylov_tol=1e-12,
                     krylov_maxit=10000, check=True, inner_tol=0.0, inner_maxit=0, criterion=0):
        sp = SolveParams(dt, resid_tol, max_steps, max_outer, krylov_tol, krylov_maxit, inner_tol,
                         inner_maxit, criterion)
        st = SolveStats()
        rc = load().solve_steady(self.h, C.byref(sp), C.byref(st))
        if check:
            _check(rc, "solve_steady")
        return rc, _stats(st)

    def solve_unsteady(self, dt, n_steps, max_outer=20, krylov_tol=1e-12, krylov_maxit=10000,
                       on_step=None, inner_tol=0.0, inner_maxit=0):
        sp = SolveParams(dt, 0.0, 0, max_outer, krylov_tol, krylov_maxit, inner_tol, inner_maxit,
                         0)
        st = SolveStats()
        cb = STEP_CB(on_step) if on_step is not None else STEP_CB()
        _check(load().solve_unsteady(self.h, C.byref(sp), int(n_steps), cb, None, C.byref(st)),
               "solve_unsteady")
        return _stats(st)


class Batch:
    """Problems advanced together: one outer iteration of every active
    member per call, the Krylov solves of all members in one launch each."""

    def __init__(self, ctx, problems):
        self.ctx = ctx
        self.problems = list(problems)
        arr = (C.c_void_p * len(self.problems))(*[p.h.value for p in self.problems])
        h = C.c_void_p()
        _check(load().rbffd_batch_create(ctx.h, len(self.problems), arr, C.byref(h)),
               "rbffd_batch_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None) is not None:
            load().rbffd_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def iterate(self, dt, active=None, alpha=(1.5, -2.0, 0.5), krylov_tol=1e-12,
                krylov_maxit=10000):
        """dt: one time step for all members, or one per member."""
        m = len(self.problems)
        per = None
        if np.ndim(dt) > 0:
            per = np.ascontiguousarray(dt, np.float64)
            dt = float(per[0])
        sp = StepParams(dt, (C.c_double * 3)(*alpha), krylov_tol, krylov_maxit, 0.0, 0)
        act = None if active is None else np.ascontiguousarray(active, np.int32)
        d = np.zeros(m)
        st = (IterStats * m)()
        status = np.zeros(m, np.int32)
        _check(load().rbffd_batch_iterate(self.h, C.byref(sp), ptr(per), ptr(act), ptr(d),
                                          C.cast(st, C.c_void_p), ptr(status)),
               "rbffd_batch_iterate")
        its = np.array([list(s.iters) for s in st])
        return d, its, status

    def graph_stats(self):
        """(graphs captured, replays, kernels per replay) of the batched
        outer iteration."""
        c, r, k = C.c_int64(0), C.c_int64(0), C.c_int64(0)
        _check(load().rbffd_batch_graph_stats(self.h, C.byref(c), C.byref(r), C.byref(k)),
               "rbffd_batch_graph_stats")
        return c.value, r.value, k.value

    def tuning(self):
        """(tuned, team-size scale per launch slot, cost table 9 x 4) of the
        work-list autotuner (rbffd_batch_tuning)."""
        t = C.c_int32(0)
        sc = (C.c_double * 9)()
        cost = (C.c_double * 36)()
        _check(load().rbffd_batch_tuning(self.h, C.byref(t), sc, cost), "rbffd_batch_tuning")
        return bool(t.value), list(sc), np.array(list(cost)).reshape(9, 4)

    def set_autotune(self, on):
        """Switch the work-list autotuner on (restart it) or off (scale 1)."""
        _check(load().rbffd_batch_set_autotune(self.h, 1 if on else 0), "rbffd_batch_set_autotune")


def amg_analyze(rowptr, col, val):
    """Host-only multigrid hierarchy of a CSR matrix: ([(rows, nnz)], ms)."""
    rowptr = np.ascontiguousarray(rowptr, np.int32)
    col = np.ascontiguousarray(col, np.int32)
    val = np.ascontiguousarray(val, np.float64)
    lv = C.c_int32(0)
    rows = (C.c_int32 * AMG_MAX_LEVELS)()
    nnz = (C.c_int64 * AMG_MAX_LEVELS)()
    ms = C.c_double(0)
    _check(load().rbffd_amg_analyze(rowptr.size - 1, ptr(rowptr), ptr(col), ptr(val),
                                    C.byref(lv), rows, nnz, C.byref(ms)), "rbffd_amg_analyze")
    return [(int(rows[i]), int(nnz[i])) for i in range(lv.value)], ms.value


def plan_work_lists(work, cap, rows, cmax, scale=1.0):
    """The batched launches' work-list plan (rbffd_plan_work_lists): (team of
    each solve, CTAs, team size, teams)."""
    work = np.ascontiguousarray(work, np.float64)
    cap = np.ascontiguousarray(cap, np.int32)
    rows = np.ascontiguousarray(rows, np.int32)
    team = np.zeros(work.size, np.int32)
    nc, ts, nt = C.c_int32(0), C.c_int32(0), C.c_int32(0)
    _check(load().rbffd_plan_work_lists(work.size, ptr(work), ptr(cap), ptr(rows), int(cmax),
                                        float(scale), C.byref(nc), C.byref(ts), C.byref(nt),
                                        ptr(team)), "rbffd_plan_work_lists")
    return team, nc.value, ts.value, nt.value


def amg_aggregates_host(rowptr, col, val):
    """Level 0's multigrid aggregates of a CSR matrix, on the host:
    (agg per row, number of aggregates)."""
    rowptr = np.ascontiguousarray(rowptr, np.int32)
    col = np.ascontiguousarray(col, np.int32)
    val = np.ascontiguousarray(val, np.float64)
    n = rowptr.size - 1
    agg = np.zeros(n, np.int32)
    na = C.c_int32(0)
    _check(load().rbffd_amg_aggregates_host(n, ptr(rowptr), ptr(col), ptr(val), ptr(agg),
                                            C.byref(na)), "rbffd_amg_aggregates_host")
    return agg, na.value


def amg_cycle_host(rowptr, col, val, b):
    """One multigrid cycle of a CSR matrix's hierarchy applied to b on the
    host in FP64, level by level and composed: (out_levels, out_composed,
    coarse entries, chunks); out_composed is zeros when not built."""
    rowptr = np.ascontiguousarray(rowptr, np.int32)
    col = np.ascontiguousarray(col, np.int32)
    val = np.ascontiguousarray(val, np.float64)
    b = np.ascontiguousarray(b, np.float64)
    n = rowptr.size - 1
    ol, oc = np.zeros(n), np.zeros(n)
    nc, ch = C.c_int32(0), C.c_int32(0)
    _check(load().rbffd_amg_cycle_host(n, ptr(rowptr), ptr(col), ptr(val), ptr(b), ptr(ol),
                                       ptr(oc), C.byref(nc), C.byref(ch)),
           "rbffd_amg_cycle_host")
    return ol, oc, nc.value, ch.value


class Server:
    """Continuous-batching request server (steady solves)."""

    def __init__(self, ctx, hbm_budget=0, max_active=0):
        self.ctx = ctx
        prm = ServerParams(hbm_budget, max_active)
        h = C.c_void_p()
        _check(load().rbffd_server_create(ctx.h, C.byref(prm), C.byref(h)), "rbffd_server_create")
        self.h = h
        self.n = {}

    def submit(self, fp, dt=None, resid_tol=1e-6, max_steps=2000, max_outer=20,
               krylov_tol=1e-12, krylov_maxit=10000, criterion=0, precond=PRECOND_JACOBI,
               precision=PREC_FP64):
        keep = {}
        d = make_desc(fp, precision, keep, precond)
        sp = SolveParams(fp.dt if dt is None else dt, resid_tol, max_steps, max_outer,
                         krylov_tol, krylov_maxit, 0.0, 0, criterion)
        t = C.c_uint64(0)
        _check(load().rbffd_server_submit(self.h, C.byref(d), C.byref(sp), C.byref(t)),
               "rbffd_server_submit")
        self.n[t.value] = fp.n
        return t.value

    def poll(self, ticket, fields=False):
        r = Result()
        n = self.n[ticket]
        u = v = p = None
        if fields:
            u, v, p = np.zeros(n), np.zeros(n), np.zeros(n)
        _check(load().rbffd_server_poll(self.h, ticket, C.byref(r), ptr(u), ptr(v), ptr(p)),
               "rbffd_server_poll")
        out = {"state": r.state, "status": r.status, "queue_s": r.queue_s,
               "latency_s": r.latency_s, "steps": r.steps, "outer": r.outer_iters,
               "resid": list(r.resid), "admit_attempts": r.admit_attempts,
               "arrive_s": r.arrive_s, "admit_s": r.admit_s, "done_s": r.done_s,
               "builds": r.builds}
        if fields:
            out.update(u=u, v=v, p=p)
        return out

    def drain(self):
        _check(load().rbffd_server_drain(self.h), "rbffd_server_drain")

    def close(self):
        if getattr(self, "h", None) is not None:
            load().rbffd_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _stats(st):
    return {"steps": st.steps, "outer": st.outer_iters, "krylov": list(st.krylov_iters),
            "resid": list(st.resid), "change": st.change}
