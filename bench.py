"""Benchmark of the semi-implicit PHS-RBF-FD hot path on one GB300.

One STEP is one pass of the whole hot path over one synthetic problem:
S1 clouds + S2 weights + S3 packed operators and the p' preconditioner
(rbffd_problem_reload), then the first BDF2 time step from rest (S4-S10
outer iterations until Delta < 1e-4, the paper's first outer tolerance, at
most --outer of them).  The metric is SIMPLE outer iterations per second of
whole-step time.

Workload (default): the lid-driven cavity, Re = 1000, 200 x 200 clustered
and jittered cloud (N = 40 000), polynomial degree 4, q = 30, dt from a
Courant number of about 10.  The p' solver (--precond): fgmres (default for
single problems): flexible GMRES(30) whose Arnoldi process runs in FP32
with one FP32 smoothed-aggregation V-cycle per step, inside FP64 restarts;
amg (default for batch and serve): FP64 BiCGSTAB with an FP64 V-cycle;
jacobi: FP64 BiCGSTAB with the diagonal.  The momentum solves (--precision):
mixed (default for single problems): FP32 BiCGSTAB inside FP64 defect
correction; ff: float-float; fp64 (batch and serve).  Every solve stops on
the same FP64 relative residual (1e-12).
Other workloads: kovasznay50, cylinder150k (outlet, symmetry and no-slip
rows, 147 827 graded points), batch (many instances per launch) and serve
(a Poisson stream of steady-solve requests through the request server).

Printed: one JSON line (rank 0).  `value` is device-resident throughput
(inputs already in HBM); `e2e` is the same metric through the C ABI from
pinned host buffers with the host<->device copies inside the timed region;
`roofline` is for the pressure-correction BiCGSTAB kernel, timed live with
CUDA events on the library's stream; `cpu_baseline` is the CPU oracle on a
bounded sample of the same step.  `--impl reference` times the oracle
itself (host cores) on the same step.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2106_07616_gb300 import clouds  # noqa: E402

FALLBACK_HBM_GBS = 6800.0
L2_FLUSH_BYTES = 256 << 20


def workload(name: str):
    if name == "cavity200":
        fp = clouds.cavity(200)
        desc = (f"lid-driven cavity Re=1000, 200x200 2x-clustered jittered cloud "
                f"(N={fp.n}), degree 4, q=30, dt={fp.dt:.4g} (Courant ~10)")
    elif name == "kovasznay50":
        fp = clouds.kovasznay(50, dt=0.4)
        desc = f"Kovasznay Re=40, 50x50 jittered cloud (N={fp.n}), degree 3, q=20, dt=0.4"
    elif name == "cylinder150k":
        fp = clouds.cylinder()
        desc = (f"flow past a cylinder Re=100 in [-5,15]x[-5,5], graded cloud h 0.02 at the "
                f"cylinder (N={fp.n}), degree 3, q=20, dt={fp.dt:.3g}, inlet / symmetry / "
                f"outlet / no-slip rows, uniform start")
    else:
        raise SystemExit(f"unknown workload {name}")
    return fp, desc


def combine_ranks(total_ms, total_units, device="cpu"):
    """Whole-job timing over the ranks of the default process group: the
    slowest rank's time and the units every rank processed (each rank runs
    its own replica: weak scaling, no collective on the data path).  One
    rank, or no process group: the inputs."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(total_ms), float(total_units)
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(total_units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t[0]), float(u[0])


def solver_codes(args, rbffd):
    """(precision, p' preconditioner) library codes of the command line."""
    prec = {"mixed": rbffd.PREC_MIXED, "ff": rbffd.PREC_MIXED_FF,
            "fp64": rbffd.PREC_FP64}[args.precision]
    pc = {"jacobi": rbffd.PRECOND_JACOBI, "amg": rbffd.PRECOND_AMG,
          "fgmres": rbffd.PRECOND_AMG_FGMRES}[args.precond]
    return prec, pc


KRYLOV_PROFILES = {
    # preconditioner: (committed ncu summary, kernel sources it was taken from)
    "jacobi": ("k_bicgstab_fp64_cavity200.md", ("krylov.cu", "krylov_dev.cuh", "common.cuh")),
    "amg": ("k_bicgstab_amg_fp64_cavity200.md",
            ("krylov.cu", "krylov_dev.cuh", "common.cuh", "amg_dev.cuh", "amg.cuh", "amg.cu",
             "amg_setup.cu")),
    "fgmres": ("k_fgmres_cavity200.md",
               ("fgmres.cu", "fgmres.cuh", "krylov_dev.cuh", "common.cuh", "amg_dev.cuh",
                "amg.cuh", "amg.cu", "amg_setup.cu")),
}


def krylov_traffic(precision, workload_name, precond="jacobi"):
    """DRAM bytes per pressure-correction launch from the committed ncu
    summary, only while the kernel sources still hash to the profiled ones."""
    import hashlib
    # the flexible GMRES kernel is the same whatever the momentum precision
    if workload_name != "cavity200" or precond not in KRYLOV_PROFILES or (
            precision != "fp64" and precond != "fgmres"):
        return None
    name, files = KRYLOV_PROFILES[precond]
    prof = os.path.join(ROOT, "profiles", name)
    csrc = os.path.join(ROOT, "paper_2106_07616_gb300", "csrc")
    try:
        h = hashlib.sha256()
        for f in files:
            h.update(open(os.path.join(csrc, f), "rb").read())
        fields = dict(l.split(":", 1) for l in open(prof) if l.startswith(("source_hash", "traffic_")))
        if fields["source_hash"].split()[0] != h.hexdigest()[:16]:
            return None
        return float(fields["traffic_bytes_per_launch"])
    except Exception:
        return None


def batch_instances(count=256, seed=4):
    """Batched workload: independent Kovasznay / cavity instances, N
    log-uniform on [1k, 64k] (square lattices), degree uniform in {2,3,4,5},
    q = 2m, dt from a Courant number of about 10."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(count):
        n = float(np.exp(rng.uniform(np.log(1000.0), np.log(64000.0))))
        side = int(np.ceil(np.sqrt(n)))
        k = int(rng.integers(2, 6))
        q = (k + 1) * (k + 2)
        if rng.uniform() < 0.5:
            out.append(clouds.kovasznay(side, seed=4000 + i, degree=k, q=q, dt=20.0 / (side - 1)))
        else:
            out.append(clouds.cavity(side, seed=4000 + i, degree=k, q=q, dt=10.0 / (side - 1)))
    return out


def run_batch(args):
    print(json.dumps(batch_line(args)), flush=True)


def batch_line(args):
    """Many instances per step: S1-S3 for every member, then one batched
    outer iteration (both Krylov solves of all members in one launch each)."""
    import torch

    from paper_2106_07616_gb300 import _build, rbffd
    _build.build()
    fps = batch_instances(args.count or 256)
    stream = torch.cuda.current_stream()
    ctx = rbffd.Context(0, stream=stream.cuda_stream)
    prec, pc = solver_codes(args, rbffd)
    probs = [rbffd.Problem(ctx, fp, prec, precond=pc) for fp in fps]
    B = rbffd.Batch(ctx, probs)
    rows = sum(fp.n for fp in fps)
    nnz = sum(fp.n * fp.q for fp in fps)

    dts = np.array([fp.dt for fp in fps])

    def iterate_all():
        d, its, st = B.iterate(dts)  # every member with its own dt, one launch per solve
        return its, int(np.sum(st == 0))

    def reload_all():
        for P, fp in zip(probs, fps):
            P.reload(fp, prec, precond=pc)

    # the work-list autotuner runs on the first nine iterations of the batch
    for _ in range(max(args.warmup, 9)):
        reload_all()
        iterate_all()
    torch.cuda.synchronize()
    tuned, scales, costs = B.tuning()
    l0 = ctx.launches
    total_ms, outer = 0.0, 0
    with ClockSampler(0) as clk:
        for k in range(args.steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            reload_all()
            its, ok = iterate_all()
            e1.record(stream)
            e1.synchronize()
            total_ms += e0.elapsed_time(e1)
            outer += ok
    launches = (ctx.launches - l0) // max(args.steps, 1)
    # end to end: the same step from host arrays (the reload copies the
    # points in) with every member's u, v, p read back
    e2e_t, e2e_it, d2h = 0.0, 0, 0
    for k in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        reload_all()
        its, ok = iterate_all()
        for P in probs:
            for f in ("u", "v", "p"):
                d2h += P.get(f).nbytes
        e2e_t += time.perf_counter() - t0
        e2e_it += ok
    h2d = sum(sum(np.asarray(getattr(fp, a)).nbytes for a in ("x", "y", "tag", "nx", "ny",
                                                                 "ubc", "vbc")) for fp in fps)
    # the kernel split, from one more step with live kernel timing
    ctx.profile(True)
    reload_all()
    iterate_all()
    torch.cuda.synchronize()
    kp = ctx.kernel_stat("krylov_p")
    km = ctx.kernel_stat("krylov_mom")
    ctx.profile(False)
    peak, src = read_peaks()
    kp_gbps = kp["bytes"] / (kp["ms"] / 1e3) / 1e9 if kp["ms"] else None
    out = {"metric": "SIMPLE outer iters/s (batched instances)", "value": outer / (total_ms / 1e3),
           "unit": "instance_outer_iter/s", "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": ("f32x2+f64" if args.precision == "ff" else
                     "f32+f64" if args.precision == "mixed" or args.precond == "fgmres"
                     else "f64"),
           "data": "synthetic",
           "e2e": {"value": e2e_it / e2e_t, "unit": "instance_outer_iter/s",
                   "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h // 2},
           "gpu_launches": launches,
           "roofline": {"bound": "hbm", "achieved": kp_gbps, "peak": peak, "unit": "GB/s",
                        "frac": kp_gbps / peak if kp_gbps else None, "traffic": None,
                        "kernel": f"batched pressure-correction launch ({args.precond})"},
           "cpu_baseline": None,
           "config": {"workload": f"batch{args.count or 256}", "instances": len(fps), "rows": rows,
                      "precond": args.precond, "precision": args.precision,
                      "l2": "inputs (~GBs of operators) exceed the 129 MB L2",
                      "nnz_per_operator": nnz,
                      "description": "Kovasznay/cavity instances, N log-uniform [1k,64k], "
                                     "degree {2..5}, q=2m; step = S1-S3 for all + one outer "
                                     "iteration of all (one batched launch per Krylov solve)"},
           "krylov_p": {"launches": kp["launches"], "ms": kp["ms"],
                        "algorithmic_GBps": kp["bytes"] / (kp["ms"] / 1e3) / 1e9 if kp["ms"] else None,
                        "frac_of_hbm": (kp["bytes"] / (kp["ms"] / 1e3) / 1e9) / peak if kp["ms"] else None},
           "krylov_mom": {"launches": km["launches"], "ms": km["ms"],
                          "algorithmic_GBps": km["bytes"] / (km["ms"] / 1e3) / 1e9 if km["ms"] else None},
           "peak_hbm_GBps": peak, "peak_source": src, "clocks": clk.summary(),
           "autotune": {"tuned": tuned, "team_scale_per_slot": scales,
                        "ms_per_row_iteration": costs.tolist(),
                        "candidates": [1.0, 2.0, 0.5, 4.0],
                        "slots": ["momentum 2-RHS", "momentum 1-RHS", "p' jacobi",
                                  "p' multigrid", "p' fgmres", "mixed f32 2-RHS",
                                  "mixed f32 single", "mixed ff 2-RHS", "mixed ff single"]}}
    for P in probs:
        P.close()
    B.close()
    ctx.close()
    return out


def serve_requests(count, seed=5, n_lo=5000.0, n_hi=50000.0, cfl=10.0):
    """Serving workload: steady solves of three geometries drawn uniformly --
    Kovasznay (Re 20-60), lid-driven cavity (Re 10-400) and flow past a
    cylinder (Re 10-40, the paper's steady range) -- N log-uniform on
    [n_lo, n_hi], degree {3, 4}, q = 2m, dt at a Courant number of about 10,
    Poisson arrivals at a mean of 20 per second."""
    rng = np.random.Generator(np.random.PCG64(seed))
    reqs, t = [], 0.0
    for i in range(count):
        t += rng.exponential(1.0 / 20.0)
        n = float(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi))))
        side = int(np.ceil(np.sqrt(n)))
        k = int(rng.integers(3, 5))
        q = (k + 1) * (k + 2)
        kind = int(rng.integers(0, 3))
        if kind == 0:
            re = float(rng.uniform(20.0, 60.0))
            fp = clouds.kovasznay(side, seed=5000 + i, degree=k, q=q, re=re,
                                  dt=cfl * 2.0 / (side - 1))
        elif kind == 1:
            re = float(rng.uniform(10.0, 400.0))
            fp = clouds.cavity(side, seed=5000 + i, degree=k, q=q, re=re,
                               dt=cfl / (side - 1))
        else:
            re = float(rng.uniform(10.0, 40.0))
            h0 = 0.1 * float(np.sqrt(5000.0 / n))
            fp = clouds.cylinder(int(n), seed=5000 + i, degree=k, q=q, re=re, dt=cfl * h0,
                                 h0=h0, hmax=0.5)
        reqs.append((t, fp))
    return reqs


def run_serve(args):
    print(json.dumps(serve_line(args)), flush=True)


def serve_line(args, n_hi=None):
    import torch  # noqa: F401

    from paper_2106_07616_gb300 import _build, rbffd
    _build.build()
    n_hi = float(n_hi or args.serve_n_hi)
    cfl = args.serve_cfl if args.resid_tol < 1e-6 else 10.0
    reqs = serve_requests(args.count or 48, n_hi=n_hi, cfl=cfl)
    ctx = rbffd.Context(0)
    S = rbffd.Server(ctx)
    t0 = time.perf_counter()
    tickets = []
    for t_arr, fp in reqs:
        wait = t_arr - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        tickets.append(S.submit(fp, resid_tol=args.resid_tol, max_steps=args.max_steps,
                                criterion=args.criterion,
                                precond=solver_codes(args, rbffd)[1],
                                precision=solver_codes(args, rbffd)[0]))
    S.drain()
    wall = time.perf_counter() - t0
    res = [S.poll(t) for t in tickets]
    S.close()
    ok = [r for r in res if r["status"] == 0]
    lat = np.array([r["latency_s"] for r in ok]) if ok else np.array([np.nan])
    fails = [{"status": r["status"], "steps": r["steps"], "outer": r["outer"],
              "R": r["resid"][2]} for r in res if r["status"] != 0]
    out = {"metric": "served latency to steady state", "unit": "s",
           "criterion": ("paper steady error (mean|u^{n+1}-u^n|+mean|v^{n+1}-v^n|)/dt"
                         if args.criterion == 1 else "steady residual R"),
           "p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
           "solves_per_s": len(ok) / wall, "requests": len(res), "ok": len(ok),
           "failed": {str(s): sum(1 for r in res if r["status"] == s)
                      for s in sorted(set(r["status"] for r in res)) if s != 0},
           "resid_tol": args.resid_tol, "wall_s": wall, "failures": fails[:12],
           "steps_ok": [r["steps"] for r in ok], "outer_ok": [r["outer"] for r in ok],
           "R_ok": [float(r["resid"][2]) for r in ok], "max_steps": args.max_steps,
           "precond": args.precond, "precision": args.precision,
           "dtype": ("f32x2+f64" if args.precision == "ff" else
                     "f32+f64" if args.precision == "mixed" or args.precond == "fgmres"
                     else "f64"),
           "config": {"workload": f"serve{args.count or 48}",
                      "description": (f"Poisson arrivals 20/s; Kovasznay Re 20-60 / cavity "
                                      f"Re 10-400 / cylinder Re 10-40, N log-uniform "
                                      f"[5k,{n_hi / 1e3:.0f}k], degree {{3,4}}, q=2m, dt = "
                                      f"{cfl:g} x spacing; continuous batching in one server")}}
    ctx.close()
    return out


def read_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            for k in ("hbm_gbs", "hbm_GBs", "hbm"):
                if k in d:
                    return float(d[k]), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.path is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [s.strip() for s in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_oracle_step(fp, outer, threads=0):
    """One step of the same hot path on the CPU oracle: build + first time
    step capped at `outer` outer iterations.  Returns (seconds, outer iters)."""
    import oracle
    cores = oracle.set_threads(threads)
    t0 = time.perf_counter()
    O = oracle.Problem(fp, krylov_tol=1e-12)
    for k, a in (fp.initial or {}).items():
        O.set(k, a)
    it, ch, last = O.time_step(fp.dt, 1e-4, max_outer=outer)
    dt = time.perf_counter() - t0
    del O
    return dt, it, cores


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    fp, desc = workload(args.workload)
    import oracle
    oracle.build()
    for _ in range(args.warmup):
        cpu_oracle_step(fp, args.outer)
    tot_t, tot_it, cores = 0.0, 0, 1
    for _ in range(args.steps):
        t, it, cores = cpu_oracle_step(fp, args.outer)
        tot_t += t
        tot_it += it
    value = tot_it / tot_t
    sample = (f"{args.steps} steps of: oracle build (clouds, weights, CSR) + first BDF2 step "
              f"capped at {args.outer} outer iterations, {desc}")
    out = {"metric": "SIMPLE outer iters/s", "value": value, "unit": "outer_iter/s",
           "impl": "reference", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * tot_t / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": args.workload, "description": desc, "outer_cap": args.outer},
           "cpu_baseline": {"value": value, "unit": "outer_iter/s", "cores": cores,
                            "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": "outer_iter/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def time_steps(step, stream, flush, steps):
    """CUDA-event time of `steps` calls of step() (L2 flushed before each,
    outside the events); returns (ms, outer iterations)."""
    import torch
    total_ms, total_it = 0.0, 0
    for k in range(steps):
        flush.fill_(float(k))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        total_it += step()
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
    return total_ms, total_it


def march_rate(P, fp, init, stream, flush, first=20, count=20):
    """Outer iterations per second of a developed march: from rest, steps
    0..first-1 untimed, then `count` steps timed, each with the paper's
    adaptive outer tolerance (1e-4, then min(1e-4, change)) and no rebuild."""
    for k, a in init.items():
        P.set(k, a)
    tol = [1e-4]

    def one():
        it, ch = P.time_step(fp.dt, tol[0], max_outer=20, krylov_maxit=100000)
        tol[0] = min(1e-4, ch)
        return it

    for _ in range(first):
        one()
    ms, it = time_steps(one, stream, flush, count)
    return {"value": it / (ms / 1e3), "unit": "outer_iter/s", "steps": f"{first}..{first + count - 1}",
            "outer_iters": it, "ms": ms}


def bench_extras(args, ctx, stream, fp, dev, desc_dev, init, flush, P):
    """Keys beside the headline (one GPU, rank 0): the plain FP64 GPU path on
    the same step (FP64 Jacobi BiCGSTAB for momentum and p', the paper's
    solver) and the ratio the mixed-precision path reaches against it; the
    outer-iteration rate of a developed march (no rebuild) for both paths;
    the batched workload and the request server."""
    from paper_2106_07616_gb300 import rbffd
    res = {}
    d64 = rbffd.desc_from_pointers(fp.n, fp.q, fp.degree, fp.pin, fp.rho, fp.mu, rbffd.PREC_FP64,
                                   dev["x"], dev["y"], dev["tag"], dev["nx"], dev["ny"],
                                   dev["ubc"], dev["vbc"], rbffd.PRECOND_JACOBI)
    Q = rbffd.Problem(ctx, desc=d64)

    def step64():
        Q.reload(desc=d64)
        for k, a in init.items():
            Q.set(k, a)
        it, _ = Q.time_step(fp.dt, 1e-4, max_outer=args.outer, krylov_maxit=100000)
        return it

    step64()
    n64 = max(2, min(args.steps, 3))
    ms64, it64 = time_steps(step64, stream, flush, n64)
    v64 = it64 / (ms64 / 1e3)
    res["fp64_plain"] = {
        "value": v64, "unit": "outer_iter/s", "steps": n64, "ms_per_step": ms64 / n64,
        "outer_iters_per_step": it64 / n64,
        "path": "FP64 BiCGSTAB with Jacobi for momentum and p' (the paper's solver), same step, "
                "same 1e-12 FP64 relative residual per solve"}
    P.reload(desc=desc_dev)
    Q.reload(desc=d64)
    m_mixed = march_rate(P, fp, init, stream, flush)
    m_64 = march_rate(Q, fp, init, stream, flush)
    res["march"] = {"default": m_mixed, "fp64_plain": m_64,
                    "ratio": m_mixed["value"] / m_64["value"]}
    res["north_star_ratio"] = {
        "first_step": res_ratio(v_default_step(P, desc_dev, init, fp, args, stream, flush), v64),
        "march": res["march"]["ratio"],
        "note": "mixed-precision path (FGMRES with FP32 Arnoldi and V-cycle for p', FP32 "
                "BiCGSTAB in FP64 refinement for momentum) over the plain FP64 GPU path "
                "(FP64 Jacobi BiCGSTAB for both), same step, same FP64 residual per solve"}
    Q.close()
    # the batched and served workloads, at sizes that keep this run short
    ba = argparse.Namespace(**vars(args))
    ba.count, ba.steps, ba.warmup = args.batch_count, 2, 1
    ba.precond, ba.precision = "amg", "fp64"
    b = batch_line(ba)
    res["batch"] = {k: b[k] for k in ("value", "unit", "ms_per_step", "e2e", "roofline",
                                      "krylov_p", "krylov_mom", "config", "gpu_launches",
                                      "autotune")}
    sa = argparse.Namespace(**vars(args))
    sa.count, sa.resid_tol, sa.criterion, sa.max_steps = args.serve_count, 1e-8, 0, 20000
    sa.precond, sa.precision = "amg", "fp64"
    sv = serve_line(sa, n_hi=args.serve_key_n_hi)
    res["serve"] = {k: sv[k] for k in ("p50", "p99", "unit", "solves_per_s", "requests", "ok",
                                       "failed", "failures", "resid_tol", "criterion", "wall_s",
                                       "config", "steps_ok", "R_ok")}
    return res


def res_ratio(a, b):
    return a / b if b else None


def v_default_step(P, desc_dev, init, fp, args, stream, flush):
    """The default path's step rate again, on the same flushed-L2 timing as
    the plain FP64 arm beside it."""
    def step():
        P.reload(desc=desc_dev)
        for k, a in init.items():
            P.set(k, a)
        it, _ = P.time_step(fp.dt, 1e-4, max_outer=args.outer, krylov_maxit=100000)
        return it
    ms, it = time_steps(step, stream, flush, 3)
    return it / (ms / 1e3)


def run_native(args):
    import torch
    import torch.distributed as dist

    from paper_2106_07616_gb300 import _build, rbffd

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    if rank == 0 or world == 1:
        _build.build()
    if world > 1:
        dist.barrier()
    _build.build()
    fp, desc = workload(args.workload)
    stream = torch.cuda.current_stream()
    ctx = rbffd.Context(local, stream=stream.cuda_stream)
    dev = {k: torch.from_numpy(np.ascontiguousarray(getattr(fp, k))).to(f"cuda:{local}")
           for k in ("x", "y", "tag", "nx", "ny", "ubc", "vbc")}
    prec = {"mixed": rbffd.PREC_MIXED, "ff": rbffd.PREC_MIXED_FF,
            "fp64": rbffd.PREC_FP64}[args.precision]
    init = {k: torch.from_numpy(np.ascontiguousarray(a)).to(f"cuda:{local}")
            for k, a in (fp.initial or {}).items()}
    pc = {"amg": rbffd.PRECOND_AMG, "fgmres": rbffd.PRECOND_AMG_FGMRES}.get(
        args.precond, rbffd.PRECOND_JACOBI)
    desc_dev = rbffd.desc_from_pointers(fp.n, fp.q, fp.degree, fp.pin, fp.rho, fp.mu, prec,
                                        dev["x"], dev["y"], dev["tag"], dev["nx"], dev["ny"],
                                        dev["ubc"], dev["vbc"], pc)
    P = rbffd.Problem(ctx, desc=desc_dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=f"cuda:{local}")

    def step(desc, start=None):
        P.reload(desc=desc)
        for k, a in (init if start is None else start).items():
            P.set(k, a)
        it, _ = P.time_step(fp.dt, 1e-4, max_outer=args.outer, krylov_maxit=100000)
        return it

    for _ in range(args.warmup):
        step(desc_dev)
    torch.cuda.synchronize()

    # ---- device-resident timed region
    ctx.profile(True)
    l0 = ctx.launches
    total_ms, total_it = 0.0, 0
    with ClockSampler(local) as clk:
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.fill_(float(k))  # evict L2 between steps (outside the timed events)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            total_it += step(desc_dev)
            e1.record(stream)
            e1.synchronize()
            total_ms += e0.elapsed_time(e1)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
    clocks = clk.summary()
    launches = ctx.launches - l0
    kp = ctx.kernel_stat("krylov_p")
    km = ctx.kernel_stat("krylov_mom")
    kw = ctx.kernel_stat("weights")
    kn = ctx.kernel_stat("knn")
    ko = ctx.kernel_stat("outer")
    ctx.profile(False)

    total_ms_max, all_it = combine_ranks(total_ms, total_it, f"cuda:{local}")
    value = all_it / (total_ms_max / 1e3)

    # ---- end to end through the C ABI from pinned host buffers
    host = {k: torch.from_numpy(np.ascontiguousarray(getattr(fp, k))).pin_memory()
            for k in ("x", "y", "tag", "nx", "ny", "ubc", "vbc")}
    desc_host = rbffd.desc_from_pointers(fp.n, fp.q, fp.degree, fp.pin, fp.rho, fp.mu, prec,
                                         host["x"], host["y"], host["tag"], host["nx"],
                                         host["ny"], host["ubc"], host["vbc"], pc)
    outs = [torch.empty(fp.n, dtype=torch.float64).pin_memory() for _ in range(3)]
    init_host = {k: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
                 for k, a in (fp.initial or {}).items()}
    h2d = sum(int(t.numel() * t.element_size())
              for t in list(host.values()) + list(init_host.values()))
    d2h = sum(int(t.numel() * t.element_size()) for t in outs)
    e2e_s, e2e_it = 0.0, 0
    for k in range(args.steps):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_it += step(desc_host, init_host)
        for name, o in zip(("u", "v", "p"), outs):
            P.get(name, out=o)
        e2e_s += time.perf_counter() - t0
    e2e = {"value": e2e_it / e2e_s, "unit": "outer_iter/s", "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h}

    peak, peak_src = read_peaks()
    l2_mb = fp.n * (fp.q * 12 + 8 * 8) / 1e6  # p' operator + indices + Krylov vectors
    achieved = kp["bytes"] / (kp["ms"] / 1e3) / 1e9 if kp["ms"] > 0 else 0.0
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": krylov_traffic(args.precision, args.workload, args.precond),
            "peak_source": peak_src,
            "kernel": ("k_fgmres<1024> (pressure-correction flexible GMRES(30), FP32 multigrid "
                       "V-cycle preconditioner, persistent)" if args.precond == "fgmres" else
                       "k_bicgstab_amg<1024> (pressure-correction BiCGSTAB, multigrid "
                       "V-cycle preconditioner, persistent)" if args.precond == "amg" and
                       args.precision == "fp64" else
                       {"mixed": "k_bicgstab_ir<1> (pressure-correction FP32 BiCGSTAB in FP64 "
                                "refinement)",
                       "ff": "k_bicgstab_ir<1> (pressure-correction float-float BiCGSTAB in "
                             "FP64 refinement)"}.get(
                           args.precision, "k_bicgstab<1> (pressure-correction BiCGSTAB, persistent)")),
            "launches": kp["launches"], "avg_launch_ms": kp["ms"] / max(kp["launches"], 1),
            "bytes_per_unit": (f"q(4+4)+8 (FP32 SpMV) + one FP32 V-cycle + FP32 Gram-Schmidt "
                               f"over the basis per row-step (pcorr_bytes)"
                               if args.precond == "fgmres" else
                               f"2q(8+4)+14*8 + 2 V-cycles (~2q(8+4)+64) = "
                               f"{2 * fp.q * 12 + 112 + 2 * (fp.q * 12 + 64)} B per row-iteration "
                               f"+ the coarse levels' operators"
                               if args.precond == "amg" else
                               f"2q(4+4)+14*4 = {2 * fp.q * 8 + 56} B per FP32 row-iteration"
                               if args.precision == "mixed" else
                               f"2q(8+4)+14*8 = {2 * fp.q * 12 + 112} B per row-iteration"),
            "units": kp["units"],
            "note": (f"operators and Krylov vectors of this workload (~{l2_mb:.0f} MB) "
                     f"{'stay resident in' if l2_mb < 100 else 'exceed'} the 129 MB L2 during a "
                     f"solve; achieved/peak is against HBM")}
    kernels = {
        "krylov_p": {"launches": kp["launches"], "ms": kp["ms"],
                     "GBps": achieved},
        "krylov_mom": {"launches": km["launches"], "ms": km["ms"],
                       "GBps": km["bytes"] / (km["ms"] / 1e3) / 1e9 if km["ms"] > 0 else None},
        "weights": {"launches": kw["launches"], "ms": kw["ms"],
                    "fp64_GFLOPs": kw["bytes"] / (kw["ms"] / 1e3) / 1e9 if kw["ms"] > 0 else None},
        "knn": {"launches": kn["launches"], "ms": kn["ms"]},
        "outer": {"count": ko["launches"], "ms": ko["ms"]},
    }

    extras = {}
    if rank == 0 and world == 1 and args.workload == "cavity200" and not args.no_extras:
        extras = bench_extras(args, ctx, stream, fp, dev, desc_dev, init, flush, P)

    cpu = None
    if rank == 0 and not args.no_cpu:
        t, it, cores = cpu_oracle_step(fp, args.outer)
        cpu = {"value": it / t, "unit": "outer_iter/s", "cores": cores, "kind": "oracle",
               "sample": (f"one step: oracle build (clouds, weights, CSR) + first BDF2 step "
                          f"capped at {args.outer} outer iterations ({it} run), {t:.1f} s")}

    if rank == 0:
        out = {"metric": "SIMPLE outer iters/s", "value": value, "unit": "outer_iter/s",
               "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
               "ms_per_step": total_ms_max / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None,
               "dtype": ("f32x2+f64" if args.precision == "ff" else
                         "f32+f64" if args.precision == "mixed" or args.precond == "fgmres"
                         else "f64"),
               "data": "synthetic",
               "config": {"workload": args.workload, "description": desc,
                          "outer_cap": args.outer, "outer_iters_per_step": all_it / args.steps / world,
                          "precision": args.precision, "precond": args.precond,
                          "amg_levels": P.amg_info(), "krylov_tol": 1e-12,
                          "l2": "flushed between steps (256 MB write)",
                          "parallelism": f"replicas x{world}"},
               "e2e": e2e, "gpu_launches": launches, "roofline": roof,
               "cpu_baseline": cpu, "clocks": clocks, "kernels": kernels}
        out.update(extras)
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="cavity200")
    ap.add_argument("--outer", type=int, default=20)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the plain-FP64, march, batch and serve keys of the default line")
    ap.add_argument("--count", type=int, default=None,
                    help="instances (batch, default 256) / requests (serve, default 48)")
    ap.add_argument("--resid-tol", type=float, default=1e-5)
    ap.add_argument("--criterion", type=int, default=1,
                    help="serve: 0 = steady residual R, 1 = the paper's steady error change/dt")
    ap.add_argument("--max-steps", type=int, default=1000)
    ap.add_argument("--serve-n-hi", type=float, default=20000.0,
                    help="serve: largest request (points)")
    ap.add_argument("--serve-cfl", type=float, default=0.75,
                    help="serve at a residual below 1e-6: dt = this x the point spacing")
    ap.add_argument("--batch-count", type=int, default=256,
                    help="instances of the batch key of the default line")
    ap.add_argument("--serve-key-n-hi", type=float, default=10000.0,
                    help="largest request of the serve key of the default line")
    ap.add_argument("--serve-count", type=int, default=6,
                    help="requests of the serve key of the default line")
    ap.add_argument("--precond", default=None, choices=["jacobi", "amg", "fgmres"],
                    help="preconditioner of the pressure-correction BiCGSTAB")
    ap.add_argument("--precision", default=None, choices=["mixed", "ff", "fp64"],
                    help="Krylov arithmetic: FP32 or float-float inside FP64 defect "
                         "correction, or FP64")
    args = ap.parse_args()
    # batches and the request server take FP64 members with a BiCGSTAB p'
    # solver; single problems run the mixed-precision path
    many = args.workload in ("batch", "serve")
    if args.precond is None:
        args.precond = "amg" if many else "fgmres"
    if args.precision is None:
        args.precision = "fp64" if many else "mixed"
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "serve":
        run_serve(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
