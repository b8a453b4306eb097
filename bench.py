"""Benchmark: supernodal Cholesky factorization throughput on one GB300 per rank.

One step = assembly + numeric factorization + the 8-RHS forward/backward solve
of the 3D 7-point Laplacian on a 64^3 grid (n = 262,144, geometric nested
dissection), all inputs resident in HBM.  The value is factor TFLOP/s:
sum_j c_j^2 of the exact factor structure divided by the step time (the solve
is inside the step, so the number is conservative).

Flags: --gpus N --steps K --warmup W [--impl reference] [--workload NAME]
       [--width W] [--precision fp64|fp32|tf32]
Under torchrun every rank factors its own replica (the single-matrix path does
not shard); value = replicas x flops / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "factor TFLOP/s (%FP64 peak) on 64^3 Laplacian; FP32+IR speedup; p50/p99 solve"
UNIT = "TFLOP/s"
# FP64 roofline denominator: 152 SMs x 2 DFMA/clk/SM x 2 flop x SM clock.  The
# DFMA rate per SM follows from NVIDIA's 1.25 TFLOP/s FP64 figure at the
# 2070 MHz maximum clock; the DFMA throughput probe (peak_probe.cu, run by
# default, reported as roofline.peak_measured) measures 1.2545 on this GPU.
FP64_FLOP_PER_CLK = 152 * 2 * 2


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


KERNEL_SOURCES = ["factor.cu", "device_common.cuh", "sched.cuh", "kernels.hpp", "plan.hpp"]
# The warp-level subtree tasks are a kernel of their own (warp_subtree_kernel,
# which single large matrices do not launch); their section of factor.cu is
# left out of factor_kernel's sources.
WARP_SECTION = ("// ---------------------------------------------------------------- warp-level subtree tasks",
                "// MODE: 0 = CUDA-core update tiles")


def kernel_sources_sha1() -> str:
    """Digest of factor_kernel's sources (KERNEL_SOURCES, factor.cu without the
    warp-level subtree section)."""
    import hashlib

    h = hashlib.sha1()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1608_00044_gb300", "csrc", f), "rb") as fh:
            data = fh.read()
        if f == "factor.cu":
            text = data.decode()
            i = text.index(WARP_SECTION[0])
            j = text.index(WARP_SECTION[1], i)
            data = (text[:i] + text[j:]).encode()
        h.update(data)
    return h.hexdigest()


def _measured_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu capture, or None
    when the kernel's sources changed since that capture."""
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))[kernel]
        return rec["bytes_per_launch"] if kernel_sources_sha1() == rec["kernel_sources_sha1"] else None
    except Exception:
        return None


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"spchol_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        except Exception:
            rows = []
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except Exception:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower() in ("active", "1", "0x1"):
                    reasons.add(nm)
        if sm:
            out["sm_mhz"] = statistics.median(sm)
            out["sm_max_mhz"] = max(mx)
            out["samples"] = len(sm)
        out["reasons"] = sorted(reasons)
        return out


def _describe(A):
    """Human-readable name of a generated grid matrix, from its kind and dims."""
    dims = "x".join(str(d) for d in A.dims)
    return {"lap2d5": f"2D 5-point Laplacian {dims}", "lap3d7": f"3D 7-point Laplacian {dims}",
            "diff3d27": f"3D 27-point variable-coefficient diffusion {dims}",
            "diff2d5": f"2D 5-point variable-coefficient diffusion {dims}"}.get(A.kind, f"{A.kind} {dims}")


def _workload(name):
    import gridgen

    A, perm, b = gridgen.workload(name)
    return A, perm, b


def _berr(A, X, B):
    """Backward error max_c ||b_c - A x_c||_inf / (||A||_inf ||x_c||_inf + ||b_c||_inf) of a solution,
    from the full symmetric matrix with scipy (the bench's own check, not the oracle)."""
    M = A.to_scipy_full()
    X = np.asarray(X, dtype=np.float64).reshape(A.n, -1, order="F")
    B = np.asarray(B, dtype=np.float64).reshape(A.n, -1, order="F")
    R = B - M @ X
    an = float(abs(M).sum(axis=1).max()) if A.n else 0.0
    worst = 0.0
    for c in range(X.shape[1]):
        den = an * float(np.abs(X[:, c]).max(initial=0.0)) + float(np.abs(B[:, c]).max(initial=0.0))
        rn = float(np.abs(R[:, c]).max(initial=0.0))
        e = rn / den if den > 0 else (np.inf if rn > 0 else 0.0)
        if not e <= worst:
            worst = e
    return worst


def _host_cpu():
    """Model name and logical core count of the host running the bench."""
    import platform

    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    return {"model": model or platform.processor() or platform.machine(), "arch": platform.machine(),
            "nproc": os.cpu_count()}


def _oracle_sample(name, reps=1, detail=False):
    """Time the oracle (single-threaded scalar C) on a bounded sample workload:
    symbolic analysis, numeric factorization and solve, each separately."""
    import oracle

    A, perm, b = _workload(name)
    t_sym = t_num = t_sol = 0.0
    for _ in range(reps):
        t0 = time.perf_counter()
        f = oracle.OracleFactor.from_csc(A, perm)
        t1 = time.perf_counter()
        info = f.factor()
        t2 = time.perf_counter()
        x = f.solve(b)
        t3 = time.perf_counter()
        t_sym += t1 - t0
        t_num += t2 - t1
        t_sol += t3 - t2
    dt = (t_sym + t_num + t_sol) / reps
    if detail:
        return {"flops": f.flops, "total_s": dt, "symbolic_s": t_sym / reps, "numeric_s": t_num / reps,
                "solve_s": t_sol / reps, "info": info, "berr": oracle.berr(A, x, b),
                "numeric_gflops": f.flops / (t_num / reps) / 1e9 if t_num > 0 else None}
    return f.flops, dt, info, oracle.berr(A, x, b)


def _oracle_batch_worker(args):
    """One host core's share of the batch for the all-cores oracle timing: build
    its matrices, wait for the other workers, then time the oracle on them."""
    idx, sides, barrier = args
    import gridgen
    import oracle

    mats = [gridgen.diffusion_2d_5pt(int(sides[i]), sigma=1.0, seed=1000 + i) for i in idx]
    perms = [gridgen.geometric_nd(M.dims) for M in mats]
    rhs = [gridgen.rhs_uniform(M.n, 1, seed=i) for i, M in zip(idx, mats)]
    oracle.build()
    barrier.wait(600)
    t0 = time.time()
    flops = 0.0
    for M, p, b in zip(mats, perms, rhs):
        f = oracle.OracleFactor.from_csc(M, p)
        f.factor()
        f.solve(b)
        flops += f.flops
    return t0, time.time(), flops


def oracle_batch_all_cores(count=512):
    """The oracle over all host cores on the 512-matrix batch (one process per
    core, matrices split by their size, each process timing its own share after
    all have built their inputs): wall time from the first start to the last
    end, and flops over it."""
    import multiprocessing as mp

    import gridgen

    sides = gridgen.batch_sides(count)
    cores = os.cpu_count() or 1
    order = sorted(range(count), key=lambda i: -int(sides[i]) ** 3)
    load = [0] * cores
    parts = [[] for _ in range(cores)]
    for i in order:  # largest first to the least loaded core (cost ~ side^3 for 2D nested dissection)
        k = min(range(cores), key=lambda c: (load[c], c))
        parts[k].append(i)
        load[k] += int(sides[i]) ** 3
    ctx = mp.get_context("spawn")
    with ctx.Manager() as man:
        barrier = man.Barrier(cores)
        with ctx.Pool(cores) as pool:
            res = pool.map(_oracle_batch_worker, [(p, sides, barrier) for p in parts], chunksize=1)
    t0 = min(r[0] for r in res)
    t1 = max(r[1] for r in res)
    flops = sum(r[2] for r in res)
    return {"value": flops / (t1 - t0) / 1e12, "unit": UNIT, "cores": cores, "kind": "oracle",
            "seconds": t1 - t0, "flops": flops,
            "sample": f"the whole {count}-matrix batch (2D 5-point variable-coefficient grids), one process per "
                      f"host core, matrices split by size; analyze + factor + 1-RHS solve each"}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle

    oracle.build()
    sample = args.ref_sample
    for _ in range(args.warmup):
        _oracle_sample(sample)
    times, flops = [], None
    for _ in range(args.steps):
        flops, dt, info, be = _oracle_sample(sample)
        times.append(dt)
    tot = sum(times)
    value = flops * len(times) / tot / 1e12
    line = {
        "impl": "reference",
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": args.gpus,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": tot / len(times) * 1e3,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"{args.workload} (reference steps run the bounded sample {sample})",
                   "sample": sample, "nrhs": 8},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{sample}: scalar left-looking FP64 factor + 8-RHS solve, single thread",
                         "host": _host_cpu()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "berr": be,
    }
    print(json.dumps(line))
    return 0


MIXED_CANDIDATES = [(64, 4, 64), (64, 16, 64), (64, 64, 64), (32, 64, 64)]


def measure_mixed(spchol, torch, dev, name="diff3d_48", width=64, tune=True):
    """Mixed-precision row: FP64 factor+solve vs FP32 factor + solve + FP64 refinement to 1e-12,
    same matrix and right-hand side, device time of each.  Each precision runs
    with the default plan (W 64, relax 4, 64-row tiles) and with the plan the
    autotuner picks for it from the same candidates; the headline speedup
    compares the tuned runs (each mode at its best)."""
    from paper_1608_00044_gb300 import autotune

    A, perm, b = _workload(name)
    out = {"workload": f"{name}: 3D 27-point variable-coefficient diffusion {A.dims}, n={A.n}, "
                       f"log-normal kappa sigma=2 clipped (contrast 1e4), 1 RHS"}
    vals = torch.from_numpy(A.values).to(dev)
    bt = torch.from_numpy(np.ascontiguousarray(b.T)).to(dev)

    def run(prec, W, relax, tile):
        o = spchol.default_options(precision=prec, max_width=W, relax_zeros=relax, tile_rows=tile, ir_max_iter=30)
        h = spchol.analyze(A.n, A.colptr, A.rowind, perm, o)
        times, ok = [], True
        for it in range(4):
            spchol.factorize(h, vals)
            X = bt.clone()
            try:
                spchol.solve(h, X, A.n, 1)
                ok = True
            except spchol.SpcholError as e:
                if e.code != spchol.ENOCONV:
                    raise
                ok = False
            st = spchol.stats(h)
            if it >= 1:
                times.append(st["factor_ms"] + st["solve_ms"])
        be = _berr(A, np.asfortranarray(X.cpu().numpy().T), b)
        spchol.destroy(h)
        return {"ms": sum(times) / len(times), "factor_ms": st["factor_ms"], "solve_ms": st["solve_ms"],
                "berr": be, "ir_iters": st["ir_iters"], "converged": bool(ok and be <= 1e-12),
                "plan": {"max_width": W, "relax_zeros": relax, "tile_rows": tile}}

    res, tuned = {}, {}
    modes = (("fp64", spchol.FP64), ("fp32_ir", spchol.FP32), ("tf32x3_ir", spchol.TF32X3), ("tf32_ir", spchol.TF32))
    for label, prec in modes:
        W = min(width, 64) if prec >= spchol.TF32 else width
        res[label] = run(prec, W, 4, 64)
        if tune:
            cfg = autotune.tune([A], [perm], prec, candidates=MIXED_CANDIDATES, reps=2)
            tuned[label] = run(prec, cfg["max_width"], cfg["relax_zeros"], cfg["tile_rows"])
    out.update(res)
    out["flops"] = float(_flops_of(spchol, A, perm))

    def speedups(r):
        sp = {k: r["fp64"]["ms"] / v["ms"] for k, v in r.items() if k != "fp64" and v["converged"]}
        conv = [k for k in ("fp32_ir", "tf32x3_ir", "tf32_ir") if r[k]["converged"]]
        best = min(conv, key=lambda k: r[k]["ms"]) if conv else None
        return sp, best, (r["fp64"]["ms"] / r[best]["ms"] if best else None)

    # speedup of each low-precision mode that reached berr <= 1e-12, against FP64 time to its own result
    out["speedup_vs_fp64"], best, sp_default = speedups(res)
    out["default_plan_speedup"] = sp_default
    if tuned:
        out["tuned"] = tuned
        out["tuned_speedup_vs_fp64"], best, sp = speedups(tuned)
        out["fp32_ir_speedup"] = sp
    else:
        out["fp32_ir_speedup"] = sp_default
    out["best_mixed_mode"] = best
    return out


def _flops_of(spchol, A, perm):
    h = spchol.analyze(A.n, A.colptr, A.rowind, perm, spchol.default_options())
    f = spchol.stats(h)["flops"]
    spchol.destroy(h)
    return f


def measure_fp64_tc(spchol, torch, dev, A, perm, b, flops, peak_fp64, width=64, relax=4):
    """FP64 factorization of the headline matrix with the update tiles of panels
    at least 16 wide on the BF16 tensor cores (7-way digit split, FP64-accurate
    result; `SPCHOL_FP64_TC`): factor time, the same flop count over it, and the
    backward error of an 8-RHS solve."""
    o = spchol.default_options(precision=spchol.FP64_TC, max_width=min(width, 64), relax_zeros=relax)
    h = spchol.analyze(A.n, A.colptr, A.rowind, perm, o)
    vals = torch.from_numpy(A.values).to(dev)
    times = []
    for it in range(4):
        spchol.factorize(h, vals)
        if it >= 1:
            times.append(spchol.stats(h)["factor_ms"])
    X = torch.from_numpy(np.ascontiguousarray(b.T)).to(dev)
    spchol.solve(h, X, A.n, b.shape[1])
    be = _berr(A, np.asfortranarray(X.cpu().numpy().T), b)
    st = spchol.stats(h)
    spchol.destroy(h)
    ms = statistics.median(times)
    tf = flops / (ms * 1e-3) / 1e12
    return {"workload": "same matrix and right-hand sides as the headline; update tiles of panels >= 16 columns on "
                        "BF16 tensor cores (Ozaki-style 7-way split, exact products, 64-bit integer combination)",
            "factor_ms": ms, "tflops_effective": tf, "frac_of_fp64_peak": tf / peak_fp64, "berr": be,
            "solve_ms": st["solve_ms"], "grid_factor": st["grid_factor"],
            "note": "FP64-accurate (berr <= 1e-13, L within 1e-11 of the oracle in the GPU tests); flops are the "
                    "exact sum c_j^2, the same numerator as the headline"}


def measure_ordering(spchol, torch, dev, A0, perm_geo, b, flops_geo, width=64, relax=4):
    """General-ordering row: the headline matrix with its rows and columns in a
    random order (seed 11), ordered by spchol_order_nd (nested dissection by
    level structures) instead of the grid's geometric dissection: host time of
    the ordering, its exact flops against the geometric ordering's, FP64 factor
    time (median of 3) and the backward error of an 8-RHS solve."""
    import scipy.sparse as sp

    import gridgen

    q = np.random.default_rng(11).permutation(A0.n)
    L0 = sp.csc_matrix((A0.values, A0.rowind, A0.colptr), shape=(A0.n, A0.n))
    M = (L0 + sp.tril(L0, -1).T).tocsc()[q][:, q]
    L = sp.csc_matrix(sp.tril(M))
    L.sort_indices()
    A = gridgen.CscLower(A0.n, L.indptr.astype(np.int64), L.indices.astype(np.int32), L.data.astype(np.float64))
    bq = np.ascontiguousarray(b[q])
    t0 = time.perf_counter()
    perm = spchol.order_nd(A.n, A.colptr, A.rowind)
    t_order = time.perf_counter() - t0
    h = spchol.analyze(A.n, A.colptr, A.rowind, perm, spchol.default_options(max_width=width, relax_zeros=relax))
    vals = torch.from_numpy(A.values).to(dev)
    times = []
    for it in range(4):
        spchol.factorize(h, vals)
        if it >= 1:
            times.append(spchol.stats(h)["factor_ms"])
    X = torch.from_numpy(np.ascontiguousarray(bq.T)).to(dev)
    spchol.solve(h, X, A.n, bq.shape[1])
    be = _berr(A, np.asfortranarray(X.cpu().numpy().T), bq)
    st = spchol.stats(h)
    spchol.destroy(h)
    ms = statistics.median(times)
    return {"workload": "the headline matrix in a random row/column order (seed 11), ordered by spchol_order_nd",
            "order_s": t_order, "flops": st["flops"], "flops_vs_geometric_nd": st["flops"] / flops_geo,
            "nnz_l": st["nnz_l"], "factor_ms": ms, "tflops": st["flops"] / (ms * 1e-3) / 1e12, "berr": be}


def measure_amalgamation(spchol, torch, dev, A, perm, b, flops, width=64, relaxes=(0, 4, 16, 32)):
    """Amalgamation row: the headline matrix factored with other relaxed-fill
    budgets (explicit zeros per column allowed when merging supernodes; the
    configuration fixes 4).  TFLOP/s always counts the exact flops sum c_j^2,
    not the zeros' extra work, so wider merged panels pay only if they are
    faster; the stored entries show the zeros added."""
    vals = torch.from_numpy(A.values).to(dev)
    out = {"workload": "the headline matrix and right-hand sides, FP64, W 64", "runs": {}}
    for relax in relaxes:
        h = spchol.analyze(A.n, A.colptr, A.rowind, perm, spchol.default_options(max_width=width, relax_zeros=relax))
        times = []
        for it in range(3):
            spchol.factorize(h, vals)
            if it >= 1:
                times.append(spchol.stats(h)["factor_ms"])
        X = torch.from_numpy(np.ascontiguousarray(b.T)).to(dev)
        spchol.solve(h, X, A.n, b.shape[1])
        be = _berr(A, np.asfortranarray(X.cpu().numpy().T), b)
        st = spchol.stats(h)
        spchol.destroy(h)
        ms = statistics.median(times)
        out["runs"][str(relax)] = {"factor_ms": ms, "tflops": flops / (ms * 1e-3) / 1e12,
                                   "nnz_l_stored": st["nnz_l_stored"], "n_supernodes": st["n_supernodes"],
                                   "berr": be}
    return out


def measure_scheduling(spchol, torch, dev, name="lap3d_40", width=64):
    """Scheduling-policy row (the Section V-A question of which ready task runs
    first, and Section IV-B's static schedule against the dynamic one, restated
    for one GPU), with the fan-in aggregation (Section II-C's fan-in family) as
    the fast deterministic mode: the same matrix factored and solved with the
    default dynamic two rings (critical-path priority), with one FIFO ring (no
    priority), with the static (target, source) order, and with fan-in buffers;
    median factor time, solve time, backward errors, device footprint, and
    whether the first and the last factor + solve runs agree bitwise."""
    A, perm, b = _workload(name)
    vals = torch.from_numpy(A.values).to(dev)
    out = {"workload": f"{name}: 3D 7-point {A.dims}, n={A.n}, {b.shape[1]} RHS"}
    arms = (("dynamic_priority", 0, 0), ("dynamic_fifo", 0, 1), ("static", 1, 0), ("fanin", 2, 0))
    for label, det, sched in arms:
        h = spchol.analyze(A.n, A.colptr, A.rowind, perm,
                           spchol.default_options(max_width=width, deterministic=det, sched=sched))
        runs = 3 if det == 1 else 4  # the static chains take seconds at 64^3
        times, xs, s_ms = [], [], []
        for it in range(runs):
            spchol.factorize(h, vals)
            if it >= 1:
                times.append(spchol.stats(h)["factor_ms"])
            if it in (0, runs - 1):
                X = torch.from_numpy(np.ascontiguousarray(b.T)).to(dev)
                spchol.solve(h, X, A.n, b.shape[1])
                s_ms.append(spchol.stats(h)["solve_ms"])
                xs.append(X.cpu().numpy())
        be = _berr(A, np.asfortranarray(xs[0].T), b)
        fp = spchol.stats(h)["footprint_bytes"]
        spchol.destroy(h)
        out[label] = {"factor_ms": statistics.median(times), "solve_ms": min(s_ms), "berr": be,
                      "footprint_bytes": int(fp), "runs_bitwise_equal": bool(np.array_equal(xs[0], xs[1]))}
    base = out["dynamic_priority"]["factor_ms"]
    for label in ("dynamic_fifo", "static", "fanin"):
        out[f"{label}_over_priority_factor"] = out[label]["factor_ms"] / base
    return out


def measure_gmres_ir(spchol, torch, dev, nx=32, eps=1e-4, width=64):
    """GMRES-IR row: the Neumann 3D Laplacian + eps I (kappa ~ 12 / eps), where a
    TF32 factor stalls classic refinement (u_f kappa >> 1) and GMRES-IR takes
    over; time to the 1e-12 target against the plain FP64 factor + solve."""
    import gridgen

    A = gridgen.neumann_laplacian_3d(nx, eps)
    perm = gridgen.geometric_nd(A.dims)
    b = gridgen.rhs_uniform(A.n, 1, seed=0)
    vals = torch.from_numpy(A.values).to(dev)
    out = {"workload": f"Neumann 3D 7-point Laplacian {nx}^3 + {eps:g} I (kappa ~ {12 / eps:.1e}), 1 RHS"}
    for label, prec in (("fp64", spchol.FP64), ("tf32_refined", spchol.TF32)):
        h = spchol.analyze(A.n, A.colptr, A.rowind, perm, spchol.default_options(max_width=width, precision=prec))
        best = None
        for it in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rc = spchol.factorize(h, vals)
            X = b.copy(order="F")
            try:
                spchol.solve(h, X, A.n, 1)
                ok = True
            except Exception:
                ok = False
            ms = (time.perf_counter() - t0) * 1e3
            st = spchol.stats(h)
            rec = {"ms": ms, "factor_ms": st["factor_ms"], "solve_ms": st["solve_ms"], "factor_rc": rc,
                   "converged": ok, "ir_iters": st["ir_iters"], "gmres_steps": st["ir_gmres_iters"],
                   "berr": _berr(A, X, b)}
            if best is None or rec["ms"] < best["ms"]:
                best = rec
        spchol.destroy(h)
        out[label] = best
    return out


def measure_small(spchol, torch, dev, width=64):
    """Latency row: 2D 5-point 64x64 (+1e-2 I), one RHS: factor + solve time,
    median of 50 after 5 warm-ups, and the backward error."""
    A, perm, b = _workload("lap2d_64")
    h = spchol.analyze(A.n, A.colptr, A.rowind, perm, spchol.default_options(max_width=width))
    vals = torch.from_numpy(A.values).to(dev)
    bt = torch.from_numpy(np.ascontiguousarray(b.T)).to(dev)
    times, dev_ms = [], []
    for it in range(55):
        X = bt.clone()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        spchol.factorize(h, vals)
        spchol.solve(h, X, A.n, 1)
        t1 = time.perf_counter()
        st = spchol.stats(h)
        if it >= 5:
            times.append((t1 - t0) * 1e3)
            dev_ms.append(st["factor_ms"] + st["solve_ms"])
    be = _berr(A, np.asfortranarray(X.cpu().numpy().T), b)
    spchol.destroy(h)
    return {"workload": f"lap2d_64: 2D 5-point 64x64 + 1e-2 I, n={A.n}, 1 RHS", "median_ms": statistics.median(times),
            "median_device_ms": statistics.median(dev_ms), "berr": be}


def measure_batch(spchol, torch, dev, count=512, width=64):
    """Batch row: 512 independent 2D 5-point variable-coefficient grids (sides from
    default_rng(1234) in [16, 128]) factored in ONE persistent launch."""
    import gridgen

    sides = gridgen.batch_sides(count)
    mats = [gridgen.diffusion_2d_5pt(int(sd), sigma=1.0, seed=1000 + i) for i, sd in enumerate(sides)]
    perms = [gridgen.geometric_nd(M.dims) for M in mats]
    out = {"workload": f"{count} x 2D 5-point variable-coefficient grids, sides U[16,128] (rng 1234), sigma=1",
           "n_total": int(sum(M.n for M in mats))}
    from paper_1608_00044_gb300 import autotune

    for label, prec in (("fp64", spchol.FP64), ("fp32_ir", spchol.FP32)):
        tuned = autotune.tune(mats, perms, precision=prec, reps=2,
                              cache_path=os.path.join("/tmp", "spchol_autotune.json"))
        o = spchol.default_options(precision=prec, max_width=tuned["max_width"], relax_zeros=tuned["relax_zeros"],
                                   tile_rows=tuned["tile_rows"])
        t0 = time.perf_counter()
        h = spchol.batch_analyze([M.n for M in mats], [M.colptr for M in mats], [M.rowind for M in mats], perms, o)
        ana = time.perf_counter() - t0
        st0 = spchol.stats(h)
        dvals = [torch.from_numpy(M.values).to(dev) for M in mats]
        fms = []
        for it in range(4):
            rc = spchol.batch_factorize(h, dvals)
            if it >= 1:
                fms.append(spchol.stats(h)["factor_ms"])
        # the whole batch factorization captured once as a CUDA graph and replayed
        flat = torch.cat(dvals)
        cs = torch.cuda.Stream()
        cs.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(cs):
            spchol.factorize_enqueue(h, flat, stream=cs)
        cs.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=cs):
            spchol.factorize_enqueue(h, flat, stream=cs)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        gms = []
        for it in range(4):
            e0.record()
            graph.replay()
            e1.record()
            torch.cuda.synchronize()
            if spchol.factorize_status(h) != 0:
                raise RuntimeError("batch graph replay failed")
            if it >= 1:
                gms.append(e0.elapsed_time(e1))
        Bs = [gridgen.rhs_uniform(M.n, 1, seed=i) for i, M in enumerate(mats)]
        Xs = [B.copy(order="F") for B in Bs]
        try:
            spchol.batch_solve(h, Xs, [M.n for M in mats], [1] * count)
        except spchol.SpcholError:
            pass
        st = spchol.stats(h)
        worst = max(_berr(M, X, B) for M, X, B in zip(mats, Xs, Bs))
        ms = sum(fms) / len(fms)
        # algorithmic bytes of the factorization: A's values and destinations read
        # once, the stored factor (with its amalgamation zeros) written once
        esz = 4 if prec == spchol.FP32 else 8
        fbytes = st0["nnz_a"] * 16 + st0["nnz_l_stored"] * esz
        out[label] = {"factor_ms_one_launch": ms, "tflops": st0["flops"] / (ms * 1e-3) / 1e12,
                      "achieved_gbs": fbytes / (ms * 1e-3) / 1e9, "algorithmic_bytes": int(fbytes),
                      "graph_replay_ms": statistics.median(gms), "autotuned": {k: tuned[k] for k in
                      ("max_width", "relax_zeros", "tile_rows", "objective", "tried_ms", "tried_factor_ms",
                       "tried_solve_ms") if k in tuned},
                      "solve_ms": st["solve_ms"], "worst_berr": worst, "analyze_s": ana, "rc": rc,
                      "panels": st0["n_supernodes"], "tasks": st0["n_tasks"]}
        spchol.destroy(h)
    out["flops"] = float(st0["flops"])
    return out


def measure_serving(full=False, slots=4):
    """Serving row: Poisson arrivals of mixed 2D/3D problems, 30% repeat solves,
    admission by device footprint; p50/p99 latency next to solves/s.  The maximum
    throughput is measured closed-loop first, then the stream runs at fractions of it."""
    from paper_1608_00044_gb300 import serve

    n_req, warm = (2000, 200) if full else (300, 50)
    fracs = (0.25, 0.5, 0.75, 0.9)
    srv = serve.Server(slots=slots)
    # closed loop: all requests at t = 0 (warm-up part discarded)
    reqs = serve.make_stream(n_req + warm, rate=0, seed=4321)
    srv.run(reqs)
    done = sorted(reqs, key=lambda q: q.done)[warm:]
    span = done[-1].done - done[0].done
    max_tp = (len(done) - 1) / span if span > 0 else 0.0
    out = {"workload": "Poisson stream: 50% 2D (32^2..256^2) / 50% 3D (16^3..48^3), Laplacian or diffusion, "
                       "1..16 RHS, 30% repeat solves, seed 4321",
           "slots": slots, "ctas_per_sm": srv.opt_kw["ctas_per_sm"], "max_requests_per_s": max_tp,
           "budget_bytes": srv.budget, "latency": "arrival (matrix in host memory) to result on the host",
           "runs": []}
    for f in fracs:
        reqs = serve.make_stream(n_req + warm, rate=f * max_tp, seed=4321 + int(100 * f))
        srv.run(reqs)
        summ = serve.latency_summary(reqs[warm:])
        summ["rate_frac_of_max"] = f
        summ["rate_per_s"] = f * max_tp
        summ["errors"] = int(sum(q.rc not in (0,) for q in reqs))
        out["runs"].append(summ)
    out["factorizations"] = srv.factorizations
    out["peak_resident_bytes"] = srv.peak_used
    srv.close()
    return out


def measure_batch_sharded(spchol, torch, dist, count=512, width=64):
    """Multi-GPU batch row (N > 1): the 512-matrix batch split over the ranks by
    exact flops, each rank factoring and solving its share in one persistent
    launch on its own GPU, solutions gathered on rank 0.  Aggregate TFLOP/s =
    the batch's flops / the slowest rank's factorization time."""
    import gridgen
    from paper_1608_00044_gb300 import shard

    sides = gridgen.batch_sides(count)
    mats = [gridgen.diffusion_2d_5pt(int(sd), sigma=1.0, seed=1000 + i) for i, sd in enumerate(sides)]
    perms = [gridgen.geometric_nd(M.dims) for M in mats]
    rhs = [gridgen.rhs_uniform(M.n, 1, seed=i) for i, M in enumerate(mats)]
    opts = dict(max_width=32, relax_zeros=16, tile_rows=32)  # the autotuner's choice for this batch on one GPU
    costs = shard.matrix_flops(mats, perms, **opts)
    shard.run_sharded(mats, perms, rhs, engine="gpu", costs=costs, **opts)  # warm-up
    dist.barrier()
    X, summ = shard.run_sharded(mats, perms, rhs, engine="gpu", costs=costs, **opts)
    if X is None:
        return None
    worst = max(_berr(M, x, B) for M, x, B in zip(mats, X, rhs))
    slowest = max(r.factor_ms for r in summ)
    return {"ranks": len(summ), "factor_ms_slowest_rank": slowest,
            "aggregate_tflops": float(sum(costs)) / (slowest * 1e-3) / 1e12,
            "per_rank": [{"rank": r.rank, "matrices": len(r.indices), "flops": r.flops, "factor_ms": r.factor_ms}
                         for r in summ],
            "worst_berr": worst, "plan": opts}


def solve_critical_path(spchol, hostplan, A, perm, b, vals, **opts):
    """Critical path of one traced solve (profile = 2): every solve task's start
    and end, walked back from the last task to finish along the latest-finishing
    predecessor of the task protocol (forward diagonal task <- the tiles into
    the panel; forward tile <- its diagonal task, or for a W panel the tiles
    into the panel; backward tile <- the panels its rows fall in once final and
    its own panel's forward tiles, or for a W panel its diagonal task; backward
    diagonal task <- the panel's backward tiles).  Returns the path's length,
    its running and waiting time by task kind (suffix w: a W panel's task), and
    the path time by pass and depth band of 32 levels."""
    import torch
    from collections import defaultdict

    plan = hostplan.HostPlan(A.n, A.colptr, A.rowind, perm,
                             **{k: v for k, v in opts.items() if k in ("max_width", "solve_w_depth")})
    sc = plan.scalars()
    ns = sc["ns"]
    fcol = plan.get(hostplan.FCOL)
    nrows = plan.get(hostplan.NROWS)
    rowoff = plan.get(hostplan.ROWOFF)
    rows = plan.get(hostplan.ROWS)
    parent = plan.get(hostplan.PARENT)
    nst = plan.get(hostplan.NST).astype(np.int64)
    plan.close()
    NST = int(nst.sum())
    h = spchol.analyze(A.n, A.colptr, A.rowind, perm, spchol.default_options(profile=2, **opts))
    spchol.factorize(h, vals)
    bt = torch.from_numpy(np.ascontiguousarray(b.T)).cuda()
    ms = []
    for _ in range(4):
        X = bt.clone()
        spchol.solve(h, X, A.n, b.shape[1])
        ms.append(spchol.stats(h)["solve_ms"])
    tr = spchol.trace_get(h, 1).astype(np.int64)
    spchol.destroy(h)
    ran = tr[:, 1] > 0
    T = np.where(ran[:, None], (tr - tr[ran, 0].min()) / 1e3, np.nan)  # microseconds
    w = np.diff(fcol)
    depth = np.zeros(ns, np.int64)
    for s in range(ns - 1, -1, -1):
        depth[s] = 0 if parent[s] < 0 else depth[parent[s]] + 1
    isw = np.array([nst[s] > 0 and not ran[ns + 2 * NST + s] for s in range(ns)])
    st_first = np.concatenate([[0], np.cumsum(nst)[:-1]]).astype(np.int64)
    tile_s = np.repeat(np.arange(ns), nst)
    col2panel = np.searchsorted(fcol, np.arange(A.n), side="right") - 1
    ts = np.zeros(ns, np.int64)  # tile rows: the near-root band's 32, else the default 64
    for s in range(ns):
        if nst[s] > 0:
            ts[s] = 32 if depth[s] < 128 else 64
            assert (nrows[s] - w[s] + ts[s] - 1) // ts[s] == nst[s]
    tgt = []
    for kt in range(NST):
        s = tile_s[kt]
        r0 = w[s] + (kt - st_first[s]) * ts[s]
        r1 = min(nrows[s], r0 + ts[s])
        tgt.append(np.unique(col2panel[rows[rowoff[s] + r0: rowoff[s] + r1]]))
    tiles_into = [[] for _ in range(ns)]
    for kt, tt in enumerate(tgt):
        for p in tt:
            tiles_into[p].append(kt)
    end = lambda t: T[t, 1]

    def tiles_of(s, base):
        return [base + k for k in range(st_first[s], st_first[s] + nst[s])]

    def xfinal(p):
        return max(tiles_of(p, ns + NST), key=end) if isw[p] else ns + 2 * NST + p

    def preds(t):
        if t < ns:
            return tiles_of(t, ns) if isw[t] else [ns + k for k in tiles_into[t]]
        if t < ns + NST:
            s = tile_s[t - ns]
            return [ns + k for k in tiles_into[s]] if isw[s] else [s]
        if t < ns + 2 * NST:
            s = tile_s[t - ns - NST]
            return [xfinal(q) for q in tgt[t - ns - NST]] + ([s] if isw[s] else tiles_of(s, ns))
        s = t - ns - 2 * NST
        return tiles_of(s, ns + NST) if nst[s] else [s]

    path, cur = [], int(np.nanargmax(T[:, 1]))
    while cur is not None:
        path.append(cur)
        p = [q for q in preds(cur) if ran[q]]
        cur = max(p, key=end) if p else None
    path.reverse()
    kind = lambda t: "FD" if t < ns else "FT" if t < ns + NST else "BT" if t < ns + 2 * NST else "BD"
    pan = lambda t: t if t < ns else tile_s[t - ns] if t < ns + NST else tile_s[t - ns - NST] if t < ns + 2 * NST else t - ns - 2 * NST
    agg = defaultdict(lambda: [0, 0.0, 0.0])
    band = defaultdict(float)
    for j, t in enumerate(path):
        k = kind(t) + ("w" if isw[pan(t)] else "")
        gap = T[t, 0] - T[path[j - 1], 1] if j else 0.0
        agg[k][0] += 1
        agg[k][1] += T[t, 1] - T[t, 0]
        agg[k][2] += gap
        band[("forward" if kind(t)[0] == "F" else "backward") + f" depth {32 * min(depth[pan(t)] // 32, 7)}+"] += \
            T[t, 1] - T[t, 0] + gap
    return {"solve_ms_traced": [round(x, 3) for x in ms], "w_panels": int(isw.sum()),
            "makespan_us": float(np.nanmax(T[:, 1])), "path_tasks": len(path),
            "path_start_us": float(T[path[0], 0]),
            "by_kind": {k: {"tasks": v[0], "running_us": round(v[1], 1), "waiting_us": round(v[2], 1),
                            "avg_running_us": round(v[1] / v[0], 2)} for k, v in sorted(agg.items())},
            "path_us_by_pass_and_depth": {k: round(v, 1) for k, v in sorted(band.items())}}


def trace_summary(args):
    """Per-task trace of one factorization per scheduling arm (profile = 2: every
    task's start and end on the device clock), summarised: makespan, busy time
    per task type, average and starved concurrency, and the span of the top
    separator's chain of panels (the critical path near the root).  Traced runs
    are slower than untraced ones; compare the arms with each other."""
    import torch

    from __graft_entry__ import build

    build()
    from paper_1608_00044_gb300 import hostplan, spchol

    torch.cuda.set_device(0)
    A, perm, b = _workload(args.workload)
    vals = torch.from_numpy(A.values).cuda()
    prec = {"fp64": spchol.FP64, "fp32": spchol.FP32, "tf32": spchol.TF32, "tf32x3": spchol.TF32X3,
            "fp64tc": spchol.FP64_TC}[args.precision]
    out = {"mode": "trace-summary", "workload": f"{args.workload}: {_describe(A)}, n={A.n}",
           "precision": args.precision, "arms": {}}
    arms = (("dynamic_priority", 0, 0), ("dynamic_fifo", 0, 1), ("static", 1, 0), ("fanin", 2, 0))
    if args.deterministic:  # one arm only
        arms = tuple(x for x in arms if x[1] == args.deterministic)
    for label, det, sched in arms:
        kw = dict(max_width=args.width, deterministic=det, sched=sched, precision=prec)
        plan = hostplan.HostPlan(A.n, A.colptr, A.rowind, perm, **{k: v for k, v in kw.items() if k != "precision"})
        sc = plan.scalars()
        parent = plan.get(hostplan.PARENT)
        fcol = plan.get(hostplan.FCOL)
        plan.close()
        h = spchol.analyze(A.n, A.colptr, A.rowind, perm, spchol.default_options(profile=2, **kw))
        for _ in range(2):
            spchol.factorize(h, vals)
        st = spchol.stats(h)
        tr = spchol.trace_get(h, 0).astype(np.int64)
        spchol.destroy(h)
        ns, nt, nu, nsub = sc["ns"], sc["n_trsm"], sc["n_u"], sc["n_sub"]
        ran = tr[:, 1] > tr[:, 0]
        t0 = tr[ran, 0].min()
        t1 = tr[ran, 1].max()
        dur = np.where(ran, tr[:, 1] - tr[:, 0], 0)
        bounds = {"diagonal": (0, ns), "panel_solve": (ns, ns + nt), "update": (ns + nt, ns + nt + nu),
                  "subtree": (ns + nt + nu, ns + nt + nu + nsub), "gather": (ns + nt + nu + nsub, len(tr))}
        busy = {k: float(dur[a:b].sum()) / 1e6 for k, (a, b) in bounds.items() if b > a}
        # concurrency over time: +1 at each start, -1 at each end
        ev = np.concatenate([tr[ran, 0], tr[ran, 1]])
        dv = np.concatenate([np.ones(ran.sum(), np.int64), -np.ones(ran.sum(), np.int64)])
        o = np.argsort(ev, kind="stable")
        ev, conc = ev[o], np.cumsum(dv[o])
        seg = np.diff(ev)
        grid = st["grid_factor"]
        starved = float(seg[conc[:-1] < 0.1 * grid].sum()) / 1e6
        # the chain of panels from the root down through the top separator: the
        # panels whose first column lies in the root's separator block
        root = int(np.where(parent[:ns] < 0)[0].max())
        chain = [root]
        while True:
            kids = np.where(parent[:ns] == chain[-1])[0]
            if len(kids) != 1:
                break
            chain.append(int(kids[0]))
        top = chain[-1]
        span = float(tr[root, 1] - tr[top, 0]) / 1e6
        out["arms"][label] = {
            "makespan_ms": float(t1 - t0) / 1e6, "factor_ms": st["factor_ms"], "grid": grid,
            "tasks": int(ran.sum()), "busy_cta_ms": busy, "avg_concurrency": float(dur.sum()) / float(t1 - t0),
            "starved_ms_below_10pct_of_grid": starved,
            "top_chain": {"panels": len(chain), "columns": int(fcol[root + 1] - fcol[top]), "span_ms": span,
                          "diagonal_busy_ms": float(dur[chain].sum()) / 1e6}}
    if not args.deterministic and args.precision == "fp64":
        out["solve_critical_path"] = {
            f"w_depth_{d}": solve_critical_path(spchol, hostplan, A, perm, b, vals, max_width=args.width, solve_w_depth=d)
            for d in (-1, 0)}
    print(json.dumps(out))
    return 0


def run_ours(args):
    import torch

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    else:
        dist = None
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    from __graft_entry__ import build

    build()
    from paper_1608_00044_gb300 import spchol

    prec = {"fp64": spchol.FP64, "fp32": spchol.FP32, "tf32": spchol.TF32, "tf32x3": spchol.TF32X3,
            "fp64tc": spchol.FP64_TC}[args.precision]
    A, perm, b = _workload(args.workload)
    nrhs = b.shape[1]
    opt = spchol.default_options(precision=prec, max_width=args.width, relax_zeros=args.relax,
                                 deterministic=args.deterministic, profile=1 if args.profile else 0)
    h = spchol.analyze(A.n, A.colptr, A.rowind, perm, opt)
    st0 = spchol.stats(h)
    flops = st0["flops"]
    vals = torch.from_numpy(A.values).to(dev)
    b_dev = torch.from_numpy(np.ascontiguousarray(b.T)).to(dev)  # (nrhs, n) == n x nrhs column-major
    X = torch.empty_like(b_dev)
    stream = torch.cuda.current_stream()

    def step():
        rc = spchol.factorize(h, vals)
        if rc != 0:
            raise RuntimeError(f"factorize returned {rc}")
        X.copy_(b_dev)
        spchol.solve(h, X, A.n, nrhs)
        return spchol.stats(h)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    fact_ms, solve_ms = [], []
    ev0.record(stream)
    for _ in range(args.steps):
        s = step()
        fact_ms.append(s["factor_ms"])
        solve_ms.append(s["solve_ms"])
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    ck = clocks.stop()
    ms = ev0.elapsed_time(ev1) / args.steps
    t_max = torch.tensor([ms], dtype=torch.float64, device=dev)
    if dist is not None:
        dist.all_reduce(t_max, op=dist.ReduceOp.MAX)
    ms_max = float(t_max.item())
    value = ws * flops / (ms_max * 1e-3) / 1e12

    # parity of the last step's solution
    Xh = np.asfortranarray(X.cpu().numpy().T)
    be = _berr(A, Xh, b)

    # repeat solves on the resident factor: p50 / p99 latency (device time)
    lat = []
    for _ in range(args.solve_reps):
        X.copy_(b_dev)
        spchol.solve(h, X, A.n, nrhs)
        lat.append(spchol.stats(h)["solve_ms"])
    lat.sort()

    # end to end through the C-ABI with host buffers (pinned), copies inside the timed region
    vals_h = torch.from_numpy(A.values).pin_memory()
    Bh = torch.empty((nrhs, A.n), dtype=torch.float64).pin_memory()
    e2e_t = []
    for it in range(0 if args.no_e2e else args.warmup + args.steps):
        Bh.copy_(torch.from_numpy(np.ascontiguousarray(b.T)))
        t0 = time.perf_counter()
        rc = spchol.factorize(h, vals_h.numpy())
        spchol.solve(h, Bh, A.n, nrhs)
        t1 = time.perf_counter()
        if it >= args.warmup:
            e2e_t.append(t1 - t0)
    e2e_value = flops / (sum(e2e_t) / len(e2e_t)) / 1e12 if e2e_t else None
    h2d = A.nnz * 8 + A.n * nrhs * 8
    d2h = A.n * nrhs * 8

    peaks = _peaks()
    sm_mhz = ck.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    peak_fp64 = FP64_FLOP_PER_CLK * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
    fact_avg = sum(fact_ms) / len(fact_ms)
    achieved = flops / (fact_avg * 1e-3) / 1e12

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        import oracle

        oracle.build()
        d = _oracle_sample(args.cpu_sample, detail=True)
        cpu = {"value": d["flops"] / d["total_s"] / 1e12, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{args.cpu_sample}: scalar left-looking FP64 factor + 8-RHS solve, single thread, "
                         f"{d['total_s']:.1f} s, {d['flops']:.3e} flops",
               "symbolic_s": d["symbolic_s"], "numeric_s": d["numeric_s"], "solve_s": d["solve_s"],
               "numeric_only_value": d["flops"] / d["numeric_s"] / 1e12, "host": _host_cpu(),
               "note": "the oracle is a plain correctness reference, not a tuned CPU solver"}
        if not args.no_rows:
            cpu["batch_all_cores"] = oracle_batch_all_cores()
        if args.cpu_full:  # the stated configurations in full: minutes of CPU time
            cpu["full_configs"] = {nm: _oracle_sample(nm, detail=True) for nm in ("lap3d_64", "diff3d_48")}

    probe = None
    if not args.no_measure_peaks and rank == 0:
        from paper_1608_00044_gb300 import build as _b

        try:
            probe = json.loads(subprocess.run([_b.build_probe()], capture_output=True, text=True, timeout=120).stdout)
        except Exception as e:  # the probe is context, not the bench
            probe = {"error": str(e)}
    line = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": max(args.warmup, 3),
        "ms_per_step": ms_max,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"fp64": "f64", "fp32": "f32", "tf32": "tf32", "tf32x3": "tf32x3",
                  "fp64tc": "f64 (updates: bf16 tensor cores on exact 7-way split)"}[args.precision],
        "data": "synthetic",
        "config": {"workload": f"{args.workload}: {_describe(A)}, n={A.n}, nnz(lower)={A.nnz}, "
                               f"geometric ND, relax {args.relax} zeros/col, {nrhs} RHS",
                   "max_width": args.width, "relax_zeros": args.relax, "precision": args.precision, "nrhs": nrhs,
                   "order": ["dynamic", "static (target, source) chains", "fan-in buffers"][args.deterministic],
                   "l2": "inputs larger than L2 (value pool %.2f GB)" % (st0["footprint_bytes"] / 1e9),
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
        "fp64_peak_frac": value / peak_fp64,
        "factor_ms": fact_avg,
        "solve_ms": sum(solve_ms) / len(solve_ms),
        "solve_p50_ms": lat[len(lat) // 2] if lat else None,
        "solve_p99_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))] if lat else None,
        "berr": be,
        "flops": flops,
        "nnz_l": st0["nnz_l"],
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_fp64, "unit": UNIT,
                     "frac": achieved / peak_fp64,
                     "traffic": _measured_traffic("factor_kernel<double, 0, false>")
                     if args.precision == "fp64" and args.workload == "lap3d_64" and args.deterministic == 0 else None,
                     "kernel": "factor_kernel<double> (persistent; includes assembly)",
                     "peak_note": "derived: 152 SMs x 2 DFMA/clk x 2 flop x max SM clock (NVIDIA's 1.25 TFLOP/s FP64 "
                                  "figure); the probe's measured DFMA rate is in peak_measured",
                     "peak_measured": probe},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": 7 * args.steps,
        "clocks": ck,
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if not args.no_rows:
        line["small_latency_row"] = measure_small(spchol, torch, dev, width=args.width)
        if args.precision == "fp64" and args.workload == "lap3d_64":
            line["fp64_tensor_core_row"] = measure_fp64_tc(spchol, torch, dev, A, perm, b, flops,
                                                           peak_fp64, width=args.width, relax=args.relax)
            line["ordering_row"] = measure_ordering(spchol, torch, dev, A, perm, b, flops,
                                                    width=args.width, relax=args.relax)
            line["amalgamation_row"] = measure_amalgamation(spchol, torch, dev, A, perm, b, flops, width=args.width)
        line["scheduling_row"] = measure_scheduling(spchol, torch, dev, width=args.width,
                                                    name="lap3d_64" if args.workload == "lap3d_64" else "lap3d_40")
        line["mixed_precision_row"] = measure_mixed(spchol, torch, dev, width=args.width)
        line["gmres_ir_row"] = measure_gmres_ir(spchol, torch, dev, width=args.width)
        line["batch_row"] = measure_batch(spchol, torch, dev, width=args.width)
        if ws > 1:
            line["batch_row"]["sharded"] = measure_batch_sharded(spchol, torch, dist, width=args.width)
        line["serving_row"] = measure_serving(full=args.serve_full)
    if args.profile:
        sp = spchol.stats(h)
        line["task_profile"] = {k: sp[k] for k in ("factor_task_ms", "factor_task_count", "factor_wait_ms",
                                                   "factor_tc_update_ms",
                                                   "solve_task_ms", "solve_wait_ms", "grid_factor", "grid_solve",
                                                   "n_supernodes", "n_tasks", "tma_staging")}
    if rank == 0:
        print(json.dumps(line))
    spchol.destroy(h)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="lap3d_64")
    ap.add_argument("--width", type=int, default=64)
    ap.add_argument("--relax", type=int, default=4, help="amalgamation: explicit zeros allowed per column")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32", "tf32", "tf32x3", "fp64tc"])
    ap.add_argument("--solve-reps", type=int, default=50)
    ap.add_argument("--cpu-sample", default="lap3d_36")
    ap.add_argument("--ref-sample", default="lap3d_28")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end loop")
    ap.add_argument("--profile", action="store_true", help="time every task inside the persistent kernels")
    ap.add_argument("--deterministic", type=int, default=0, choices=[0, 1, 2],
                    help="order of the headline factorization: 0 dynamic, 1 static chains, 2 fan-in buffers")
    ap.add_argument("--no-rows", action="store_true", help="skip the mixed-precision, batch and serving rows")
    ap.add_argument("--no-measure-peaks", action="store_true", help="skip the DFMA / DMMA / FFMA throughput probe")
    ap.add_argument("--serve-full", action="store_true",
                    help="serving row with 2000 requests per rate after 200 warm-up (default: 300 after 50)")
    ap.add_argument("--trace-summary", action="store_true",
                    help="instead of the bench line: per-task trace summaries of the scheduling arms")
    ap.add_argument("--cpu-full", action="store_true",
                    help="also time the oracle once on the full 64^3 Laplacian and 48^3 diffusion (minutes)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.trace_summary:
        return trace_summary(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
