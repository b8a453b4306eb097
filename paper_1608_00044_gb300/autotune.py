"""Autotuner for the panel width, amalgamation budget and update-tile rows.

For a given set of matrices (one matrix, or a batch factored in one launch) it
analyzes and factors each candidate configuration on the GPU, times the
factorization and a one-right-hand-side solve with the library's device timer
(medians of a few runs after one warm-up), and returns the configuration with
the shortest time to a solution (objective "solution"; "factor": the
factorization alone).  The two can disagree: a plan of many narrow panels
factors a batch of small matrices fastest but makes its solve a long chain of
small tasks.  Results are cached in a JSON file keyed by
a digest of the sparsity patterns and the precision, so a workload is tuned
once per machine.
"""
from __future__ import annotations

import hashlib
import json
import os
import statistics

import numpy as np

from . import spchol

DEFAULT_CANDIDATES = [
    # (max_width, relax_zeros, tile_rows)
    (64, 4, 64),
    (64, 16, 64),
    (64, 64, 64),
    (32, 8, 16),
    (32, 16, 32),
    (32, 64, 64),
    (128, 64, 64),
    (16, 16, 32),
]


def _digest(mats, precision: int, objective: str = "factor") -> str:
    h = hashlib.sha1()
    h.update(str(precision).encode())
    if objective != "factor":
        h.update(objective.encode())
    for M in mats:
        h.update(np.int64(M.n).tobytes())
        h.update(np.ascontiguousarray(M.colptr, np.int64).tobytes())
        h.update(np.ascontiguousarray(M.rowind, np.int32).tobytes())
    return h.hexdigest()


def _time_config(mats, perms, precision, cfg, reps, dev_values, objective="solution"):
    """(objective time, factorization ms, solve ms) of one configuration, or None."""
    W, relax, tile = cfg
    if precision in (spchol.TF32, spchol.TF32X3, spchol.FP64_TC) and W > 64:
        return None
    opt = spchol.default_options(precision=precision, max_width=W, relax_zeros=relax, tile_rows=min(tile, 64))
    rhs = [np.ones((M.n, 1), order="F") for M in mats]
    if len(mats) == 1:
        h = spchol.analyze(mats[0].n, mats[0].colptr, mats[0].rowind, perms[0], opt)
        run = lambda: spchol.factorize(h, dev_values[0])

        def solve():
            X = rhs[0].copy(order="F")
            spchol.solve(h, X, mats[0].n, 1)
    else:
        h = spchol.batch_analyze([M.n for M in mats], [M.colptr for M in mats], [M.rowind for M in mats],
                                 perms, opt)
        run = lambda: spchol.batch_factorize(h, dev_values)

        def solve():
            Xs = [B.copy(order="F") for B in rhs]
            spchol.batch_solve(h, Xs, [M.n for M in mats], [1] * len(mats))
    try:
        run()
        times, stimes = [], []
        for _ in range(reps):
            if run() != 0:
                return None
            times.append(spchol.stats(h)["factor_ms"])
            if objective == "solution":
                try:
                    solve()
                except spchol.SpcholError as e:
                    if e.code != spchol.ENOCONV:
                        raise
                stimes.append(spchol.stats(h)["solve_ms"])
        f = statistics.median(times)
        sv = statistics.median(stimes) if stimes else 0.0
        return f + sv, f, sv
    finally:
        spchol.destroy(h)


def tune(mats, perms, precision: int = spchol.FP64, candidates=None, reps: int = 3,
         cache_path: str | None = None, objective: str = "solution") -> dict:
    """Best (max_width, relax_zeros, tile_rows) for `mats` (lower CSC matrices)
    with `perms` under the objective ("solution": factorization + a
    one-right-hand-side solve; "factor": the factorization), and the objective
    time of every candidate tried (tried_ms; tried_factor_ms, tried_solve_ms
    the parts)."""
    if objective not in ("solution", "factor"):
        raise ValueError("objective must be 'solution' or 'factor'")
    import torch

    key = _digest(mats, precision, objective)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        try:
            with open(cache_path) as f:
                cache = json.load(f)
        except Exception:
            cache = {}
        if key in cache:
            out = dict(cache[key])
            out["cached"] = True
            return out
    dev_values = [torch.from_numpy(np.ascontiguousarray(M.values)).cuda() for M in mats]
    results, fparts, sparts = {}, {}, {}
    for cfg in candidates or DEFAULT_CANDIDATES:
        r = _time_config(mats, perms, precision, cfg, reps, dev_values, objective)
        if r is not None:
            k = ",".join(map(str, cfg))
            results[k], fparts[k], sparts[k] = r
    best = min(results, key=results.get)
    W, relax, tile = (int(x) for x in best.split(","))
    out = {"max_width": W, "relax_zeros": relax, "tile_rows": min(tile, 64), "objective": objective,
           "objective_ms": results[best], "factor_ms": fparts[best], "solve_ms": sparts[best],
           "tried_ms": results, "tried_factor_ms": fparts, "tried_solve_ms": sparts, "cached": False}
    if cache_path:
        cache[key] = {k: v for k, v in out.items() if k != "cached"}
        tmp = cache_path + f".{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, cache_path)
    return out
