"""Autotuner for the panel width, amalgamation budget and update-tile rows.

For a given set of matrices (one matrix, or a batch factored in one launch) it
analyzes and factors each candidate configuration on the GPU, times the
factorization with the library's device timer (median of a few runs after one
warm-up), and returns the fastest.  Results are cached in a JSON file keyed by
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


def _digest(mats, precision: int) -> str:
    h = hashlib.sha1()
    h.update(str(precision).encode())
    for M in mats:
        h.update(np.int64(M.n).tobytes())
        h.update(np.ascontiguousarray(M.colptr, np.int64).tobytes())
        h.update(np.ascontiguousarray(M.rowind, np.int32).tobytes())
    return h.hexdigest()


def _time_config(mats, perms, precision, cfg, reps, dev_values):
    W, relax, tile = cfg
    if precision in (spchol.TF32, spchol.TF32X3, spchol.FP64_TC) and W > 64:
        return None
    opt = spchol.default_options(precision=precision, max_width=W, relax_zeros=relax, tile_rows=min(tile, 64))
    if len(mats) == 1:
        h = spchol.analyze(mats[0].n, mats[0].colptr, mats[0].rowind, perms[0], opt)
        run = lambda: spchol.factorize(h, dev_values[0])
    else:
        h = spchol.batch_analyze([M.n for M in mats], [M.colptr for M in mats], [M.rowind for M in mats],
                                 perms, opt)
        run = lambda: spchol.batch_factorize(h, dev_values)
    try:
        run()
        times = []
        for _ in range(reps):
            if run() != 0:
                return None
            times.append(spchol.stats(h)["factor_ms"])
        return statistics.median(times)
    finally:
        spchol.destroy(h)


def tune(mats, perms, precision: int = spchol.FP64, candidates=None, reps: int = 3,
         cache_path: str | None = None) -> dict:
    """Best (max_width, relax_zeros, tile_rows) for factoring `mats` (lower CSC
    matrices) with `perms`, and the time of every candidate tried."""
    import torch

    key = _digest(mats, precision)
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
    results = {}
    for cfg in candidates or DEFAULT_CANDIDATES:
        ms = _time_config(mats, perms, precision, cfg, reps, dev_values)
        if ms is not None:
            results[",".join(map(str, cfg))] = ms
    best = min(results, key=results.get)
    W, relax, tile = (int(x) for x in best.split(","))
    out = {"max_width": W, "relax_zeros": relax, "tile_rows": min(tile, 64), "factor_ms": results[best],
           "tried_ms": results, "cached": False}
    if cache_path:
        cache[key] = {k: v for k, v in out.items() if k != "cached"}
        tmp = cache_path + f".{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, cache_path)
    return out
