"""Independent matrices split over the GPUs of one node, one rank per GPU.

A single factorization stays on one GPU: sharding it would need the paper's
fan-both exchange of update blocks between the owners of subtrees and of the
top separators (Sections III-B and IV), so on one-GPU machines it runs as
replicas.  Independent matrices -- a batch, or the requests of a serving
stream -- need no exchange at all: each rank factors and solves its share on
its own GPU (for a batch, in one persistent launch) and the results are
gathered on the host.  The partition balances the exact factorization flops
(sum over columns of c_j^2, from the host symbolic analysis, the same on every
rank, so no communication is needed to agree on it).

No collective touches the data path; the only exchange is the host-side
gather of the solutions (``torch.distributed.gather_object``) after every rank
has finished.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np


def partition_by_flops(costs, world: int) -> list[list[int]]:
    """Split items of the given costs over `world` ranks (greedy longest first).

    Items are taken in decreasing cost (ties: lower index first) and each goes to
    the rank with the least total so far (ties: lower rank).  Every rank's
    total then exceeds the mean by at most the largest single cost.  Each
    rank's list is in increasing item order (batch order).
    """
    if world < 1:
        raise ValueError("world must be >= 1")
    costs = np.asarray(costs, dtype=np.float64)
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * world
    parts: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += float(costs[i])
    return [sorted(p) for p in parts]


def matrix_flops(mats, perms, **options) -> np.ndarray:
    """Exact factorization flops of each matrix under the plan options, from the
    host symbolic analysis (libspchol_host: the analysis the GPU library runs)."""
    from . import hostplan

    out = np.empty(len(mats), np.float64)
    for i, (A, p) in enumerate(zip(mats, perms)):
        plan = hostplan.HostPlan(A.n, A.colptr, A.rowind, p, **options)
        out[i] = plan.flops
        plan.close()
    return out


@dataclasses.dataclass
class ShareResult:
    rank: int
    indices: list            # batch positions this rank factored, increasing
    X: list                  # solutions, in the order of `indices`
    rc: int                  # 0, or the first failing factorization's code
    factor_ms: float         # device time of the share's factorization (host engine: wall time)
    flops: float             # exact flops of the share


def factor_solve_share(mats, perms, rhs, indices, engine: str = "gpu", **options) -> ShareResult:
    """Factor and solve the matrices at `indices` on this rank.

    engine "gpu": one batch handle of libspchol on the current CUDA device (one
    persistent launch for the whole share), host buffers in and out.
    engine "host": the host task-protocol simulator of libspchol_host, matrix by
    matrix (for CPU-only runs of the multi-rank path).
    """
    indices = list(indices)
    if not indices:
        return ShareResult(-1, [], [], 0, 0.0, 0.0)
    if engine == "gpu":
        from . import spchol

        sub = [mats[i] for i in indices]
        opt = spchol.default_options(**options)
        h = spchol.batch_analyze([A.n for A in sub], [A.colptr for A in sub], [A.rowind for A in sub],
                                 [perms[i] for i in indices], opt)
        try:
            flops = spchol.stats(h)["flops"]
            rc = spchol.batch_factorize(h, [np.ascontiguousarray(A.values) for A in sub])
            factor_ms = spchol.stats(h)["factor_ms"]
            Xs = [np.array(rhs[i], dtype=np.float64, order="F", copy=True) for i in indices]
            Xs = [X.reshape(-1, 1, order="F") if X.ndim == 1 else X for X in Xs]
            if rc == 0:
                try:
                    spchol.batch_solve(h, Xs, [A.n for A in sub], [X.shape[1] for X in Xs])
                except spchol.SpcholError as e:
                    if e.code != spchol.ENOCONV:
                        raise
        finally:
            spchol.destroy(h)
        return ShareResult(-1, indices, Xs, int(rc), float(factor_ms), float(flops))
    if engine == "host":
        from . import hostplan

        Xs, rc, flops = [], 0, 0.0
        t0 = time.perf_counter()
        for i in indices:
            A = mats[i]
            plan = hostplan.HostPlan(A.n, A.colptr, A.rowind, perms[i], **options)
            flops += plan.flops
            r, X, _ = plan.simulate(A.values, rhs[i], seed=i)
            plan.close()
            if r != 0 and rc == 0:
                rc = int(r)
            Xs.append(X)
        return ShareResult(-1, indices, Xs, rc, (time.perf_counter() - t0) * 1e3, flops)
    raise ValueError(f"unknown engine {engine!r}")


def run_sharded(mats, perms, rhs, engine: str = "gpu", group=None, costs=None, **options):
    """Every rank of the (initialised) default process group, or of `group`, runs
    its share; rank 0 returns (X list in batch order, list of ShareResult per
    rank without the solutions), the other ranks (None, None).  Without an
    initialised process group the whole batch runs on this process.

    costs: per-matrix flops (default: ``matrix_flops`` of the same options).
    """
    import torch.distributed as dist

    dist_on = dist.is_available() and dist.is_initialized()
    world = dist.get_world_size(group) if dist_on else 1
    rank = dist.get_rank(group) if dist_on else 0
    if costs is None:
        costs = matrix_flops(mats, perms, **{k: v for k, v in options.items()
                                             if k in ("max_width", "relax_zeros", "tile_rows", "precision",
                                                      "deterministic")})
    parts = partition_by_flops(costs, world)
    res = factor_solve_share(mats, perms, rhs, parts[rank], engine=engine, **options)
    res.rank = rank
    if world == 1:
        gathered = [res]
    else:
        gathered = [None] * world if rank == 0 else None
        dist.gather_object(res, gathered, dst=0, group=group)
    if rank != 0:
        return None, None
    X = [None] * len(mats)
    for r in gathered:
        for i, x in zip(r.indices, r.X):
            X[i] = x
    summary = [ShareResult(r.rank, r.indices, [], r.rc, r.factor_ms, r.flops) for r in gathered]
    return X, summary
