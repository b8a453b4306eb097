"""The multi-rank split of independent matrices and requests, on the CPU.

* partition_by_flops covers every matrix once, keeps batch order inside each
  share and bounds every rank's flops by the mean plus the largest matrix.
* Two gloo ranks (separate processes) each factor and solve their share with
  the host task-protocol simulator (libspchol_host); rank 0 gathers the
  solutions, which come back in batch order and match the oracle's.
* The serving dispatcher keeps a pattern on one device and balances new
  patterns by their estimated work.
"""
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest

import gridgen
import oracle
from paper_1608_00044_gb300 import build, serve, shard


@pytest.mark.parametrize("world,seed", [(1, 0), (2, 1), (3, 2), (8, 3), (40, 4)])
def test_partition_covers_and_balances(world, seed):
    rng = np.random.default_rng(seed)
    costs = rng.lognormal(10, 1.5, 33)
    parts = shard.partition_by_flops(costs, world)
    assert len(parts) == world
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(len(costs)))
    for p in parts:
        assert p == sorted(p)
    loads = [costs[p].sum() if p else 0.0 for p in parts]
    assert max(loads) <= costs.sum() / world + costs.max() + 1e-6 * costs.sum()
    if world >= len(costs):  # one matrix per rank at most
        assert all(len(p) <= 1 for p in parts)


def test_partition_is_deterministic_and_breaks_ties_by_index():
    parts = shard.partition_by_flops([5.0, 5.0, 5.0, 5.0], 2)
    assert parts == [[0, 2], [1, 3]]
    assert shard.partition_by_flops([1.0, 2.0, 3.0], 2) == shard.partition_by_flops([1.0, 2.0, 3.0], 2)


def _batch():
    sides = [6, 9, 12, 15, 7, 20, 11, 14, 8, 17]
    mats = [gridgen.diffusion_2d_5pt(s, sigma=1.0, seed=100 + i) for i, s in enumerate(sides)]
    mats += [gridgen.laplacian_3d(5), gridgen.diffusion_3d_27pt(4, sigma=2.0, seed=7)]
    perms = [gridgen.geometric_nd(A.dims) for A in mats]
    rhs = [gridgen.rhs_uniform(A.n, 1 + i % 3, seed=i) for i, A in enumerate(mats)]
    return mats, perms, rhs


def _rank_main(rank, world, port, out_q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mats, perms, rhs = _batch()
        X, summary = shard.run_sharded(mats, perms, rhs, engine="host")
        if rank == 0:
            out_q.put((X, [(s.rank, s.indices, s.rc, s.flops) for s in summary]))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_gather_in_batch_order_and_match_the_oracle():
    build.build_host()
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    X, summary = q.get()
    mats, perms, rhs = _batch()
    costs = shard.matrix_flops(mats, perms)
    parts = shard.partition_by_flops(costs, 2)
    assert [s[0] for s in summary] == [0, 1]
    for r, idx, rc, fl in summary:
        assert idx == parts[r] and rc == 0
        assert fl == pytest.approx(costs[idx].sum(), rel=1e-12)
    assert len(X) == len(mats)
    for A, p, B, Xi in zip(mats, perms, rhs, X):
        assert Xi.shape == (A.n, B.shape[1])
        f = oracle.OracleFactor.from_csc(A, p)
        assert f.factor() == 0
        Xo = f.solve(B)
        assert np.abs(Xi - Xo).max() <= 1e-12 * np.abs(Xo).max()
        assert oracle.berr(A, Xi, B) <= 1e-13


def test_single_process_runs_the_whole_batch():
    build.build_host()
    mats, perms, rhs = _batch()
    X, summary = shard.run_sharded(mats, perms, rhs, engine="host")
    assert len(summary) == 1 and summary[0].indices == list(range(len(mats)))
    for A, B, Xi in zip(mats, rhs, X):
        assert oracle.berr(A, Xi, B) <= 1e-13


def test_serving_dispatch_affinity_and_balance():
    reqs = serve.make_stream(200, rate=50.0, seed=3, patterns=24, small=True)
    where = serve.MultiServer.assign(reqs, 4)
    dev_of = {}
    for q, d in zip(reqs, where):
        assert dev_of.setdefault(q.key, d) == d  # a pattern never moves
    load = np.zeros(4)
    for q, d in zip(reqs, where):
        n, k = q.B.shape
        load[d] += (0.0 if q.repeat else n ** 1.5) + n * k
    biggest = max((q.B.shape[0] ** 1.5 + q.B.shape[0] * q.B.shape[1]) for q in reqs)
    # greedy over patterns in arrival order: no device idles while another holds the bulk
    assert load.max() - load.min() <= 8 * biggest
    assert len(set(where)) == 4
    assert serve.MultiServer.assign(reqs, 1) == [0] * len(reqs)
