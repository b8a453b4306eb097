"""The per-rank GPU path of the multi-GPU batch split, on one GPU.

Each rank factors its share of a batch in one persistent launch of its own.
Here the two shares of a two-rank partition run one after the other on the one
GPU (the launches never wait on each other), and each matrix's solution must be
bitwise the one of the whole batch in a single launch (deterministic fan-in
mode: a matrix's sums land in the same order whatever else is in the launch),
with backward error <= 1e-13 against the oracle's definition.  The serving
dispatcher with one device is the plain server.
"""
import numpy as np
import pytest

import gridgen
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1608_00044_gb300 import serve, shard  # noqa: E402


def test_two_shares_equal_the_whole_batch():
    sides = gridgen.batch_sides(24)
    mats = [gridgen.diffusion_2d_5pt(int(s), sigma=1.0, seed=1000 + i) for i, s in enumerate(sides)]
    perms = [gridgen.geometric_nd(A.dims) for A in mats]
    rhs = [gridgen.rhs_uniform(A.n, 1 + i % 4, seed=i) for i, A in enumerate(mats)]
    X_all, summ = shard.run_sharded(mats, perms, rhs, engine="gpu", deterministic=2)
    assert summ[0].rc == 0 and summ[0].indices == list(range(len(mats)))
    costs = shard.matrix_flops(mats, perms, deterministic=2)
    parts = shard.partition_by_flops(costs, 2)
    assert abs(costs[parts[0]].sum() - costs[parts[1]].sum()) <= costs.max()
    for p in parts:
        r = shard.factor_solve_share(mats, perms, rhs, p, engine="gpu", deterministic=2)
        assert r.rc == 0 and r.flops == pytest.approx(costs[p].sum(), rel=1e-12)
        for i, X in zip(p, r.X):
            assert np.array_equal(X, X_all[i])
    for A, B, X in zip(mats, rhs, X_all):
        assert oracle.berr(A, X, B) <= 1e-13


def test_multiserver_on_one_device():
    reqs = serve.make_stream(16, rate=0, seed=21, patterns=5, small=True)
    ms = serve.MultiServer([0], slots=2)
    ms.run(reqs)
    assert all(q.rc == 0 for q in reqs)
    for q in reqs:
        A, _ = q.make()
        assert oracle.berr(A, q.X, q.B) <= 1e-13
    ms.close()
