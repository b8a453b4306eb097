"""Serving: continuous batching with footprint admission and resident factors.

Each request's result must be the same alone and in the mix, within the FP64
tolerance (the update order differs between runs, so equality is up to
rounding): backward error <= 1e-13 for both, and relative difference of the
solutions <= 1e-10.  Admission never exceeds the memory budget; repeat solves
reuse the resident factor (no extra factorization)."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1608_00044_gb300 import serve, spchol  # noqa: E402


def _matrix(req):
    A, perm = req.make()
    return A


def test_alone_equals_in_the_mix():
    reqs = serve.make_stream(36, rate=0, seed=7, patterns=10, small=True)
    mix = serve.Server(slots=4)
    mix.run(reqs)
    assert all(q.rc == 0 for q in reqs)
    fresh = {q.vkey for q in reqs if not q.repeat}
    # every fresh request factors once; a repeat refactors only if its values were replaced meanwhile
    assert len(fresh) <= mix.factorizations <= len(fresh) + sum(q.repeat for q in reqs)
    assert mix.peak_used <= mix.budget
    mix.close()
    alone_reqs = serve.make_stream(36, rate=0, seed=7, patterns=10, small=True)
    for q in alone_reqs:
        s1 = serve.Server(slots=1)
        s1.run([q])
        s1.close()
    for qm, qa in zip(reqs, alone_reqs):
        A = _matrix(qm)
        assert oracle.berr(A, qm.X, qm.B) <= 1e-13
        assert oracle.berr(A, qa.X, qa.B) <= 1e-13
        rel = np.abs(qm.X - qa.X).max() / max(np.abs(qa.X).max(), 1e-300)
        assert rel <= 1e-10, rel


def test_admission_respects_a_small_budget():
    reqs = serve.make_stream(30, rate=0, seed=11, patterns=12, small=True)
    # footprint of the largest single problem, times three: forces evictions
    fps = []
    for q in {q.key: q for q in reqs}.values():
        A, perm = q.make()
        h = spchol.analyze(A.n, A.colptr, A.rowind, perm, spchol.default_options(ctas_per_sm=1))
        fps.append(spchol.stats(h)["footprint_bytes"])
        spchol.destroy(h)
    budget = 3 * max(fps) + 16 * 10**6
    s = serve.Server(slots=3, budget_bytes=budget)
    s.run(reqs)
    assert s.peak_used <= budget
    assert all(q.rc == 0 for q in reqs)
    for q in reqs:
        assert oracle.berr(_matrix(q), q.X, q.B) <= 1e-13
    s.close()


def test_repeat_solves_reuse_the_resident_factor():
    reqs = serve.make_stream(20, rate=0, seed=5, patterns=3, small=True, repeat_frac=0.0)
    s = serve.Server(slots=1)
    s.run(reqs)
    before = s.factorizations
    last = {}
    for q in reqs:  # one slot: requests ran in arrival order, so the last one per pattern is resident
        last[q.key] = q
    again = [serve.Request(100 + i, 0.0, q.key, q.vkey, q.make, q.B, repeat=True)
             for i, q in enumerate(last.values())]
    s.run(again)
    assert s.factorizations == before  # the last factor of each pattern is still resident
    for q in again:
        assert oracle.berr(_matrix(q), q.X, q.B) <= 1e-13
    s.close()


def test_poisson_stream_latency_summary():
    reqs = serve.make_stream(24, rate=200.0, seed=3, patterns=8, small=True)
    s = serve.Server(slots=3)
    s.run(reqs)
    out = serve.latency_summary(reqs)
    s.close()
    assert out["requests"] == 24 and out["p99_ms"] >= out["p50_ms"] > 0
    assert all(q.done >= q.arrival for q in reqs)


def test_request_larger_than_the_budget_is_rejected_not_hung():
    # a budget smaller than any single footprint: every request is refused with
    # ENOMEM at once (the slot does not wait for memory that can never free up)
    reqs = serve.make_stream(6, rate=0, seed=13, patterns=3, small=True)
    s = serve.Server(slots=2, budget_bytes=4096)
    s.run(reqs)
    assert all(q.rc == spchol.ENOMEM for q in reqs)
    assert s.rejected == len(reqs) and s.used == 0 and not s.resident
    s.close()


def test_repeat_solve_with_more_rhs_stays_inside_the_budget():
    # the footprint charged at admission covers the largest workspace a request
    # may bring, so repeat solves with up to max_nrhs right-hand sides fit
    reqs = serve.make_stream(12, rate=0, seed=17, patterns=2, small=True, repeat_frac=0.5)
    s = serve.Server(slots=2, max_nrhs=16)
    s.run(reqs)
    assert all(q.rc == 0 for q in reqs)
    for r in s.resident.values():
        st = spchol.stats(r.h)
        assert r.footprint >= st["footprint_bytes"] + 2 * st["n"] * 16 * 8
    assert s.peak_used <= s.budget
    s.close()
