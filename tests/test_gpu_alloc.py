"""Device memory of a handle: the caller's allocator hook and the stream-ordered default.

* A handle whose memory comes from PyTorch's caching allocator (through
  spchol_options.dev_alloc / dev_free) gives bitwise the factor and solution of
  a handle on the default memory pool (deterministic fan-in mode, whose sums
  land in one fixed order), holds its footprint in torch's cache while it lives
  and returns all of it on destroy, also across solves that grow the workspace.
* Neither spchol_destroy nor a solve that grows its workspace waits for work
  on other streams: with a long factorization in flight on one stream, another
  handle is destroyed and the call returns while that stream is still busy
  (cudaFree would have waited for it).
* An allocator that fails makes analyze and solve return SPCHOL_ENOMEM and
  leaks nothing.
* Two slots: one handle's factorization in flight while the other evicts and
  grows its workspace; each result equals its solo run bitwise.
* The one-ring FIFO schedule (sched = 1) gives the same factor up to rounding
  (FP64, FP32, FP64_TC) and, in the fan-in mode, bitwise the same factor and
  solution as the priority rings.
"""
import threading
import time

import numpy as np
import pytest

import gridgen
import oracle
from tests.gpu_util import BERR_FP64, gpu_factor_solve, l_max_diff

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1608_00044_gb300 import spchol  # noqa: E402


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _solve_dev(h, B, stream=None):
    Bt = _dev(np.asfortranarray(B).T)  # (nrhs, n) row-major == n x nrhs column-major
    spchol.solve(h, Bt, B.shape[0], B.shape[1], stream=stream)  # returns with its stream complete
    return np.asfortranarray(Bt.cpu().numpy().T)


def _factor(A, perm, **opt):
    h = spchol.analyze(A.n, A.colptr, A.rowind, perm, spchol.default_options(**opt))
    assert spchol.factorize(h, _dev(A.values)) == 0
    return h


def test_torch_allocator_bitwise_and_accounting():
    alloc = spchol.torch_allocator()
    A, perm, _ = gridgen.workload("lap3d_14")
    held0 = alloc.held_bytes()
    ref = _factor(A, perm, deterministic=2)
    h = _factor(A, perm, deterministic=2, allocator="torch")
    st = spchol.stats(h)
    # the whole footprint lives in torch's cache (plus rounding to 256 bytes per block)
    assert alloc.held_bytes() - held0 >= st["footprint_bytes"]
    Lr = spchol.export_factor(ref)
    Lh = spchol.export_factor(h)
    assert np.array_equal(Lr[2], Lh[2]) and np.array_equal(Lr[1], Lh[1])
    grown = []
    for nrhs, seed in ((1, 1), (5, 2), (12, 3), (2, 4)):  # the workspace grows twice
        B = gridgen.rhs_uniform(A.n, nrhs, seed=seed)
        Xr = _solve_dev(ref, B)
        Xh = _solve_dev(h, B)
        assert np.array_equal(Xr, Xh)
        assert oracle.berr(A, Xh, B) <= BERR_FP64
        grown.append(alloc.held_bytes())
    assert grown[2] > grown[0]  # the 12-column workspace came from the cache too
    spchol.destroy(h)
    spchol.destroy(ref)
    assert alloc.held_bytes() == held0


@pytest.mark.parametrize("allocator", [None, "torch"])
def test_destroy_does_not_wait_for_other_streams(allocator):
    big, bperm, _ = gridgen.workload("lap3d_40")  # a factorization of tens of milliseconds
    small, sperm, _ = gridgen.workload("lap3d_10")
    hb = spchol.analyze(big.n, big.colptr, big.rowind, bperm, spchol.default_options(allocator=allocator))
    hs = _factor(small, sperm, allocator=allocator)
    _solve_dev(hs, gridgen.rhs_uniform(small.n, 4, seed=1))  # it holds a workspace too
    vals = _dev(big.values)
    sa = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(sa):
        spchol.factorize_enqueue(hb, vals, stream=sa)
    t0 = time.perf_counter()
    spchol.destroy(hs)
    dt = time.perf_counter() - t0
    busy = not sa.query()  # still factoring: destroy did not wait for the stream
    sa.synchronize()
    assert spchol.factorize_status(hb) == 0
    spchol.destroy(hb)
    assert busy, f"destroy returned after the other stream finished ({dt * 1e3:.2f} ms)"
    assert dt < 5e-3, dt


def test_failing_allocator_returns_enomem_without_leaks():
    import ctypes

    base = spchol.torch_allocator()
    state = {"left": 0, "live": {}, "bad_free": 0}

    def alloc(nbytes, stream, ctx):
        if state["left"] <= 0:
            return None
        state["left"] -= 1
        p = base._alloc(nbytes, stream, ctx)
        if p:
            state["live"][p] = nbytes
        return p

    def free(ptr, nbytes, stream, ctx):  # (an exception here would not reach the test)
        if state["live"].pop(int(ptr), None) != nbytes:
            state["bad_free"] += 1
        base._free(ptr, nbytes, stream, ctx)

    acb, fcb = spchol.DEV_ALLOC_FN(alloc), spchol.DEV_FREE_FN(free)
    A, perm, _ = gridgen.workload("lap3d_10")

    def opts():
        o = spchol.default_options()
        o.dev_alloc = ctypes.cast(acb, ctypes.c_void_p).value
        o.dev_free = ctypes.cast(fcb, ctypes.c_void_p).value
        return o

    for budget in (0, 1, 3):  # fail at the first, second and fourth allocation of analyze
        state["left"] = budget
        with pytest.raises(spchol.SpcholError) as e:
            spchol.analyze(A.n, A.colptr, A.rowind, perm, opts())
        assert e.value.code == spchol.ENOMEM
        assert state["live"] == {}
    # analyze succeeds; the solve's workspace allocation fails, then succeeds
    state["left"] = 1000
    h = spchol.analyze(A.n, A.colptr, A.rowind, perm, opts())
    assert spchol.factorize(h, _dev(A.values)) == 0
    state["left"] = 0
    B = gridgen.rhs_uniform(A.n, 2, seed=5)
    with pytest.raises(spchol.SpcholError) as e:
        _solve_dev(h, B)
    assert e.value.code == spchol.ENOMEM
    state["left"] = 1000
    X = _solve_dev(h, B)
    assert oracle.berr(A, X, B) <= BERR_FP64
    spchol.destroy(h)
    assert state["live"] == {} and state["bad_free"] == 0


def test_only_one_of_the_hooks_is_rejected():
    import ctypes

    acb = spchol.DEV_ALLOC_FN(lambda n, s, c: None)
    o = spchol.default_options()
    o.dev_alloc = ctypes.cast(acb, ctypes.c_void_p).value
    A = gridgen.laplacian_2d(4)
    with pytest.raises(spchol.SpcholError) as e:
        spchol.analyze(A.n, A.colptr, A.rowind, None, o)
    assert e.value.code == -5


def test_two_slots_eviction_and_growth_during_a_factorization():
    # slot 1 factors a large matrix; slot 2, meanwhile, cycles small handles
    # through factor, solves with growing nrhs and destroy.  Fan-in mode: every
    # result is bitwise that of its solo run.
    big, bperm, _ = gridgen.workload("lap3d_32")
    small, sperm, _ = gridgen.workload("lap3d_12")
    Bb = gridgen.rhs_uniform(big.n, 3, seed=9)
    solo_big = _factor(big, bperm, deterministic=2, allocator="torch")
    Xb_solo = _solve_dev(solo_big, Bb)
    spchol.destroy(solo_big)
    rhs = [gridgen.rhs_uniform(small.n, k, seed=20 + k) for k in (1, 4, 9, 16)]
    solo_small = _factor(small, sperm, deterministic=2, allocator="torch")
    Xs_solo = [_solve_dev(solo_small, B) for B in rhs]
    spchol.destroy(solo_small)

    out = {}

    def slot_big():
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            h = spchol.analyze(big.n, big.colptr, big.rowind, bperm,
                               spchol.default_options(deterministic=2, allocator="torch"))
            for _ in range(3):
                assert spchol.factorize(h, _dev(big.values), stream=s) == 0
            out["big"] = _solve_dev(h, Bb, stream=s)
            spchol.destroy(h)

    def slot_small():
        s = torch.cuda.Stream()
        res = []
        with torch.cuda.stream(s):
            for _ in range(4):
                h = spchol.analyze(small.n, small.colptr, small.rowind, sperm,
                                   spchol.default_options(deterministic=2, allocator="torch"))
                assert spchol.factorize(h, _dev(small.values), stream=s) == 0
                res.append([_solve_dev(h, B, stream=s) for B in rhs])  # nrhs 1 -> 16: three growths
                spchol.destroy(h)  # an eviction
        out["small"] = res

    ths = [threading.Thread(target=slot_big), threading.Thread(target=slot_small)]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    assert np.array_equal(out["big"], Xb_solo)
    for res in out["small"]:
        for X, Xs in zip(res, Xs_solo):
            assert np.array_equal(X, Xs)


@pytest.mark.parametrize("name,precision,l_tol", [
    ("lap3d_16", spchol.FP64, 1e-11),
    ("diff3d_10", spchol.FP64, 1e-11),
    ("lap3d_16", spchol.FP64_TC, 1e-11),
    ("lap3d_16", spchol.FP32, 1e-5),
])
def test_fifo_schedule_parity(name, precision, l_tol):
    A, perm, B = gridgen.workload(name)
    rc, X, st, h = gpu_factor_solve(A, perm, B, precision=precision, sched=1)
    assert rc == 0
    assert oracle.berr(A, X, B) <= (BERR_FP64 if precision in (spchol.FP64, spchol.FP64_TC) else 1e-12)
    d, lmax = l_max_diff(h, A)
    assert d <= l_tol * lmax, (d, lmax)
    spchol.destroy(h)


@pytest.mark.parametrize("precision", [spchol.FP64, spchol.FP64_TC])
def test_fifo_fanin_bitwise_equals_priority_fanin(precision):
    A, perm, B = gridgen.workload("lap3d_18")
    res = []
    for sched in (0, 1):
        rc, X, st, h = gpu_factor_solve(A, perm, B, precision=precision, deterministic=2, sched=sched)
        assert rc == 0
        res.append((spchol.export_factor(h)[2], X))
        spchol.destroy(h)
    assert np.array_equal(res[0][0], res[1][0])
    assert np.array_equal(res[0][1], res[1][1])


def test_torch_allocator_with_gmres_refinement_and_growth():
    # A TF32 factor in the static order with one classic refinement step
    # allowed: GMRES-IR takes over and allocates its Krylov workspace during the
    # solve; with the PyTorch allocator the results are bitwise those of the
    # default pool, and the handle returns every byte on destroy.
    alloc = spchol.torch_allocator()
    held0 = alloc.held_bytes()
    A, perm, _ = gridgen.workload("lap3d_16")
    res = []
    for allocator in (None, "torch"):
        out = []
        rc, X, st, h = gpu_factor_solve(A, perm, gridgen.rhs_uniform(A.n, 3, seed=2), precision=spchol.TF32,
                                        deterministic=1, ir_max_iter=1, allocator=allocator)
        assert rc == 0 and st["ir_gmres_iters"] > 0
        out.append(X)
        B9 = gridgen.rhs_uniform(A.n, 9, seed=4)  # more right-hand sides: the workspace grows
        X9 = B9.copy(order="F")
        spchol.solve(h, X9, A.n, 9)
        out.append(X9)
        res.append(out)
        spchol.destroy(h)
    for a_, b_ in zip(res[0], res[1]):
        assert np.array_equal(a_, b_)
    assert alloc.held_bytes() == held0


def test_torch_allocator_batch_handle():
    sides = gridgen.batch_sides(12)
    mats = [gridgen.diffusion_2d_5pt(int(s), sigma=1.0, seed=50 + i) for i, s in enumerate(sides)]
    perms = [gridgen.geometric_nd(M.dims) for M in mats]
    alloc = spchol.torch_allocator()
    held0 = alloc.held_bytes()
    Xs_all = []
    for allocator in (None, "torch"):
        h = spchol.batch_analyze([M.n for M in mats], [M.colptr for M in mats], [M.rowind for M in mats], perms,
                                 spchol.default_options(deterministic=2, allocator=allocator))
        assert spchol.batch_factorize(h, [M.values for M in mats]) == 0
        Bs = [gridgen.rhs_uniform(M.n, 2, seed=i) for i, M in enumerate(mats)]
        Xs = [B.copy(order="F") for B in Bs]
        spchol.batch_solve(h, Xs, [M.n for M in mats], [2] * len(mats))
        if allocator == "torch":
            assert alloc.held_bytes() > held0
        spchol.destroy(h)
        Xs_all.append(Xs)
        for M, X, B in zip(mats, Xs, Bs):
            assert oracle.berr(M, X, B) <= BERR_FP64
    for a_, b_ in zip(*Xs_all):
        assert np.array_equal(a_, b_)
    assert alloc.held_bytes() == held0
