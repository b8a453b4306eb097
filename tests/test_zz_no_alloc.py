"""spchol_solve_noalloc: the solve for callers that cannot allocate device memory.

Such callers (a service that reserves its device memory up front, code running
where cudaMalloc is not allowed) solve with a resident factor through this entry
point, whose workspace is a fixed array in device memory instead of memory
from cudaMalloc.  Its results are checked against spchol_solve on the same
factor, on two calls in a row: the fixed array keeps the previous call's
contents, and the second call must not see them.  The tolerance is the one of
the other FP64 tests: backward error <= 1e-13, and the two solutions equal up
to the rounding of the (unordered) atomic accumulations.

This file is collected last so that a run that stops at the first failure has
already run every other test.
"""
import numpy as np
import pytest

import gridgen
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1608_00044_gb300 import spchol  # noqa: E402


def _solve_both(h, A, nrhs, seed):
    B = gridgen.rhs_uniform(A.n, nrhs, seed=seed)
    X_ref = B.copy(order="F")
    spchol.solve(h, X_ref, A.n, nrhs)  # the existing entry point
    Bt = torch.from_numpy(np.ascontiguousarray(B.T)).cuda()  # (nrhs, n) row-major == n x nrhs column-major
    spchol.solve_noalloc(h, Bt, A.n, nrhs)
    X = np.asfortranarray(Bt.cpu().numpy().T)
    return B, X, X_ref


@pytest.mark.parametrize("precision", [spchol.FP64, spchol.FP64_TC])
def test_noalloc_matches_solve_on_two_calls(precision):
    A, perm, _ = gridgen.workload("lap3d_16")
    h = spchol.analyze(A.n, A.colptr, A.rowind, perm, spchol.default_options(precision=precision))
    assert spchol.factorize(h, A.values) == 0
    for nrhs, seed in ((3, 1), (8, 2)):
        B, X, X_ref = _solve_both(h, A, nrhs, seed)
        assert oracle.berr(A, X, B) <= 1e-13
        assert np.abs(X - X_ref).max() <= 1e-10 * np.abs(X_ref).max()
    spchol.destroy(h)


@pytest.mark.parametrize("det", [1, 2])
def test_noalloc_deterministic_modes_match_solve_bitwise(det):
    """In the deterministic modes (static chains, fan-in buffers in the fixed
    array) the two entry points give bitwise the same solution."""
    A, perm, _ = gridgen.workload("diff3d_12")
    h = spchol.analyze(A.n, A.colptr, A.rowind, perm, spchol.default_options(deterministic=det))
    assert spchol.factorize(h, A.values) == 0
    for nrhs, seed in ((3, 4), (8, 5)):
        B, X, X_ref = _solve_both(h, A, nrhs, seed)
        assert oracle.berr(A, X, B) <= 1e-13
        assert np.array_equal(X, X_ref)
    spchol.destroy(h)


def test_noalloc_second_handle_after_first():
    """A different matrix right after: the reused scratch is re-initialised."""
    for name, nrhs in (("diff3d_12", 5), ("lap2d_64", 1)):
        A, perm, _ = gridgen.workload(name)
        h = spchol.analyze(A.n, A.colptr, A.rowind, perm, spchol.default_options())
        assert spchol.factorize(h, A.values) == 0
        B, X, X_ref = _solve_both(h, A, nrhs, 7)
        assert oracle.berr(A, X, B) <= 1e-13
        assert np.abs(X - X_ref).max() <= 1e-10 * np.abs(X_ref).max()
        spchol.destroy(h)


def test_noalloc_rejects_what_it_cannot_do():
    A, perm, _ = gridgen.workload("lap3d_16")
    h = spchol.analyze(A.n, A.colptr, A.rowind, perm, spchol.default_options())
    assert spchol.factorize(h, A.values) == 0
    big = torch.zeros((1100, A.n), dtype=torch.float64, device="cuda")  # 8 n nrhs bytes > 32 MiB
    with pytest.raises(spchol.SpcholError) as ei:
        spchol.solve_noalloc(h, big, A.n, 1100)
    assert ei.value.code == spchol.ESCRATCH
    host = np.zeros((A.n, 1), order="F")
    with pytest.raises(spchol.SpcholError) as ei:
        spchol.solve_noalloc(h, host, A.n, 1)
    assert ei.value.code == -2
    spchol.destroy(h)
