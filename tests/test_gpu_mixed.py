"""Mixed precision: FP32 panels and updates, FP64 diagonal factorization, FP64
residual and iterative refinement.  The bar is a backward error <= 1e-12 after
refinement against the same right-hand sides, with the iteration count stated."""
import numpy as np
import pytest

import gridgen
import oracle
from tests.gpu_util import gpu_factor_solve

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1608_00044_gb300 import spchol  # noqa: E402

BERR_MIXED = 1e-12


@pytest.mark.parametrize("name", ["lap2d_64", "lap3d_16", "diff3d_12", "diff2d_40"])
@pytest.mark.parametrize("dev", [True, False])
def test_fp32_refined_reaches_target(name, dev):
    A, perm, b = gridgen.workload(name)
    B = gridgen.rhs_uniform(A.n, 3, seed=5)
    rc, X, st, h = gpu_factor_solve(A, perm, B, use_device=dev, precision=spchol.FP32)
    assert rc == 0
    st = spchol.stats(h)
    be = oracle.berr(A, X, B)
    assert be <= BERR_MIXED, (be, st["ir_iters"])
    # the library's own FP64 estimate agrees with the oracle's
    assert st["berr"] <= BERR_MIXED and st["ir_iters"] >= 1
    assert abs(st["berr"] - be) <= 0.5 * max(be, 1e-16) + 1e-16
    spchol.destroy(h)


def test_fp32_ill_conditioned_diffusion():
    """27-point diffusion with log-normal conductivity (contrast 1e4)."""
    A, perm, b = gridgen.workload("diff3d_16")
    rc, X, st, h = gpu_factor_solve(A, perm, b, precision=spchol.FP32, ir_max_iter=30)
    assert rc == 0
    st = spchol.stats(h)
    assert oracle.berr(A, X, b) <= BERR_MIXED, st
    spchol.destroy(h)


def test_refinement_reports_non_convergence():
    """With no refinement steps allowed, the FP32 factor alone cannot reach 1e-12:
    the solve must say so (ENOCONV) and still return its iterate."""
    A, perm, b = gridgen.workload("diff3d_12")
    o = spchol.default_options(precision=spchol.FP32, ir_max_iter=0)
    h = spchol.analyze(A.n, A.colptr, A.rowind, perm, o)
    assert spchol.factorize(h, A.values) == 0
    X = b.copy(order="F")
    with pytest.raises(spchol.SpcholError) as ei:
        spchol.solve(h, X, A.n, 1)
    assert ei.value.code == spchol.ENOCONV
    be = oracle.berr(A, X, b)
    assert 1e-12 < be < 1e-4
    assert abs(spchol.stats(h)["berr"] - be) <= 0.5 * be
    spchol.destroy(h)


def test_gmres_ir_takes_over_when_classic_refinement_stalls():
    """A TF32 factor of the Neumann Laplacian + 1e-4 I (kappa ~ 1.2e5, so
    u_f kappa >> 1): classic refinement stops contracting, and GMRES-IR -- FP64
    GMRES on the system left-preconditioned by the low-precision factor
    (Carson and Higham 2018) -- continues from its iterate to the target."""
    A = gridgen.neumann_laplacian_3d(16, 1e-4)
    perm = gridgen.geometric_nd(A.dims)
    B = gridgen.rhs_uniform(A.n, 2, seed=5)
    rc, X, st, h = gpu_factor_solve(A, perm, B, precision=spchol.TF32)
    assert rc == 0
    assert st["ir_gmres_iters"] > 0, st
    assert oracle.berr(A, X, B) <= BERR_MIXED
    assert st["berr"] <= BERR_MIXED
    spchol.destroy(h)


@pytest.mark.parametrize("name", ["diff3d_12", "lap3d_16"])
def test_gmres_ir_after_one_classic_step(name):
    """With one classic step allowed, a TF32 factor (which needs more) hands
    over to GMRES-IR, one right-hand side at a time; the result reaches the
    target and agrees with the oracle's FP64 solution."""
    A, perm, _ = gridgen.workload(name)
    B = gridgen.rhs_uniform(A.n, 3, seed=6)
    rc, X, st, h = gpu_factor_solve(A, perm, B, precision=spchol.TF32, ir_max_iter=1)
    assert rc == 0
    assert st["ir_gmres_iters"] > 0, st
    assert oracle.berr(A, X, B) <= BERR_MIXED
    f = oracle.OracleFactor.from_csc(A, perm)
    assert f.factor() == 0
    np.testing.assert_allclose(X, f.solve(B), rtol=1e-9, atol=1e-11)
    spchol.destroy(h)


def test_gmres_ir_is_bitwise_reproducible_in_deterministic_mode():
    """GMRES-IR's reductions run in one fixed order, so with the deterministic
    factor and solve the refined solution is bitwise equal run to run."""
    A, perm, _ = gridgen.workload("lap3d_16")
    B = gridgen.rhs_uniform(A.n, 1, seed=7)
    xs = []
    for _ in range(2):
        rc, X, st, h = gpu_factor_solve(A, perm, B, precision=spchol.TF32, deterministic=1, ir_max_iter=1)
        assert rc == 0 and st["ir_gmres_iters"] > 0
        xs.append(X)
        spchol.destroy(h)
    assert np.array_equal(xs[0], xs[1])


def test_mixed_batch():
    sides = [12, 20, 7, 33]
    mats = [gridgen.diffusion_2d_5pt(s, sigma=1.0, seed=s) for s in sides]
    perms = [gridgen.geometric_nd(M.dims) for M in mats]
    Bs = [gridgen.rhs_uniform(M.n, 2, seed=i) for i, M in enumerate(mats)]
    o = spchol.default_options(precision=spchol.FP32)
    h = spchol.batch_analyze([M.n for M in mats], [M.colptr for M in mats], [M.rowind for M in mats], perms, o)
    assert spchol.batch_factorize(h, [M.values for M in mats]) == 0
    Xs = [B.copy(order="F") for B in Bs]
    spchol.batch_solve(h, Xs, [M.n for M in mats], [2] * len(mats))
    for M, B, X in zip(mats, Bs, Xs):
        assert oracle.berr(M, X, B) <= BERR_MIXED
    spchol.destroy(h)


def _l_rel_diff(h, A):
    import scipy.sparse as sp

    Lp, Li, Lx, perm = spchol.export_factor(h)
    f = oracle.OracleFactor.from_csc(A, perm)
    assert f.factor() == 0
    op, oi, ox = f.L()
    Lg = sp.csc_matrix((Lx, Li, Lp), shape=(A.n, A.n))
    Lo = sp.csc_matrix((ox, oi, op), shape=(A.n, A.n))
    return abs(Lg - Lo).max() / abs(Lo).max()


@pytest.mark.parametrize("prec,l_tol", [(spchol.FP32, 1e-5), (spchol.TF32X3, 1e-5), (spchol.TF32, 3e-2)])
@pytest.mark.parametrize("name", ["lap3d_12", "diff3d_10", "lap2d_40"])
def test_tensor_core_factor_accuracy(prec, l_tol, name):
    """The factor itself against the oracle's FP64 L: FP32 and split-TF32 updates
    keep FP32-level accuracy (unit roundoff 6e-8, times a modest growth), plain
    TF32 (unit roundoff 4.9e-4) a few 1e-3.  Refinement then reaches 1e-12."""
    A, perm, b = gridgen.workload(name)
    B = gridgen.rhs_uniform(A.n, 2, seed=9)
    rc, X, st, h = gpu_factor_solve(A, perm, B, precision=prec, ir_max_iter=40)
    assert rc == 0
    d = _l_rel_diff(h, A)
    assert d <= l_tol, d
    assert oracle.berr(A, X, B) <= BERR_MIXED
    spchol.destroy(h)


@pytest.mark.parametrize("W", [7, 16, 33, 64])
def test_tensor_core_ragged_widths(W):
    """Panel widths that are not multiples of the MMA K step (8) and segments that
    are not multiples of 16 columns exercise the zero padding of the operand tiles."""
    A, perm, b = gridgen.workload("diff3d_11")
    rc, X, st, h = gpu_factor_solve(A, perm, b, precision=spchol.TF32X3, max_width=W)
    assert rc == 0
    assert _l_rel_diff(h, A) <= 1e-5
    assert oracle.berr(A, X, b) <= BERR_MIXED
    spchol.destroy(h)
