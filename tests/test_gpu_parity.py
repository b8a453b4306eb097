"""GPU parity: the CUDA path through the C-ABI against the CPU oracle.

Tolerances (FP64): backward error <= 1e-13 (the stated bar of the method's FP64
path), and max |L_gpu - L_oracle| <= 1e-11 max |L|: the Cholesky factor is
unique, the two computations differ only in the order of the updates
(Section II-C), and for these well-conditioned inputs the forward error of L is
a few hundred units of roundoff at most.
"""
import numpy as np
import pytest

import gridgen
import oracle
from tests import fig1
from tests.gpu_util import BERR_FP64, gpu_factor_solve, l_max_diff

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1608_00044_gb300 import spchol  # noqa: E402


def _check(A, perm, B, l_tol=1e-11, **opts):
    rc, X, st, h = gpu_factor_solve(A, perm, B, **opts)
    assert rc == 0, spchol.strerror(rc)
    be = oracle.berr(A, X, B)
    assert be <= BERR_FP64, be
    d, lmax = l_max_diff(h, A)
    assert d <= l_tol * lmax, (d, lmax)
    spchol.destroy(h)
    return X, st


def _csc(M):
    import scipy.sparse as sp

    L = sp.csc_matrix(np.tril(M))
    L.sort_indices()
    return gridgen.CscLower(M.shape[0], L.indptr.astype(np.int64), L.indices.astype(np.int32),
                            L.data.astype(np.float64))


@pytest.mark.parametrize("W,relax", [(64, 0), (2, 0), (1, 0), (128, 4)])
def test_fig1(W, relax):
    n, a_pat, fill, blocks, edges = fig1.load()
    colptr, rowind, vals = fig1.spd_from_pattern(n, a_pat)
    A = gridgen.CscLower(n, colptr, rowind, vals)
    B = gridgen.rhs_uniform(n, 2, seed=3)
    _check(A, None, B, max_width=W, relax_zeros=relax)


@pytest.mark.parametrize("n", [1, 2, 7, 31, 33, 64, 65, 150, 257])
def test_dense(n):
    rng = np.random.default_rng(n)
    G = rng.standard_normal((n, n))
    M = G @ G.T + n * np.eye(n)
    A = _csc(M)
    B = gridgen.rhs_uniform(n, 3, seed=n)
    _check(A, rng.permutation(n), B)


@pytest.mark.parametrize("W", [1, 64])
def test_pivot_square_root_accuracy(W):
    """The diagonal factorization's pivots (reciprocals by Newton's iteration in
    the normal range, a division outside it; square roots after the loop)
    against the correctly rounded square root: a diagonal matrix whose entries
    span 1e-60 .. 1e60 gives l_jj within 2 units in the last place and exact
    reciprocals within 4 (the solve uses them)."""
    n = 512
    rng = np.random.default_rng(7)
    d = 10.0 ** rng.uniform(-60, 60, n)
    M = np.diag(d)
    A = _csc(M)
    rc, X, st, h = gpu_factor_solve(A, np.arange(n), np.ones((n, 1)), max_width=W)
    assert rc == 0
    Lp, Li, Lx, perm = spchol.export_factor(h)
    ljj = Lx[Lp[:-1]]  # the diagonal heads each column
    dp = d[perm]
    np.testing.assert_allclose(ljj, np.sqrt(dp), rtol=2 * np.finfo(float).eps, atol=0)
    np.testing.assert_allclose(X[:, 0], 1.0 / d, rtol=4 * np.finfo(float).eps, atol=0)
    spchol.destroy(h)


@pytest.mark.parametrize("seed", range(6))
def test_random_sparse(seed):
    rng = np.random.default_rng(500 + seed)
    n = int(rng.integers(20, 300))
    dens = rng.uniform(0.005, 0.08)
    M = np.tril(rng.random((n, n)) < dens, -1)
    M = M | M.T
    V = np.where(M, -rng.uniform(0.1, 1.0, (n, n)), 0.0)
    V = np.tril(V) + np.tril(V, -1).T
    V[np.diag_indices(n)] = np.abs(V).sum(1) + 1.0
    A = _csc(V)
    B = gridgen.rhs_uniform(n, int(rng.integers(1, 17)), seed=seed)
    W = int(rng.choice([1, 7, 31, 33, 64, 128]))
    _check(A, rng.permutation(n), B, max_width=W, relax_zeros=int(rng.integers(0, 6)))


def test_1d_chain():
    n = 5000
    colptr = np.zeros(n + 1, np.int64)
    rows, vals = [], []
    for j in range(n):
        rows.append(j)
        vals.append(2.0)
        if j + 1 < n:
            rows.append(j + 1)
            vals.append(-1.0)
        colptr[j + 1] = len(rows)
    A = gridgen.CscLower(n, colptr, np.array(rows, np.int32), np.array(vals))
    k = np.arange(1, n + 1, dtype=np.float64)
    rc, X, st, h = gpu_factor_solve(A, None, np.eye(n, 1))
    assert rc == 0
    # closed form of A^{-1} e_1
    np.testing.assert_allclose(X[:, 0], (n + 1 - k) / (n + 1), rtol=1e-10, atol=1e-13)
    spchol.destroy(h)


@pytest.mark.parametrize("name,W", [("lap2d_64", 64), ("lap2d_64", 8), ("lap2d_64", 128), ("lap3d_16", 64),
                                    ("lap3d_16", 32), ("diff3d_12", 64), ("diff3d_11", 31), ("diff2d_37", 64)])
def test_grids(name, W):
    A, perm, b = gridgen.workload(name)
    B = gridgen.rhs_uniform(A.n, 3, seed=1)
    _check(A, perm, B, max_width=W)


@pytest.mark.parametrize("nrhs", [1, 8, 16, 17])
def test_nrhs_and_host_pointers(nrhs):
    A, perm, _ = gridgen.workload("lap3d_12")
    B = gridgen.rhs_uniform(A.n, nrhs, seed=nrhs)
    for dev in (True, False):
        rc, X, st, h = gpu_factor_solve(A, perm, B, use_device=dev)
        assert rc == 0
        assert oracle.berr(A, X, B) <= BERR_FP64
        spchol.destroy(h)


def _scaled_lap3d_12(seed):
    """lap3d_12 scaled symmetrically by D = diag(10^[-4, 4]): the rows of L = D L0
    span eight orders of magnitude."""
    A0, perm, _ = gridgen.workload("lap3d_12")
    d = 10.0 ** np.random.default_rng(seed).uniform(-4, 4, A0.n)
    cols = np.repeat(np.arange(A0.n), np.diff(A0.colptr))
    return gridgen.CscLower(A0.n, A0.colptr, A0.rowind, A0.values * d[A0.rowind] * d[cols]), perm, d


def test_fp64_solve_keeps_forward_accuracy_under_scaling():
    """The FP64 path's solves (Section II-A) round each product on its own: on a
    diagonally scaled system every component of D x agrees with the oracle's to
    the conditioning of the unscaled matrix."""
    A, perm, d = _scaled_lap3d_12(11)
    B = gridgen.rhs_uniform(A.n, 3, seed=3)
    rc, X, st, h = gpu_factor_solve(A, perm, B)
    assert rc == 0
    assert oracle.berr(A, X, B) <= BERR_FP64
    spchol.destroy(h)
    f = oracle.OracleFactor.from_csc(A, perm)
    assert f.factor() == 0
    Xo = f.solve(B)
    err = np.abs((X - Xo) * d[:, None]).max()
    assert err <= 1e-11 * np.abs(Xo * d[:, None]).max(), err


@pytest.mark.parametrize("nrhs", [1, 3, 11])
def test_fp64_tc_solve_tiles_on_tensor_cores(nrhs):
    """FP64_TC mode also runs the solves' panel tiles as split products on the
    tensor cores: FP64 backward error, also with rows spanning eight orders of
    magnitude, and with one, three and eleven right-hand sides (a partial and
    a second group of eight)."""
    for A, perm in (gridgen.workload("lap3d_12")[:2], _scaled_lap3d_12(12)[:2]):
        B = gridgen.rhs_uniform(A.n, nrhs, seed=nrhs)
        rc, X, st, h = gpu_factor_solve(A, perm, B, precision=spchol.FP64_TC)
        assert rc == 0
        assert st["max_width"] >= 16
        assert oracle.berr(A, X, B) <= BERR_FP64
        spchol.destroy(h)


@pytest.mark.parametrize("case", ["scrambled_lap3d_12", "scrambled_diff3d_9", "random"])
def test_general_ordering_through_the_library(case):
    """spchol_order_nd (Section V's fill-reducing permutation, for inputs without
    one) feeds spchol_analyze: FP64 backward error against the same b."""
    import scipy.sparse as sp

    rng = np.random.default_rng(21)
    if case == "random":
        R = sp.random(1500, 1500, density=0.004, random_state=rng, format="csc")
        S = R + R.T
        S.data[:] = -np.abs(S.data)
        M = (S + sp.diags(np.asarray(np.abs(S).sum(axis=1)).ravel() + 1.0)).tocsc()
    else:
        A0 = gridgen.workload(case.split("_", 1)[1])[0]
        L = sp.csc_matrix((A0.values, A0.rowind, A0.colptr), shape=(A0.n, A0.n))
        q = rng.permutation(A0.n)
        M = (L + sp.tril(L, -1).T).tocsc()[q][:, q]
    L = sp.csc_matrix(sp.tril(M))
    L.sort_indices()
    A = gridgen.CscLower(M.shape[0], L.indptr.astype(np.int64), L.indices.astype(np.int32), L.data.astype(np.float64))
    perm = spchol.order_nd(A.n, A.colptr, A.rowind)
    B = gridgen.rhs_uniform(A.n, 3, seed=4)
    rc, X, st, h = gpu_factor_solve(A, perm, B)
    assert rc == 0
    assert oracle.berr(A, X, B) <= BERR_FP64
    spchol.destroy(h)


@pytest.mark.parametrize("precision", ["FP64", "FP32"])
def test_deterministic_mode_is_bitwise_reproducible(precision):
    """options.deterministic (the static (target, source) order, Section IV-B):
    the factor and the solution are bitwise equal across runs and across
    launch geometries (1 and all CTAs per SM), and the backward error is the
    mode's."""
    A, perm, _ = gridgen.workload("diff3d_12")
    B = gridgen.rhs_uniform(A.n, 3, seed=8)
    prec = getattr(spchol, precision)
    runs = []
    for cps in (0, 1, 0):
        rc, X, st, h = gpu_factor_solve(A, perm, B, deterministic=1, ctas_per_sm=cps, precision=prec)
        assert rc == 0
        assert oracle.berr(A, X, B) <= (BERR_FP64 if precision == "FP64" else 1e-12)
        Lx = spchol.export_factor(h)[2] if precision == "FP64" else None
        runs.append((X, Lx))
        spchol.destroy(h)
    for X, Lx in runs[1:]:
        assert np.array_equal(X, runs[0][0])
        if Lx is not None:
            assert np.array_equal(Lx, runs[0][1])


@pytest.mark.parametrize("precision", ["FP64", "FP32", "TF32", "FP64_TC"])
def test_fanin_mode_is_bitwise_reproducible(precision):
    """options.deterministic = 2 (fan-in aggregation, the fan-in family of
    Section II-C): every update tile stores its product in a private buffer
    and each panel adds the buffers into its rows in one fixed order, so the
    factor and the solution are bitwise equal across runs and launch
    geometries, with the mode's backward error, and the FP64 factors agree
    with the oracle's."""
    A, perm, _ = gridgen.workload("diff3d_12")
    B = gridgen.rhs_uniform(A.n, 3, seed=8)
    prec = getattr(spchol, precision)
    fp64 = precision in ("FP64", "FP64_TC")
    runs = []
    for cps in (0, 1, 0):
        rc, X, st, h = gpu_factor_solve(A, perm, B, deterministic=2, ctas_per_sm=cps, precision=prec)
        assert rc == 0
        assert oracle.berr(A, X, B) <= (BERR_FP64 if fp64 else 1e-12)
        Lx = None
        if fp64:
            d, lmax = l_max_diff(h, A)
            assert d <= 1e-11 * lmax, (d, lmax)
            Lx = spchol.export_factor(h)[2]
        runs.append((X, Lx))
        spchol.destroy(h)
    for X, Lx in runs[1:]:
        assert np.array_equal(X, runs[0][0])
        if Lx is not None:
            assert np.array_equal(Lx, runs[0][1])


@pytest.mark.parametrize("name,W", [("lap2d_64", 64), ("lap3d_16", 64), ("diff3d_10", 128), ("diff3d_12", 7)])
def test_fanin_mode_matches_oracle(name, W):
    """Fan-in mode on panels of several widths (one row piece or several in
    the diagonal block, tall and short panel-solve tiles)."""
    A, perm, _ = gridgen.workload(name)
    B = gridgen.rhs_uniform(A.n, 2, seed=5)
    _check(A, perm, B, deterministic=2, max_width=W)


@pytest.mark.parametrize("precision", ["FP64", "FP32", "FP64_TC"])
def test_fanin_reproduces_the_static_order_bitwise(precision):
    """Fan-in aggregation adds each entry's updates in update-tile order, the
    order of the static (target, source) chains, and the fan-in solves add the
    tiles' products into each panel in tile order, the order of the solve
    chains: modes 2 and 1 give bitwise the same solution (and, in FP64, the
    same factor), with 1, 8 and 11 right-hand sides."""
    A, perm, _ = gridgen.workload("diff3d_12")
    prec = getattr(spchol, precision)
    for nrhs in (1, 8, 11):
        B = gridgen.rhs_uniform(A.n, nrhs, seed=9 + nrhs)
        out = []
        for det in (1, 2):
            rc, X, st, h = gpu_factor_solve(A, perm, B, deterministic=det, precision=prec)
            assert rc == 0
            out.append((X, spchol.export_factor(h)[2] if precision == "FP64" else None))
            spchol.destroy(h)
        assert np.array_equal(out[0][0], out[1][0])
        if precision == "FP64":
            assert np.array_equal(out[0][1], out[1][1])


def test_fanin_batch_matches_solo_bitwise():
    """Fan-in mode: each matrix of a batch gets bitwise the solution it gets
    alone."""
    mats = [gridgen.diffusion_2d_5pt(sd, sigma=1.0, seed=80 + i) for i, sd in enumerate((19, 28, 23))]
    perms = [gridgen.geometric_nd(M.dims) for M in mats]
    Bs = [gridgen.rhs_uniform(M.n, 2, seed=90 + i) for i, M in enumerate(mats)]
    o = spchol.default_options(deterministic=2)
    hb = spchol.batch_analyze([M.n for M in mats], [M.colptr for M in mats], [M.rowind for M in mats], perms, o)
    assert spchol.batch_factorize(hb, [M.values for M in mats]) == 0
    Xb = [Bi.copy(order="F") for Bi in Bs]
    spchol.batch_solve(hb, Xb, [M.n for M in mats], [Bi.shape[1] for Bi in Bs])
    spchol.destroy(hb)
    for M, p, Bi, Xi in zip(mats, perms, Bs, Xb):
        rc, X, st, h = gpu_factor_solve(M, p, Bi, deterministic=2)
        assert rc == 0
        assert np.array_equal(X, Xi)
        spchol.destroy(h)


def test_fanin_reports_non_spd_column():
    """Fan-in mode: a matrix that is not positive definite reports the first
    failing column like the other modes (the gathers of the later panels skip
    with their tasks)."""
    A, perm, _ = gridgen.workload("lap3d_12")
    vals = A.values.copy()
    diag = A.rowind[A.colptr[:-1]] == np.arange(A.n)
    assert diag.all()
    k = perm[A.n // 2]
    vals[A.colptr[k]] = -1.0
    B = gridgen.CscLower(A.n, A.colptr, A.rowind, vals)
    rc_dyn, _, _, h = gpu_factor_solve(B, perm, None)
    spchol.destroy(h)
    rc_fan, _, _, h = gpu_factor_solve(B, perm, None, deterministic=2)
    spchol.destroy(h)
    assert rc_dyn > 0 and rc_fan == rc_dyn


def test_deterministic_batch_matches_solo_bitwise():
    """In deterministic mode each matrix of a batch gets bitwise the solution
    it gets alone."""
    mats = [gridgen.diffusion_2d_5pt(sd, sigma=1.0, seed=60 + i) for i, sd in enumerate((17, 30, 24))]
    perms = [gridgen.geometric_nd(M.dims) for M in mats]
    Bs = [gridgen.rhs_uniform(M.n, 2, seed=70 + i) for i, M in enumerate(mats)]
    o = spchol.default_options(deterministic=1)
    hb = spchol.batch_analyze([M.n for M in mats], [M.colptr for M in mats], [M.rowind for M in mats], perms, o)
    assert spchol.batch_factorize(hb, [M.values for M in mats]) == 0
    Xb = [Bi.copy(order="F") for Bi in Bs]
    spchol.batch_solve(hb, Xb, [M.n for M in mats], [Bi.shape[1] for Bi in Bs])
    spchol.destroy(hb)
    for M, p, Bi, Xi in zip(mats, perms, Bs, Xb):
        rc, X, st, h = gpu_factor_solve(M, p, Bi, deterministic=1)
        assert rc == 0
        assert np.array_equal(X, Xi)
        spchol.destroy(h)


def test_repeat_solve_and_refactorize():
    A, perm, _ = gridgen.workload("diff3d_10")
    o = spchol.default_options()
    h = spchol.analyze(A.n, A.colptr, A.rowind, perm, o)
    assert spchol.factorize(h, A.values) == 0
    for it in range(3):
        B = gridgen.rhs_uniform(A.n, 2, seed=10 + it)
        X = B.copy(order="F")
        spchol.solve(h, X, A.n, 2)
        assert oracle.berr(A, X, B) <= BERR_FP64
    # new values, same pattern: 2A
    A2 = gridgen.CscLower(A.n, A.colptr, A.rowind, A.values * 2.0)
    assert spchol.factorize(h, A2.values) == 0
    B = gridgen.rhs_uniform(A.n, 1, seed=99)
    X = B.copy(order="F")
    spchol.solve(h, X, A.n, 1)
    assert oracle.berr(A2, X, B) <= BERR_FP64
    spchol.destroy(h)


def test_side_stream():
    A, perm, b = gridgen.workload("lap2d_64")
    s = torch.cuda.Stream()
    o = spchol.default_options()
    h = spchol.analyze(A.n, A.colptr, A.rowind, perm, o)
    with torch.cuda.stream(s):
        vals = torch.from_numpy(A.values).cuda()
        Bt = torch.from_numpy(np.ascontiguousarray(b.T)).cuda()
        assert spchol.factorize(h, vals, stream=s) == 0
        spchol.solve(h, Bt, A.n, 1, stream=s)
    s.synchronize()
    assert oracle.berr(A, Bt.cpu().numpy().T, b) <= BERR_FP64
    spchol.destroy(h)


@pytest.mark.parametrize("which", ["first", "middle", "last"])
def test_not_spd_reports_smallest_column(which):
    A, perm, b = gridgen.workload("lap2d_64")
    o = spchol.default_options()
    h = spchol.analyze(A.n, A.colptr, A.rowind, perm, o)
    fp = spchol.final_perm(h)
    pinv = np.empty_like(fp)
    pinv[fp] = np.arange(A.n)
    bad = {"first": int(fp[0]), "middle": 1234, "last": int(fp[-1])}[which]
    vals = A.values.copy()
    vals[A.colptr[bad]] = -5.0
    rc = spchol.factorize(h, vals)
    assert rc == pinv[bad] + 1
    # the oracle agrees on the failing column
    f = oracle.OracleFactor(A.n, A.colptr, A.rowind, vals, fp)
    assert f.factor() == rc
    # the handle is usable again with good values
    assert spchol.factorize(h, A.values) == 0
    X = b.copy(order="F")
    spchol.solve(h, X, A.n, 1)
    assert oracle.berr(A, X, b) <= BERR_FP64
    spchol.destroy(h)


def test_wait_budget_times_out_cleanly():
    """A phantom dependency keeps the last panel from ever becoming ready: every
    CTA's bounded wait must give up and factorize must report ETIMEOUT."""
    A, perm, b = gridgen.workload("lap2d_32")
    o = spchol.default_options(fault_inject=1, wait_budget_ns=50_000_000)
    h = spchol.analyze(A.n, A.colptr, A.rowind, perm, o)
    with pytest.raises(spchol.SpcholError) as ei:
        spchol.factorize(h, A.values)
    assert ei.value.code == spchol.ETIMEOUT
    spchol.destroy(h)
    # the context is still healthy
    rc, X, st, h2 = gpu_factor_solve(A, perm, b)
    assert rc == 0 and oracle.berr(A, X, b) <= BERR_FP64
    spchol.destroy(h2)


def test_solve_before_factorize():
    A, perm, b = gridgen.workload("lap2d_16")
    h = spchol.analyze(A.n, A.colptr, A.rowind, perm, spchol.default_options())
    with pytest.raises(spchol.SpcholError) as ei:
        spchol.solve(h, b.copy(order="F"), A.n, 1)
    assert ei.value.code == spchol.ESTATE
    spchol.destroy(h)


def test_empty_matrix():
    A = gridgen.CscLower(0, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0))
    h = spchol.analyze(0, A.colptr, A.rowind, None, spchol.default_options())
    assert spchol.factorize(h, A.values) == 0
    spchol.destroy(h)


def test_batch_matches_solo():
    sides = [5, 16, 23, 9, 31]
    mats = [gridgen.diffusion_2d_5pt(s, sigma=1.0, seed=s) for s in sides]
    perms = [gridgen.geometric_nd(M.dims) for M in mats]
    Bs = [gridgen.rhs_uniform(M.n, 1 + (i % 3), seed=i) for i, M in enumerate(mats)]
    o = spchol.default_options()
    h = spchol.batch_analyze([M.n for M in mats], [M.colptr for M in mats], [M.rowind for M in mats], perms, o)
    assert spchol.batch_factorize(h, [M.values for M in mats]) == 0
    Xs = [B.copy(order="F") for B in Bs]
    spchol.batch_solve(h, Xs, [M.n for M in mats], [B.shape[1] for B in Bs])
    for M, P, B, X in zip(mats, perms, Bs, Xs):
        assert oracle.berr(M, X, B) <= BERR_FP64
        rc, Xs1, st, h1 = gpu_factor_solve(M, P, B)
        np.testing.assert_allclose(X, Xs1, rtol=1e-11, atol=1e-13)
        spchol.destroy(h1)
    # a non-SPD matrix inside the batch is located
    bad_vals = [M.values.copy() for M in mats]
    bad_vals[3][mats[3].colptr[4]] = -1.0
    k = spchol.batch_factorize(h, bad_vals)
    assert k > 0
    m, col = spchol.batch_info(h, k)
    assert m == 3 and 1 <= col <= mats[3].n
    spchol.destroy(h)


@pytest.mark.slow
def test_full_size_lap3d_64_sampled():
    """64^3 7-point Laplacian at full size in the benchmark's configuration:
    backward error of all 8 solutions, and sampled entries of L L^T - P A P^T."""
    A, perm, b = gridgen.workload("lap3d_64")
    rc, X, st, h = gpu_factor_solve(A, perm, b)
    assert rc == 0
    assert oracle.berr(A, X, b) <= BERR_FP64
    Lp, Li, Lx, fperm = spchol.export_factor(h)
    import scipy.sparse as sp

    n = A.n
    L = sp.csc_matrix((Lx, Li, Lp), shape=(n, n)).tocsr()
    full = A.to_scipy_full()
    Bp = full[fperm][:, fperm].tocsr()
    rng = np.random.default_rng(0)
    cols = np.concatenate([rng.integers(0, n, 40), np.arange(n - 64, n)])  # includes the top separator
    worst = 0.0
    for j in cols:
        rows = np.concatenate([Bp[:, [j]].nonzero()[0], rng.integers(j, n, 4)])
        for i in rows[rows >= j]:
            v = L[i].multiply(L[j]).sum()
            worst = max(worst, abs(v - Bp[i, j]))
    assert worst <= 1e-12 * abs(A.values).max()
    spchol.destroy(h)


def test_handles_with_different_panel_widths_coexist():
    """A handle with wide panels (large shared-memory tiles) stays usable after
    another handle with narrow panels has been analyzed: the kernels' shared
    memory limits are not owned by one handle."""
    rng = np.random.default_rng(3)
    G = rng.standard_normal((120, 120))
    wide = _csc(G @ G.T + 120 * np.eye(120))
    narrow, nperm, nb = gridgen.workload("lap2d_16")
    hw = spchol.analyze(wide.n, wide.colptr, wide.rowind, None, spchol.default_options(max_width=128))
    hn = spchol.analyze(narrow.n, narrow.colptr, narrow.rowind, nperm, spchol.default_options(max_width=4))
    assert spchol.factorize(hw, wide.values) == 0
    assert spchol.factorize(hn, narrow.values) == 0
    B = gridgen.rhs_uniform(wide.n, 2, seed=1)
    X = B.copy(order="F")
    spchol.solve(hw, X, wide.n, 2)
    assert oracle.berr(wide, X, B) <= BERR_FP64
    spchol.destroy(hw)
    spchol.destroy(hn)


# ---------------------------------------------------------------- FP64 result, BF16 tensor-core updates


@pytest.mark.parametrize("name,W", [("lap2d_64", 64), ("lap3d_16", 64), ("diff3d_12", 64), ("diff3d_11", 33),
                                    ("lap3d_12", 16), ("diff2d_37", 7)])
def test_fp64_tc_matches_oracle(name, W):
    """The split-operand tensor-core updates keep the FP64 bar: backward error
    <= 1e-13 with no refinement and L within 1e-11 of the oracle's."""
    A, perm, b = gridgen.workload(name)
    B = gridgen.rhs_uniform(A.n, 3, seed=2)
    _check(A, perm, B, precision=spchol.FP64_TC, max_width=W)


@pytest.mark.parametrize("n", [1, 9, 64, 130])
def test_fp64_tc_dense(n):
    rng = np.random.default_rng(40 + n)
    G = rng.standard_normal((n, n))
    A = _csc(G @ G.T + n * np.eye(n))
    _check(A, rng.permutation(n), gridgen.rhs_uniform(n, 2, seed=n), precision=spchol.FP64_TC)


def test_fp64_tc_wide_dynamic_range():
    """Rows whose entries span many orders of magnitude: the row-relative split
    must still deliver FP64 backward error (diagonal scaling by 10^[-4, 4])."""
    A0, perm, b = gridgen.workload("lap3d_10")
    rng = np.random.default_rng(5)
    d = 10.0 ** rng.uniform(-4, 4, A0.n)
    cols = np.repeat(np.arange(A0.n), np.diff(A0.colptr))
    vals = A0.values * d[A0.rowind] * d[cols]
    A = gridgen.CscLower(A0.n, A0.colptr, A0.rowind, vals)
    rc, X, st, h = gpu_factor_solve(A, perm, b, precision=spchol.FP64_TC)
    assert rc == 0
    assert oracle.berr(A, X, b) <= BERR_FP64
    spchol.destroy(h)


# ---------------------------------------------------------------- CUDA graphs, autotuning


def _capture_factorization(h, vals):
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):  # one eager run first: nothing is allocated during capture
        spchol.factorize_enqueue(h, vals, stream=s)
    s.synchronize()
    assert spchol.factorize_status(h) == 0
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        spchol.factorize_enqueue(h, vals, stream=s)
    return g


def test_factorization_captured_in_a_cuda_graph():
    A, perm, b = gridgen.workload("lap3d_12")
    h = spchol.analyze(A.n, A.colptr, A.rowind, perm, spchol.default_options())
    vals = torch.from_numpy(A.values).cuda()
    g = _capture_factorization(h, vals)
    for scale in (1.0, 2.5, 0.5):
        vals.copy_(torch.from_numpy(A.values * scale))
        g.replay()
        torch.cuda.synchronize()
        assert spchol.factorize_status(h) == 0
        X = b.copy(order="F")
        spchol.solve(h, X, A.n, b.shape[1])
        As = gridgen.CscLower(A.n, A.colptr, A.rowind, A.values * scale)
        assert oracle.berr(As, X, b) <= BERR_FP64
    spchol.destroy(h)


def test_fanin_factorization_captured_in_a_cuda_graph():
    """Fan-in mode through a captured graph: its counters are reset inside the
    graph, so every replay gives bitwise the eager factor."""
    A, perm, b = gridgen.workload("diff3d_10")
    h = spchol.analyze(A.n, A.colptr, A.rowind, perm, spchol.default_options(deterministic=2))
    vals = torch.from_numpy(A.values).cuda()
    assert spchol.factorize(h, vals) == 0
    L0 = spchol.export_factor(h)[2]
    g = _capture_factorization(h, vals)
    for _ in range(3):
        g.replay()
        torch.cuda.synchronize()
        assert spchol.factorize_status(h) == 0
        assert np.array_equal(spchol.export_factor(h)[2], L0)
    X = b.copy(order="F")
    spchol.solve(h, X, A.n, b.shape[1])
    assert oracle.berr(A, X, b) <= BERR_FP64
    spchol.destroy(h)


def test_batch_factorization_captured_in_a_cuda_graph():
    sides = [9, 20, 13, 31]
    mats = [gridgen.diffusion_2d_5pt(s, sigma=1.0, seed=s) for s in sides]
    perms = [gridgen.geometric_nd(M.dims) for M in mats]
    h = spchol.batch_analyze([M.n for M in mats], [M.colptr for M in mats], [M.rowind for M in mats], perms,
                             spchol.default_options())
    vals = torch.cat([torch.from_numpy(M.values) for M in mats]).cuda()
    g = _capture_factorization(h, vals)
    g.replay()
    torch.cuda.synchronize()
    assert spchol.factorize_status(h) == 0
    Bs = [gridgen.rhs_uniform(M.n, 2, seed=i) for i, M in enumerate(mats)]
    Xs = [B.copy(order="F") for B in Bs]
    spchol.batch_solve(h, Xs, [M.n for M in mats], [2] * len(mats))
    for M, B, X in zip(mats, Bs, Xs):
        assert oracle.berr(M, X, B) <= BERR_FP64
    spchol.destroy(h)


def test_autotuner_picks_a_working_configuration(tmp_path):
    from paper_1608_00044_gb300 import autotune

    sides = [17, 25, 40]
    mats = [gridgen.diffusion_2d_5pt(s, sigma=1.0, seed=s) for s in sides]
    perms = [gridgen.geometric_nd(M.dims) for M in mats]
    cache = str(tmp_path / "tune.json")
    res = autotune.tune(mats, perms, candidates=[(64, 4, 64), (32, 16, 32)], reps=2, cache_path=cache)
    assert len(res["tried_ms"]) == 2 and not res["cached"]
    again = autotune.tune(mats, perms, candidates=[(64, 4, 64), (32, 16, 32)], reps=2, cache_path=cache)
    assert again["cached"] and again["max_width"] == res["max_width"]
    o = spchol.default_options(max_width=res["max_width"], relax_zeros=res["relax_zeros"], tile_rows=res["tile_rows"])
    h = spchol.batch_analyze([M.n for M in mats], [M.colptr for M in mats], [M.rowind for M in mats], perms, o)
    assert spchol.batch_factorize(h, [M.values for M in mats]) == 0
    spchol.destroy(h)


@pytest.mark.parametrize("name,W,precision,det", [
    ("lap3d_32", 16, "FP64", 0), ("lap3d_24", 8, "FP64", 0), ("lap2d_256", 4, "FP64", 0),
    ("lap3d_40", 32, "FP64", 0), ("lap3d_32", 16, "FP64_TC", 0), ("lap3d_24", 8, "FP64", 2),
])
def test_deep_panel_trees_elementwise(name, W, precision, det):
    # Panel trees deeper than the 128 levels near the root whose panels get the
    # short tiles: the 64-row update and panel-solve tiles and the 256-row solve
    # tiles of the deeper panels are compared with the oracle entry by entry
    # (L within 1e-11 of max |L|) and through the solution (within 1e-10 of
    # the oracle's, berr <= 1e-13).
    A, perm, B = gridgen.workload(name)
    X, st = _check(A, perm, B, max_width=W, precision=getattr(spchol, precision), deterministic=det)
    f = oracle.OracleFactor.from_csc(A, perm)
    assert f.factor() == 0
    Xo = f.solve(B)
    assert np.abs(X - Xo).max() <= 1e-10 * np.abs(Xo).max()


@pytest.mark.parametrize("rows", [8, 32, 256])
@pytest.mark.parametrize("nrhs", [1, 8, 11])
def test_solve_tile_rows_extremes(rows, nrhs):
    # The deep panels' solve tiles from 8 to 256 rows (chunks of 32 rows staged
    # in shared memory, k-split over warps for few right-hand sides, more than
    # one pass of eight right-hand sides): solutions within 1e-10 of the
    # oracle's, berr <= 1e-13.
    A, perm, _ = gridgen.workload("lap3d_24")
    B = gridgen.rhs_uniform(A.n, nrhs, seed=rows + nrhs)
    X, st = _check(A, perm, B, max_width=8, solve_tile_rows=rows)
    f = oracle.OracleFactor.from_csc(A, perm)
    assert f.factor() == 0
    Xo = f.solve(B)
    assert np.abs(X - Xo).max() <= 1e-10 * np.abs(Xo).max()


def test_fifo_schedule_with_static_chains_is_bitwise_reproducible():
    A, perm, B = gridgen.workload("lap3d_14")
    res = []
    for sched in (0, 1, 1):
        rc, X, st, h = gpu_factor_solve(A, perm, B, deterministic=1, sched=sched)
        assert rc == 0
        res.append((spchol.export_factor(h)[2], X))
        spchol.destroy(h)
    for Lx, X in res[1:]:  # the static order fixes every sum: the ring's order does not matter
        assert np.array_equal(Lx, res[0][0]) and np.array_equal(X, res[0][1])


@pytest.mark.parametrize("depth", [-1, 4, 64, 1000])
@pytest.mark.parametrize("nrhs", [1, 3, 8, 11])
def test_w_panels_match_the_oracle(depth, nrhs):
    # Panels within solve_w_depth levels of the root keep W = L21 L11^{-1}:
    # their forward tiles subtract W b_s as soon as b_s is complete, their
    # diagonal task forms A11^{-1} b_s off the chain, and their backward tiles
    # subtract W^T x (the last one releasing the panel's readers).  None, a few,
    # the default and every panel outside the subtree tasks: solutions within
    # 1e-10 of the oracle's, berr <= 1e-13, L unchanged (within 1e-11), and the
    # W buffer counted in the footprint.
    A, perm, _ = gridgen.workload("lap3d_24")
    B = gridgen.rhs_uniform(A.n, nrhs, seed=nrhs + depth)
    X, st = _check(A, perm, B, max_width=16, solve_w_depth=depth)
    f = oracle.OracleFactor.from_csc(A, perm)
    assert f.factor() == 0
    Xo = f.solve(B)
    assert np.abs(X - Xo).max() <= 1e-10 * np.abs(Xo).max()
    if depth != -1:
        rc, _, st0, h0 = gpu_factor_solve(A, perm, None, max_width=16, solve_w_depth=-1)
        spchol.destroy(h0)
        assert st["footprint_bytes"] > st0["footprint_bytes"]


@pytest.mark.parametrize("precision,sched", [("FP32", 0), ("FP64_TC", 0), ("TF32X3", 0), ("FP64", 1)])
def test_w_panels_other_precisions_and_fifo(precision, sched):
    # W in the panels' precision (FP32 for the mixed modes, whose refinement
    # then reaches its 1e-12 target), on the tensor-core solve tiles (FP64_TC)
    # and with the single FIFO ring.  Several handles in a row: W is formed
    # anew by every factorization, whatever the memory held before.
    A, perm, _ = gridgen.workload("lap3d_24")
    B = gridgen.rhs_uniform(A.n, 4, seed=5)
    bar = BERR_FP64 if precision.startswith("FP64") else 1e-12
    for _ in range(3):
        rc, X, st, h = gpu_factor_solve(A, perm, B, max_width=32, solve_w_depth=1000,
                                        precision=getattr(spchol, precision), sched=sched)
        assert rc == 0, spchol.strerror(rc)
        spchol.destroy(h)
        assert oracle.berr(A, X, B) <= bar


def test_w_depth_is_ignored_by_the_deterministic_modes():
    A, perm, B = gridgen.workload("lap3d_14")
    res = []
    for det, depth in ((1, -1), (1, 1000), (2, 1000)):
        rc, X, st, h = gpu_factor_solve(A, perm, B, deterministic=det, solve_w_depth=depth)
        assert rc == 0
        res.append(X)
        spchol.destroy(h)
    assert np.array_equal(res[0], res[1]) and np.array_equal(res[0], res[2])


def test_batch_with_w_panels_matches_solo():
    # A batch keeps no W panels by default; asked for them, every matrix's
    # near-root panels get W and the batch still matches the solo solves.
    sides = [9, 24, 17, 31]
    mats = [gridgen.diffusion_2d_5pt(s, sigma=1.0, seed=50 + s) for s in sides]
    perms = [gridgen.geometric_nd(M.dims) for M in mats]
    Bs = [gridgen.rhs_uniform(M.n, 2, seed=i) for i, M in enumerate(mats)]
    for depth in (-1, 1000):
        o = spchol.default_options(solve_w_depth=depth)
        h = spchol.batch_analyze([M.n for M in mats], [M.colptr for M in mats], [M.rowind for M in mats], perms, o)
        fp = spchol.stats(h)["footprint_bytes"]
        if depth == -1:
            fp_none = fp
        else:
            assert fp > fp_none
        assert spchol.batch_factorize(h, [M.values for M in mats]) == 0
        Xs = [B.copy(order="F") for B in Bs]
        spchol.batch_solve(h, Xs, [M.n for M in mats], [B.shape[1] for B in Bs])
        spchol.destroy(h)
        for M, P, B, X in zip(mats, perms, Bs, Xs):
            assert oracle.berr(M, X, B) <= BERR_FP64
            rc, X1, st, h1 = gpu_factor_solve(M, P, B)
            spchol.destroy(h1)
            np.testing.assert_allclose(X, X1, rtol=1e-11, atol=1e-13)


def _merged(mats, perms):
    """The block-diagonal matrix of a batch (lower CSC) and its permutation."""
    n = sum(M.n for M in mats)
    cp, ri, vals, pm = [0], [], [], []
    off = 0
    for M, p in zip(mats, perms):
        for j in range(M.n):
            a, b = M.colptr[j], M.colptr[j + 1]
            ri.extend((M.rowind[a:b] + off).tolist())
            vals.extend(M.values[a:b].tolist())
            cp.append(len(ri))
        pm.extend((np.asarray(p) + off).tolist())
        off += M.n
    A = gridgen.CscLower(n, np.array(cp, np.int64), np.array(ri, np.int32), np.array(vals))
    return A, np.array(pm, np.int64)


@pytest.mark.parametrize("precision,l_tol,bar", [("FP64", 1e-11, BERR_FP64), ("FP32", 1e-5, 1e-12)])
def test_warp_subtrees_match_the_oracle(precision, l_tol, bar):
    # A batch whose subtree tasks all qualify for single warps (panels <= 32
    # wide, most of the work in the subtrees): L entry by entry against the
    # oracle's factor of the block-diagonal matrix (1e-11 of max |L| in FP64,
    # 1e-5 in FP32), the solutions against the oracle's (1e-10) and the
    # backward error (1e-13; after refinement 1e-12); a single large matrix
    # keeps its subtrees on CTAs.
    sides = np.random.default_rng(7).integers(16, 64, 160)  # enough work for subtree tasks of many panels
    mats = [gridgen.diffusion_2d_5pt(int(s), sigma=1.0, seed=300 + i) for i, s in enumerate(sides)]
    perms = [gridgen.geometric_nd(M.dims) for M in mats]
    Bs = [gridgen.rhs_uniform(M.n, 2, seed=i) for i, M in enumerate(mats)]
    o = spchol.default_options(max_width=32, relax_zeros=16, tile_rows=32, precision=getattr(spchol, precision))
    h = spchol.batch_analyze([M.n for M in mats], [M.colptr for M in mats], [M.rowind for M in mats], perms, o)
    st = spchol.stats(h)
    assert st["n_subtrees"] > 0 and st["n_warp_subtrees"] == st["n_subtrees"]
    assert spchol.batch_factorize(h, [M.values for M in mats]) == 0
    A, _ = _merged(mats, perms)
    d, lmax = l_max_diff(h, A)
    assert d <= l_tol * lmax, (d, lmax)
    Xs = [B.copy(order="F") for B in Bs]
    spchol.batch_solve(h, Xs, [M.n for M in mats], [B.shape[1] for B in Bs])
    spchol.destroy(h)
    for M, P, B, X in zip(mats, perms, Bs, Xs):
        assert oracle.berr(M, X, B) <= bar
        f = oracle.OracleFactor.from_csc(M, P)
        assert f.factor() == 0
        Xo = f.solve(B)
        assert np.abs(X - Xo).max() <= 1e-10 * np.abs(Xo).max()
    A1, p1, _ = gridgen.workload("lap3d_24")
    h1 = spchol.analyze(A1.n, A1.colptr, A1.rowind, p1, spchol.default_options(max_width=32))
    assert spchol.stats(h1)["n_warp_subtrees"] == 0
    spchol.destroy(h1)


def test_warp_subtrees_report_a_failed_pivot():
    # A matrix of the batch that is not SPD in a column its subtree holds: the
    # batch reports it (the smallest failing permuted column, here that
    # matrix's), and a later factorization of the repaired values succeeds.
    sides = np.random.default_rng(8).integers(16, 64, 160)
    mats = [gridgen.diffusion_2d_5pt(int(s), sigma=1.0, seed=400 + i) for i, s in enumerate(sides)]
    perms = [gridgen.geometric_nd(M.dims) for M in mats]
    o = spchol.default_options(max_width=32, relax_zeros=16, tile_rows=32)
    h = spchol.batch_analyze([M.n for M in mats], [M.colptr for M in mats], [M.rowind for M in mats], perms, o)
    assert spchol.stats(h)["n_warp_subtrees"] > 0
    bad = [M.values.copy() for M in mats]
    j = int(perms[2][0])  # the first column eliminated in matrix 2 (a leaf of its tree)
    bad[2][mats[2].colptr[j]] = -5.0
    k = spchol.batch_factorize(h, bad)
    assert k > 0
    m, col = spchol.batch_info(h, k)
    assert m == 2
    assert spchol.batch_factorize(h, [M.values for M in mats]) == 0
    spchol.destroy(h)
