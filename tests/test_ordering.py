"""The fill-reducing ordering for general patterns (spchol_order_nd), on the CPU.

Section V applies a fill-reducing symmetric permutation before the
factorization.  The ordering is a heuristic, so it is pinned by what must hold
for any valid one -- a permutation of 0..n-1, the same factor and solution as
the oracle's on the same permutation -- and by fill measured with the exact
symbolic count: far below the identity's on a scrambled grid, at or below the
geometric nested dissection's on the 7-point grids, and within a stated factor
of it on the 27-point grid (where breadth-first levels are cube shells).
"""
import numpy as np
import pytest

import gridgen
import oracle
from paper_1608_00044_gb300 import build
from paper_1608_00044_gb300 import hostplan as hp

build.build_host()
sp = pytest.importorskip("scipy.sparse")


def _lower(M):
    """CscLower of the lower triangle (diagonal included) of a symmetric scipy matrix."""
    L = sp.csc_matrix(sp.tril(M))
    L.sort_indices()
    return gridgen.CscLower(M.shape[0], L.indptr.astype(np.int64), L.indices.astype(np.int32),
                            L.data.astype(np.float64))


def _full(A):
    L = sp.csc_matrix((A.values, A.rowind, A.colptr), shape=(A.n, A.n))
    return (L + sp.tril(L, -1).T).tocsc()


def _scrambled(A, seed):
    """Q A Q^T for a random permutation Q: the grid with its rows in random order."""
    q = np.random.default_rng(seed).permutation(A.n)
    M = _full(A)[q][:, q]
    return _lower(M)


def _random_spd(n, density, seed, blocks=1):
    """A random sparse SPD matrix (diagonally dominant), optionally block diagonal
    (disconnected components), with some isolated vertices."""
    rng = np.random.default_rng(seed)
    parts = []
    for b in range(blocks):
        m = n // blocks + (1 if b < n % blocks else 0)
        R = sp.random(m, m, density=density, random_state=rng, format="csc")
        S = R + R.T
        S.data[:] = -np.abs(S.data)
        parts.append(S)
    M = sp.block_diag(parts, format="csc")
    d = np.asarray(np.abs(M).sum(axis=1)).ravel() + 1.0
    M = (M + sp.diags(d)).tocsc()
    return _lower(M)


def _flops(A, perm):
    return hp.HostPlan(A.n, A.colptr, A.rowind, perm).flops


@pytest.mark.parametrize("n,density,blocks", [(0, 0, 1), (1, 0, 1), (2, 0.5, 1), (5, 0.3, 1), (64, 0.05, 1),
                                              (65, 0.05, 1), (300, 0.01, 1), (2000, 0.002, 1), (2000, 0.001, 7),
                                              (500, 0.0, 1)])
def test_order_is_a_permutation(n, density, blocks):
    A = _random_spd(n, density, seed=n + blocks, blocks=blocks) if n > 0 else gridgen.CscLower(
        0, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0))
    p = hp.order_nd(A.n, A.colptr, A.rowind)
    assert p.dtype == np.int64 and sorted(p.tolist()) == list(range(A.n))


def test_order_of_special_graphs():
    # complete graph (no level can separate), star, path, and a grid: all permutations
    for M in (sp.csc_matrix(np.ones((100, 100)) + 100 * np.eye(100)),
              sp.csc_matrix(sp.diags([np.ones(99), 3 * np.ones(100), np.ones(99)], [-1, 0, 1])),
              _full(gridgen.laplacian_2d(9))):
        A = _lower(M)
        p = hp.order_nd(A.n, A.colptr, A.rowind)
        assert sorted(p.tolist()) == list(range(A.n))
    star = sp.lil_matrix((200, 200))
    star[0, 1:] = 1.0
    star[1:, 0] = 1.0
    A = _lower((star + 300 * sp.eye(200)).tocsc())
    p = hp.order_nd(A.n, A.colptr, A.rowind)
    assert sorted(p.tolist()) == list(range(A.n))
    # a star is a tree: minimum-degree leaves first, centre last, no fill at all
    assert hp.HostPlan(A.n, A.colptr, A.rowind, p).scalars()["nnz_l"] == A.colptr[-1]


@pytest.mark.parametrize("name", ["lap2d_64", "lap3d_16"])
def test_fill_on_scrambled_grids(name):
    A0, perm_geo, _ = gridgen.workload(name)
    A = _scrambled(A0, seed=3)
    p = hp.order_nd(A.n, A.colptr, A.rowind)
    f_nd = _flops(A, p)
    assert f_nd <= _flops(A0, perm_geo)           # at or below the geometric dissection
    assert 5 * f_nd <= _flops(A, None)            # and far below the scrambled order


@pytest.mark.parametrize("name,factor", [("diff3d_16", 3.2), ("diff3d_24", 2.5)])
def test_fill_on_27_point_grid_within_stated_factor(name, factor):
    """On a 27-point stencil breadth-first levels are cube shells (L-infinity
    spheres) rather than planes, so the separators are larger than the
    geometric dissection's: its flops stay within the stated factor."""
    A, perm_geo, _ = gridgen.workload(name)
    p = hp.order_nd(A.n, A.colptr, A.rowind)
    assert _flops(A, p) <= factor * _flops(A, perm_geo)


def test_factor_and_solve_with_the_ordering_match_the_oracle():
    A = _scrambled(gridgen.workload("diff3d_8")[0], seed=5)
    p = hp.order_nd(A.n, A.colptr, A.rowind)
    B = gridgen.rhs_uniform(A.n, 2, seed=1)
    P = hp.HostPlan(A.n, A.colptr, A.rowind, p)
    rc, X, _ = P.simulate(A.values, B, seed=2)
    assert rc == 0
    assert oracle.berr(A, X, B) <= 1e-14
    f = oracle.OracleFactor.from_csc(A, P.get(hp.PERM))
    assert P.flops == f.flops
    assert f.factor() == 0
    np.testing.assert_allclose(X, f.solve(B), rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("bad,code", [("n", -1), ("colptr0", -2), ("nonmono", -2), ("upper", -3),
                                      ("unsorted", -3), ("range", -3), ("out", -4)])
def test_argument_checks(bad, code):
    import ctypes

    lib = hp.load()
    colptr = np.array([0, 2, 4, 5], np.int64)
    rowind = np.array([0, 1, 1, 2, 2], np.int32)
    n = 3
    out = np.empty(3, np.int64)
    if bad == "n":
        n = -1
    elif bad == "colptr0":
        colptr = np.array([1, 2, 4, 5], np.int64)
    elif bad == "nonmono":
        colptr = np.array([0, 3, 2, 5], np.int64)
    elif bad == "upper":
        rowind = np.array([0, 0, 1, 2, 2], np.int32)
    elif bad == "unsorted":
        rowind = np.array([1, 0, 1, 2, 2], np.int32)
    elif bad == "range":
        rowind = np.array([0, 1, 1, 3, 2], np.int32)
    ptr = None if bad == "out" else out.ctypes.data
    rc = lib.spchol_order_nd(n, colptr.ctypes.data, rowind.ctypes.data, ctypes.c_void_p(ptr))
    assert rc == code
