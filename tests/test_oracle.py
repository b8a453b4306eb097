"""Pins for the CPU oracle: each test checks it against something other than itself.

* The paper's worked example (Fig. 1): exact factor structure, fill, supernodes
  and supernodal elimination tree.
* Brute-force symbolic elimination on dense boolean matrices (the elimination
  game) for random patterns and orderings.
* LAPACK's dense Cholesky (through numpy) on dense SPD inputs.
* Closed forms: the 1D Laplacian factor, diagonal matrices, and an exactly
  representable factor.
* Non-SPD detection at a known column, berr against a dense recomputation.
* fact_err of perturbed factors against the dense product formed by numpy /
  scipy, closed forms with exact arithmetic, and +inf outside the pattern.
* Symbolic counts of the nested-dissection grids against reference counts
  computed independently (``golden/nd_counts.txt``).
"""
import numpy as np
import pytest
import scipy.sparse as sp

import gridgen
import oracle
from tests import fig1


def _csc_from_dense_lower(M):
    L = sp.csc_matrix(np.tril(M))
    L.sort_indices()
    # keep explicit structural entries only where M is nonzero
    return L.shape[0], L.indptr.astype(np.int64), L.indices.astype(np.int32), L.data.astype(np.float64)


def _dense_from_L(n, Lp, Li, Lx):
    L = np.zeros((n, n))
    for j in range(n):
        for p in range(Lp[j], Lp[j + 1]):
            L[Li[p], j] = Lx[p]
    return L


def _pattern_from_L(n, Lp, Li):
    return {(int(Li[p]), j) for j in range(n) for p in range(Lp[j], Lp[j + 1])}


# --------------------------------------------------------------------------- Fig. 1


def test_fig1_structure_matches_paper():
    n, a_pat, fill, blocks, edges = fig1.load()
    assert n == 30
    assert len(fill) == 9
    assert not (a_pat & fill)
    colptr, rowind, vals = fig1.spd_from_pattern(n, a_pat)
    f = oracle.OracleFactor(n, colptr, rowind, vals, None)
    Lp, Li, _ = f.L()
    # exact structure of L: original entries plus exactly the drawn fill
    assert _pattern_from_L(n, Lp, Li) == a_pat | fill
    # supernodes by the paper's definition are the drawn diagonal blocks
    start = f.supernodes()
    want = [blocks[k][0] for k in sorted(blocks)] + [n]
    assert list(start) == want
    # supernodal elimination tree of Fig. 1b
    parent, cc = f.structure()
    sn_of = np.searchsorted(start, np.arange(n), side="right") - 1
    got = {}
    for s in range(len(start) - 1):
        last = start[s + 1] - 1
        if parent[last] >= 0:
            got[s + 1] = int(sn_of[parent[last]]) + 1
    assert got == edges
    # counts implied by the figure
    assert f.nnzL == len(a_pat | fill)
    assert int(f.flops) == int(np.sum(cc.astype(np.int64) ** 2))
    assert f.factor() == 0
    assert f.fact_err() <= 1e-15


def test_fig1_supernodes_are_not_fundamental():
    # Column 11 (0-based) lies inside supernode 5 (columns 10..15) and has two
    # elimination-tree children, columns 3 and 10.  The paper's definition
    # (Section II-B) keeps it in supernode 5; a fundamental-supernode partition
    # would start a new supernode there.
    n, a_pat, fill, blocks, edges = fig1.load()
    colptr, rowind, vals = fig1.spd_from_pattern(n, a_pat)
    f = oracle.OracleFactor(n, colptr, rowind, vals, None)
    parent, cc = f.structure()
    assert sorted(int(c) for c in np.nonzero(parent == 11)[0]) == [3, 10]
    assert blocks[5] == (10, 16)
    assert int(np.sum(cc)) == 155 and int(np.sum(cc ** 2)) == 903


# --------------------------------------------------------------------------- brute force


def _elimination_game(G):
    """Dense boolean symbolic elimination: returns the lower pattern of L."""
    G = G.copy()
    n = G.shape[0]
    for k in range(n):
        nz = np.nonzero(G[k + 1:, k])[0] + k + 1
        for a in nz:
            G[a, nz[nz <= a]] = True
    return {(i, j) for j in range(n) for i in range(j, n) if G[i, j] or i == j}


@pytest.mark.parametrize("seed", range(12))
def test_symbolic_vs_elimination_game(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(1, 41))
    dens = rng.uniform(0.02, 0.3)
    M = np.tril(rng.random((n, n)) < dens, -1)
    M = M | M.T
    A = np.where(M, -rng.uniform(0.1, 1.0, (n, n)), 0.0)
    A = np.tril(A) + np.tril(A, -1).T
    A[np.diag_indices(n)] = np.abs(A).sum(1) + 1.0
    perm = rng.permutation(n).astype(np.int64)
    n_, colptr, rowind, vals = _csc_from_dense_lower(A)
    f = oracle.OracleFactor(n, colptr, rowind, vals, perm)
    P = A[np.ix_(perm, perm)]
    want = _elimination_game(P != 0)
    Lp, Li, _ = f.L()
    assert _pattern_from_L(n, Lp, Li) == want
    parent, cc = f.structure()
    for j in range(n):
        below = sorted(i for (i, jj) in want if jj == j and i > j)
        assert parent[j] == (below[0] if below else -1)
        assert cc[j] == len(below) + 1
    assert f.flops == float(sum(int(c) ** 2 for c in cc))
    # numeric factor of P A P^T against LAPACK
    assert f.factor() == 0
    L = _dense_from_L(n, *f.L())
    np.testing.assert_allclose(L, np.linalg.cholesky(P), rtol=0, atol=1e-13 * np.abs(P).max())


# --------------------------------------------------------------------------- dense / closed forms


@pytest.mark.parametrize("n", [1, 2, 3, 7, 16, 31])
def test_dense_spd_vs_lapack(n):
    rng = np.random.default_rng(n)
    G = rng.standard_normal((n, n))
    A = G @ G.T + n * np.eye(n)
    _, colptr, rowind, vals = _csc_from_dense_lower(A)
    perm = rng.permutation(n).astype(np.int64)
    f = oracle.OracleFactor(n, colptr, rowind, vals, perm)
    assert f.factor() == 0
    L = _dense_from_L(n, *f.L())
    ref = np.linalg.cholesky(A[np.ix_(perm, perm)])
    np.testing.assert_allclose(L, ref, rtol=1e-13, atol=1e-14 * np.abs(ref).max())
    assert f.fact_err() <= 1e-14
    b = rng.uniform(-1, 1, (n, 3))
    x = f.solve(b)
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("n", [1, 2, 5, 50, 1000])
def test_1d_laplacian_closed_form(n):
    # tridiag(-1, 2, -1): l_kk = sqrt((k+1)/k), l_{k+1,k} = -sqrt(k/(k+1)) (1-based k)
    colptr = np.zeros(n + 1, np.int64)
    rows, vals = [], []
    for j in range(n):
        rows.append(j)
        vals.append(2.0)
        if j + 1 < n:
            rows.append(j + 1)
            vals.append(-1.0)
        colptr[j + 1] = len(rows)
    f = oracle.OracleFactor(n, colptr, np.array(rows, np.int32), np.array(vals), None)
    parent, cc = f.structure()
    assert list(parent) == list(range(1, n)) + [-1]
    assert list(cc) == [2] * (n - 1) + [1]
    assert f.factor() == 0
    Lp, Li, Lx = f.L()
    k = np.arange(1, n + 1, dtype=np.float64)
    diag = Lx[Lp[:-1]]
    np.testing.assert_allclose(diag, np.sqrt((k + 1) / k), rtol=4e-16 * max(1.0, np.sqrt(n)))
    sub = np.array([Lx[Lp[j] + 1] for j in range(n - 1)])
    np.testing.assert_allclose(sub, -np.sqrt(k[:-1] / (k[:-1] + 1)), rtol=4e-16 * max(1.0, np.sqrt(n)))
    # exact solution of A x = e_1: x_i = (n + 1 - i) / (n + 1) (1-based i)
    e1 = np.zeros((n, 1))
    e1[0] = 1.0
    x = f.solve(e1)[:, 0]
    np.testing.assert_allclose(x, (n + 1 - k) / (n + 1), rtol=1e-12, atol=1e-14)


def test_diagonal_is_exact_sqrt():
    rng = np.random.default_rng(7)
    d = rng.uniform(0.5, 9.0, 40)
    colptr = np.arange(41, dtype=np.int64)
    f = oracle.OracleFactor(40, colptr, np.arange(40, dtype=np.int32), d, rng.permutation(40))
    assert f.factor() == 0
    Lp, Li, Lx = f.L()
    perm = f.perm
    assert np.array_equal(Lx, np.sqrt(d[perm]))


def test_exactly_representable_factor():
    # A = L0 L0^T with L0 = bidiag(2, -1): Cholesky reproduces L0 bit for bit.
    n = 25
    L0 = 2.0 * np.eye(n) - np.eye(n, k=-1)
    A = L0 @ L0.T
    _, colptr, rowind, vals = _csc_from_dense_lower(A)
    f = oracle.OracleFactor(n, colptr, rowind, vals, None)
    assert f.factor() == 0
    assert np.array_equal(_dense_from_L(n, *f.L()), L0)
    assert f.fact_err() == 0.0


def test_not_spd_reports_first_permuted_column():
    A = gridgen.laplacian_2d(12, shift=0.5)
    perm = gridgen.geometric_nd(A.dims)
    pinv = np.empty_like(perm)
    pinv[perm] = np.arange(A.n)
    for bad in (0, 77, A.n - 1, int(perm[0]), int(perm[-1])):
        vals = A.values.copy()
        vals[A.colptr[bad]] = -1.0  # diagonal entry comes first in each column
        f = oracle.OracleFactor(A.n, A.colptr, A.rowind, vals, perm)
        assert f.factor() == pinv[bad] + 1


def test_invalid_inputs_rejected():
    colptr = np.array([0, 2, 3], np.int64)
    with pytest.raises(ValueError):  # upper-triangle entry
        oracle.OracleFactor(2, colptr, np.array([0, 1, 0], np.int32), np.ones(3), None)
    with pytest.raises(ValueError):  # not a permutation
        oracle.OracleFactor(2, colptr, np.array([0, 1, 1], np.int32), np.ones(3), np.array([0, 0]))


# --------------------------------------------------------------------------- grids, norms


def test_berr_matches_dense_definition():
    A = gridgen.diffusion_2d_5pt(9, sigma=1.0, seed=3)
    F = A.to_scipy_full().toarray()
    rng = np.random.default_rng(1)
    X = rng.standard_normal((A.n, 3))
    B = rng.standard_normal((A.n, 3))
    want = max(np.abs(B[:, k] - F @ X[:, k]).max() /
               (np.abs(F).sum(1).max() * np.abs(X[:, k]).max() + np.abs(B[:, k]).max())
               for k in range(3))
    assert abs(oracle.berr(A, X, B) - want) <= 1e-15 * want


@pytest.mark.parametrize("name", ["lap2d_64", "lap3d_8", "lap3d_16", "diff3d_8", "diff2d_20"])
def test_grids_fact_err_and_berr(name):
    A, perm, b = gridgen.workload(name)
    f = oracle.OracleFactor.from_csc(A, perm)
    assert f.factor() == 0
    assert f.fact_err() <= 1e-14
    x = f.solve(b)
    assert oracle.berr(A, x, b) <= 1e-15 * 10
    # permutation invariance of the solution
    g = oracle.OracleFactor.from_csc(A, None)
    assert g.factor() == 0
    x0 = g.solve(b)
    cond_bound = 1e-9
    assert np.abs(x - x0).max() <= cond_bound * max(1.0, np.abs(x0).max())


def test_grid_solution_against_scipy():
    A, perm, b = gridgen.workload("diff3d_6")
    f = oracle.OracleFactor.from_csc(A, perm)
    assert f.factor() == 0
    x = f.solve(b)
    import scipy.sparse.linalg as sla
    ref = sla.spsolve(A.to_scipy_full(), b[:, 0])
    np.testing.assert_allclose(x[:, 0], ref, rtol=1e-9, atol=1e-12 * np.abs(ref).max())


def test_nd_fill_far_below_natural_order():
    A = gridgen.laplacian_3d(10)
    nd = oracle.OracleFactor.from_csc(A, gridgen.geometric_nd(A.dims))
    nat = oracle.OracleFactor.from_csc(A, None)
    assert nd.nnzL < 0.8 * nat.nnzL


# --------------------------------------------------------------------------- fact_err


def _dense_lower_csc(M):
    """Every lower entry of M as a structural entry (a dense lower pattern)."""
    n = M.shape[0]
    Lp = np.zeros(n + 1, np.int64)
    Li, Lx = [], []
    for j in range(n):
        for i in range(j, n):
            Li.append(i)
            Lx.append(M[i, j])
        Lp[j + 1] = len(Li)
    return Lp, np.array(Li, np.int64), np.array(Lx, np.float64)


@pytest.mark.parametrize("seed", range(4))
def test_fact_err_perturbed_dense_vs_numpy(seed):
    # A perturbed Cholesky factor has a known, nonzero ||LL^T - A||_F / ||A||_F,
    # computed here from the full dense matrices with numpy.  A value off by the
    # weight of the mirrored off-diagonal entries, by a wrong norm of A or by a
    # constant zero fails this.
    rng = np.random.default_rng(seed)
    n = 7
    G = rng.standard_normal((n, n))
    A = G @ G.T + n * np.eye(n)
    L = np.linalg.cholesky(A)
    L[4, 1] += 1e-3 * (1 + seed)
    L[5, 5] *= 1 + 2e-3
    L[6, 0] -= 5e-4
    want = np.linalg.norm(L @ L.T - A, "fro") / np.linalg.norm(A, "fro")
    Lp, Li, Lx = _dense_lower_csc(L)
    Bp, Bi, Bx = _dense_lower_csc(A)
    got = oracle.fact_err_csc(n, Lp, Li, Lx, Bp, Bi, Bx)
    assert want > 1e-5
    assert abs(got - want) <= 1e-12 * want


def test_fact_err_only_off_diagonal_and_only_diagonal_perturbations():
    # The two halves of the sum separately: an error only off the diagonal of
    # LL^T (counted twice in the Frobenius norm of the symmetric difference) and
    # an error only on it.
    A = np.diag([4.0, 9.0, 16.0])
    Bp, Bi, Bx = _dense_lower_csc(A)
    # L = diag(2, 3, 4) with l_10 = d: (LL^T)_{10} = 2d, (LL^T)_{11} = 9 + d^2.
    d = 2.0**-10  # powers of two: every product and difference is exact
    L = np.diag([2.0, 3.0, 4.0])
    L[1, 0] = d
    Lp, Li, Lx = _dense_lower_csc(L)
    want = np.sqrt(2 * (2 * d) ** 2 + d**4) / np.sqrt(16 + 81 + 256)
    assert abs(oracle.fact_err_csc(3, Lp, Li, Lx, Bp, Bi, Bx) - want) <= 1e-14 * want
    # only the diagonal: l_22 = 4 + e gives (LL^T)_{22} - 16 = 8e + e^2.
    e = 2.0**-13
    L = np.diag([2.0, 3.0, 4.0 + e])
    Lp, Li, Lx = _dense_lower_csc(L)
    want = abs(8 * e + e * e) / np.sqrt(16 + 81 + 256)
    assert abs(oracle.fact_err_csc(3, Lp, Li, Lx, Bp, Bi, Bx) - want) <= 1e-12 * want


def test_fact_err_of_handle_equals_csc_form_and_perturbed_sparse_factor():
    A, perm, _ = gridgen.workload("lap2d_16")
    f = oracle.OracleFactor.from_csc(A, perm)
    assert f.factor() == 0
    Lp, Li, Lx = f.L()
    Bp, Bi, Bx = f.B()
    n = A.n
    assert oracle.fact_err_csc(n, Lp, Li, Lx, Bp, Bi, Bx) == f.fact_err()
    # perturb one off-diagonal and one diagonal entry of the sparse factor and
    # compare with the product formed by scipy on the full symmetric matrices
    Lx2 = Lx.copy()
    off = next(p for j in range(n // 2, n) for p in range(Lp[j] + 1, Lp[j + 1]))
    Lx2[off] += 1e-6
    Lx2[Lp[n // 3]] *= 1 + 1e-7
    Ls = sp.csc_matrix((Lx2, Li, Lp), shape=(n, n))
    Bl = sp.csc_matrix((Bx, Bi, Bp), shape=(n, n))
    Bfull = Bl + Bl.T - sp.diags(Bl.diagonal())
    D = (Ls @ Ls.T - Bfull).toarray()
    want = np.linalg.norm(D, "fro") / np.linalg.norm(Bfull.toarray(), "fro")
    got = oracle.fact_err_csc(n, Lp, Li, Lx2, Bp, Bi, Bx)
    assert want > 1e-8
    assert abs(got - want) <= 1e-9 * want


def test_fact_err_outside_pattern_is_inf():
    # A product entry outside L's pattern: column 0 holds rows 0, 1, 2, so
    # l_20 l_10 lands at (2, 1), which column 1 (row 1 only) does not hold.
    Lp = np.array([0, 3, 4, 5], np.int64)
    Li = np.array([0, 1, 2, 1, 2], np.int64)
    Lx = np.array([2.0, 0.5, 0.25, 3.0, 4.0])
    Bp, Bi, Bx = _dense_lower_csc(np.diag([4.0, 9.0, 16.0]))
    assert oracle.fact_err_csc(3, Lp, Li, Lx, Bp, Bi, Bx) == np.inf
    # An entry of B outside L's pattern (L diagonal, b_10 != 0).
    Lp = np.array([0, 1, 2, 3], np.int64)
    Li = np.array([0, 1, 2], np.int64)
    Lx = np.array([2.0, 3.0, 4.0])
    B = np.diag([4.0, 9.0, 16.0])
    B[1, 0] = B[0, 1] = 1.0
    Bp, Bi, Bx = _dense_lower_csc(B)
    Bx[Bx == 0] = 0.0
    assert oracle.fact_err_csc(3, Lp, Li, Lx, Bp, Bi, Bx) == np.inf


# --------------------------------------------------------------------------- ND counts


def _golden_nd_counts():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "nd_counts.txt")
    rows = []
    for line in open(path):
        line = line.split("#", 1)[0].split()
        if line:
            rows.append((line[0], float(line[1]), float(line[2])))
    return rows


def _sig4(x):
    return float(f"{x:.3e}")


@pytest.mark.parametrize("name,nnzl,flops", _golden_nd_counts())
def test_nd_reference_counts(name, nnzl, flops):
    # The geometric dissection of the grid recipe and the oracle's symbolic
    # pass together reproduce counts computed independently of this code.
    A, perm, _ = gridgen.workload(name)
    f = oracle.OracleFactor.from_csc(A, perm)
    if name == "lap2d_8":
        assert f.nnzL == int(nnzl) and int(f.flops) == int(flops)
    else:
        assert _sig4(f.nnzL) == nnzl
        assert _sig4(f.flops) == flops
