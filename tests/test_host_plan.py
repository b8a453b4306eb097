"""Host logic without a GPU: the symbolic plan against the oracle, its
invariants, and the task protocol run in random ready orders (Section II-C: any
order that respects the dependencies gives the same factor up to rounding)."""
import numpy as np
import pytest

import gridgen
import oracle
from paper_1608_00044_gb300 import build
from paper_1608_00044_gb300 import hostplan as hp
from tests import fig1

build.build_host()


def _plan(A, perm, **kw):
    return hp.HostPlan(A.n, A.colptr, A.rowind, perm, **kw)


@pytest.mark.parametrize("name", ["lap2d_64", "lap3d_12", "diff3d_9", "diff2d_21"])
@pytest.mark.parametrize("W", [1, 7, 64, 128])
def test_counts_and_etree_match_oracle(name, W):
    A, perm, b = gridgen.workload(name)
    P = _plan(A, perm, max_width=W)
    fperm = P.get(hp.PERM)
    assert sorted(fperm) == list(range(A.n))
    f = oracle.OracleFactor.from_csc(A, fperm)
    parent, cc = f.structure()
    assert np.array_equal(P.get(hp.COLCOUNT), cc)
    assert np.array_equal(P.get(hp.ETREE), parent)
    assert P.flops == f.flops
    assert P.scalars()["nnz_l"] == f.nnzL


@pytest.mark.parametrize("seed", range(8))
def test_counts_on_random_patterns_match_oracle(seed):
    """Column counts (computed without forming L) against the oracle's symbolic
    elimination on random patterns: forests, dense blocks, isolated columns,
    some diagonal entries absent from the pattern, random orderings."""
    import scipy.sparse as sp

    rng = np.random.default_rng(900 + seed)
    n = int(rng.integers(1, 400))
    M = sp.random(n, n, density=float(rng.uniform(0.0, 0.03)), random_state=rng, format="csc")
    M = (M + M.T).tocsc()
    if seed % 2 == 0:  # a dense block
        k = int(rng.integers(1, min(n, 40) + 1))
        o = int(rng.integers(0, n - k + 1))
        D = sp.lil_matrix((n, n))
        D[o:o + k, o:o + k] = 1.0
        M = (M + D.tocsc()).tocsc()
    d = np.ones(n)
    if seed % 3 == 0:  # some diagonal entries absent
        d[rng.random(n) < 0.2] = 0.0
    M = (sp.tril(M, -1) + sp.diags(d)).tocsc()
    M.eliminate_zeros()
    M.sort_indices()
    A = gridgen.CscLower(n, M.indptr.astype(np.int64), M.indices.astype(np.int32), np.ones(M.nnz))
    P = _plan(A, rng.permutation(n), max_width=int(rng.choice([1, 16, 64])))
    fperm = P.get(hp.PERM)
    f = oracle.OracleFactor.from_csc(A, fperm)
    parent, cc = f.structure()
    assert np.array_equal(P.get(hp.COLCOUNT), cc)
    assert np.array_equal(P.get(hp.ETREE), parent)


def test_fig1_supernodes_without_amalgamation():
    n, a_pat, fill, blocks, edges = fig1.load()
    colptr, rowind, vals = fig1.spd_from_pattern(n, a_pat)
    P = hp.HostPlan(n, colptr, rowind, None, max_width=128, relax_zeros=0)
    assert np.array_equal(P.get(hp.PERM), np.arange(n))  # the figure's order is already a postorder
    fcol = P.get(hp.FCOL)
    assert list(fcol) == [blocks[k][0] for k in sorted(blocks)] + [n]
    par = P.get(hp.PARENT)
    assert {s + 1: int(par[s]) + 1 for s in range(len(par)) if par[s] >= 0} == edges


def _panel_rows(P):
    fcol, nrows, rowoff, rows = P.get(hp.FCOL), P.get(hp.NROWS), P.get(hp.ROWOFF), P.get(hp.ROWS)
    return [rows[rowoff[s]:rowoff[s] + nrows[s]] for s in range(len(nrows))], fcol


@pytest.mark.parametrize("relax,W", [(0, 128), (4, 64), (4, 16), (9, 32)])
def test_panel_structure_invariants(relax, W):
    A, perm, b = gridgen.workload("lap3d_12")
    P = _plan(A, perm, max_width=W, relax_zeros=relax)
    f = oracle.OracleFactor.from_csc(A, P.get(hp.PERM))
    Lp, Li, _ = f.L()
    cc = P.get(hp.COLCOUNT)
    R, fcol = _panel_rows(P)
    for s, rows in enumerate(R):
        w = fcol[s + 1] - fcol[s]
        assert 1 <= w <= W
        # the diagonal block first, then strictly increasing rows below it
        assert np.array_equal(rows[:w], np.arange(fcol[s], fcol[s + 1]))
        assert np.all(np.diff(rows) > 0)
        for j in range(fcol[s], fcol[s + 1]):
            exact = Li[Lp[j]:Lp[j + 1]]
            stored = rows[rows >= j]
            # every structural nonzero of column j is stored; extra rows are amalgamation zeros
            assert set(exact) <= set(stored)
            assert len(stored) - cc[j] <= relax
        if relax == 0:
            j = fcol[s]
            assert np.array_equal(rows, Li[Lp[j]:Lp[j + 1]])


def test_update_tiles_cover_and_relative_indices():
    A, perm, b = gridgen.workload("diff3d_9")
    P = _plan(A, perm, max_width=32)
    R, fcol = _panel_rows(P)
    ut = P.get(hp.UTASKS).reshape(-1, 6)
    depf = P.get(hp.DEPF)
    assert np.array_equal(np.bincount(ut[:, 1], minlength=len(R)), depf)
    for s, t, seg0, seglen, row0, rowlen in ut:
        rs, rt = R[s], R[t]
        seg = rs[seg0:seg0 + seglen]
        # the segment is exactly s's rows inside t's columns
        assert np.all((seg >= fcol[t]) & (seg < fcol[t + 1]))
        assert seg0 >= fcol[s + 1] - fcol[s] and row0 >= seg0
        # rows of the tile exist in t's row list (relative indices are defined)
        tile = rs[row0:row0 + rowlen]
        pos = np.searchsorted(rt, tile)
        assert np.all(pos < len(rt)) and np.array_equal(rt[pos], tile)
        assert np.all(np.diff(pos) > 0)  # monotone map
    # tiles of each (s, t) pair cover rows seg0 .. end exactly once
    for (s, t) in {(int(a), int(b)) for a, b in ut[:, :2]}:
        sel = ut[(ut[:, 0] == s) & (ut[:, 1] == t)]
        covered = np.concatenate([np.arange(r0, r0 + rl) for r0, rl in sel[:, 4:6]])
        assert np.array_equal(np.sort(covered), np.arange(sel[0, 2], len(R[s])))


@pytest.mark.parametrize("seed", range(5))
def test_random_orders_reach_oracle_accuracy(seed):
    A, perm, b = gridgen.workload("diff3d_8")
    B = gridgen.rhs_uniform(A.n, 3, seed=seed)
    P = _plan(A, perm, max_width=[1, 8, 16, 64, 128][seed])
    rc, X, pool = P.simulate(A.values, B, seed=seed)
    assert rc == 0
    assert oracle.berr(A, X, B) <= 1e-14
    f = oracle.OracleFactor.from_csc(A, P.get(hp.PERM))
    f.factor()
    np.testing.assert_allclose(X, f.solve(B), rtol=1e-11, atol=1e-13)


def test_simulated_not_spd_column():
    A, perm, b = gridgen.workload("lap2d_24")
    P = _plan(A, perm)
    fperm = P.get(hp.PERM)
    pinv = np.empty_like(fperm)
    pinv[fperm] = np.arange(A.n)
    for bad in (3, 300, int(fperm[-1])):
        vals = A.values.copy()
        vals[A.colptr[bad]] = -2.0
        for seed in range(3):
            rc, _, _ = P.simulate(vals, None, seed=seed)
            assert rc == pinv[bad] + 1


@pytest.mark.parametrize("bad,arg", [
    ("colptr0", -2), ("nonmono", -2), ("upper", -3), ("unsorted", -3), ("dup", -3), ("range", -3), ("perm", -4),
])
def test_invalid_arguments(bad, arg):
    colptr = np.array([0, 2, 4, 5], np.int64)
    rowind = np.array([0, 1, 1, 2, 2], np.int32)
    perm = None
    if bad == "colptr0":
        colptr = colptr + 1
    elif bad == "nonmono":
        colptr = np.array([0, 3, 2, 5], np.int64)
    elif bad == "upper":
        rowind = np.array([0, 1, 0, 2, 2], np.int32)
    elif bad == "unsorted":
        rowind = np.array([1, 0, 1, 2, 2], np.int32)
    elif bad == "dup":
        rowind = np.array([0, 0, 1, 2, 2], np.int32)
    elif bad == "range":
        rowind = np.array([0, 3, 1, 2, 2], np.int32)
    elif bad == "perm":
        perm = np.array([0, 0, 1], np.int64)
    with pytest.raises(ValueError) as ei:
        hp.HostPlan(3, colptr, rowind, perm)
    assert str(arg) in str(ei.value)


def test_nested_dissection_top_separator():
    perm = gridgen.geometric_nd((64, 64, 64))
    top = perm[-4096:]
    x = top // (64 * 64)
    assert np.all(x == 32)
    # the ordering is already a postorder of the elimination tree on a smaller grid
    A = gridgen.laplacian_3d(12)
    P = _plan(A, gridgen.geometric_nd(A.dims))
    assert np.array_equal(P.get(hp.PERM), gridgen.geometric_nd(A.dims))


def test_amalgamation_reduces_panels_within_budget():
    A, perm, b = gridgen.workload("lap3d_16")
    p0 = _plan(A, perm, relax_zeros=0).scalars()
    p4 = _plan(A, perm, relax_zeros=4).scalars()
    assert p4["ns"] < p0["ns"]
    assert p4["nnz_l_stored"] >= p4["nnz_l"] == p0["nnz_l"]


@pytest.mark.parametrize("name,W", [("lap3d_12", 16), ("diff3d_9", 8), ("lap2d_64", 64)])
def test_high_priority_tiles_are_parent_tiles_near_the_root(name, W):
    """The update tiles scheduled with high priority are, for the panels within
    128 levels of the root, the leading tiles of each panel, exactly those into
    its etree parent; the ring sizes add up to the task count."""
    A, perm, b = gridgen.workload(name)
    P = _plan(A, perm, max_width=W)
    sc = P.scalars()
    par = P.get(hp.PARENT)
    nu, nuhi = P.get(hp.NU), P.get(hp.NUHI)
    ut = P.get(hp.UTASKS).reshape(-1, 6)
    ns = len(par)
    depth = np.zeros(ns, int)
    for s in range(ns - 1, -1, -1):
        depth[s] = 0 if par[s] < 0 else depth[par[s]] + 1
    first = np.concatenate([[0], np.cumsum(nu)])
    for s in range(ns):
        tiles = ut[first[s]:first[s + 1]]
        n_par = int(np.sum(tiles[:, 1] == par[s])) if par[s] >= 0 else 0
        assert nuhi[s] == (n_par if depth[s] < 128 else 0)
        assert np.all(tiles[:nuhi[s], 1] == par[s])
    # scheduled tasks: one per subtree task, and for each panel outside the
    # subtree tasks its diagonal task, panel-solve tiles and update tiles (the
    # leading parent tiles near the root in the high-priority ring)
    ntr = P.get(hp.NTRSM)
    lo, hi = P.get(hp.SUBLO), P.get(hp.SUBHI)
    inside = np.zeros(ns, bool)
    for a, b in zip(lo, hi):
        inside[a:b + 1] = True
    out = ~inside
    assert sc["n_sub"] == len(lo)
    assert sc["n_hi_tasks"] == len(lo) + int((1 + ntr[out] + nuhi[out]).sum())
    assert sc["factor_tasks"] == len(lo) + int((1 + ntr[out] + nu[out]).sum())
    assert 0 < sc["n_hi_tasks"] <= sc["factor_tasks"]



@pytest.mark.parametrize("name,W", [("lap3d_20", 8), ("lap2d_64", 16), ("diff3d_9", 64)])
def test_subtree_tasks_are_maximal_small_subtrees(name, W):
    """Subtree tasks are disjoint, each exactly the set of descendants of its
    root (a contiguous range in the postorder), within the flop budget
    (1e6, capped at 1/4096 of the whole factorization), and maximal: the
    root's parent's subtree exceeds the budget."""
    A, perm, b = gridgen.workload(name)
    P = _plan(A, perm, max_width=W)
    par, fcol, nrows = P.get(hp.PARENT), P.get(hp.FCOL), P.get(hp.NROWS)
    ut = P.get(hp.UTASKS).reshape(-1, 6)
    lo, hi = P.get(hp.SUBLO), P.get(hp.SUBHI)
    ns = len(par)
    w = np.diff(fcol).astype(float)
    fl = w ** 3 / 3 + (nrows - w) * w ** 2
    np.add.at(fl, ut[:, 0], 2.0 * w[ut[:, 0]] * ut[:, 5] * ut[:, 3])
    sub = fl.copy()
    for s in range(ns):
        if par[s] >= 0:
            sub[par[s]] += sub[s]
    seen = np.zeros(ns, bool)
    assert len(lo) > 0
    for a, r in zip(lo, hi):
        assert a < r and not seen[a:r + 1].any()
        seen[a:r + 1] = True
        # descendants of r: walk every panel of the range up to r
        for q in range(a, r + 1):
            x = q
            while x != r:
                x = par[x]
                assert a <= x <= r
        if a > 0:  # the panel before the range is not a descendant of r
            x = a - 1
            while x >= 0 and x != r:
                x = par[x]
            assert x != r
        budget = min(1e6, sub[par < 0].sum() / 4096)
        assert sub[r] <= budget * (1 + 1e-9)
        assert par[r] < 0 or sub[par[r]] > budget


def test_random_order_with_subtree_tasks():
    """A plan with subtree tasks runs the protocol (subtree tasks alongside the
    panel-level tasks of the rest) to the oracle's accuracy."""
    A, perm, b = gridgen.workload("lap3d_20")
    P = _plan(A, perm, max_width=16)
    assert P.scalars()["n_sub"] > 0
    B = gridgen.rhs_uniform(A.n, 2, seed=3)
    for seed in range(3):
        rc, X, pool = P.simulate(A.values, B, seed=seed)
        assert rc == 0
        assert oracle.berr(A, X, B) <= 1e-14


@pytest.mark.parametrize("name,W", [("diff3d_8", 16), ("lap3d_12", 64), ("lap2d_24", 8)])
def test_deterministic_order_is_bitwise_stable(name, W):
    """Deterministic mode (the static (target, source) order of Section IV-B):
    the update tiles into a target and the solve tiles into a panel run in one
    fixed order, so the simulated factor and solution are bitwise equal in
    every random ready order -- and still match the oracle.  The dynamic mode
    differs between orders in the last bits (a check that the test can see a
    difference)."""
    A, perm, b = gridgen.workload(name)
    B = gridgen.rhs_uniform(A.n, 3, seed=2)
    results = {}
    for det in (0, 1, 2):
        P = _plan(A, perm, deterministic=det, max_width=W)
        if det:
            assert P.scalars()["n_sub"] == 0  # no subtree tasks in this mode
        outs = []
        for seed in range(4):
            rc, X, pool = P.simulate(A.values, B, seed=seed, want_pool=True)
            assert rc == 0
            assert oracle.berr(A, X, B) <= 1e-14
            outs.append((X, pool))
        results[det] = all(np.array_equal(outs[0][0], o[0]) and np.array_equal(outs[0][1], o[1]) for o in outs[1:])
    assert results[1] and results[2]
    assert not results[0]


@pytest.mark.parametrize("name,W", [("diff3d_8", 16), ("lap3d_12", 64), ("lap2d_24", 8), ("diff3d_10", 128)])
def test_fanin_gather_lists(name, W):
    """Fan-in mode (deterministic = 2): every update tile's rows are listed
    exactly once over the row pieces of its target, in order and without
    gaps; each piece's list is in update-tile order (the fixed order in which
    an entry receives its updates); a piece holds at most 32 consecutive row
    positions of one target, never across the end of its diagonal block, and
    the diagonal block's pieces start at multiples of 32.  Positions are found
    here by a search in the target's row list, independently of the plan."""
    A, perm, b = gridgen.workload(name)
    P = _plan(A, perm, deterministic=2, max_width=W)
    ut = P.get(hp.UTASKS).reshape(-1, 6)
    fcol, rows, rowoff = P.get(hp.FCOL), P.get(hp.ROWS), P.get(hp.ROWOFF)
    off, task, ptr = P.get(hp.FANOFF), P.get(hp.FANTASK), P.get(hp.FANPTR)
    ent = P.get(hp.FANENT).reshape(-1, 3)
    ns = len(fcol) - 1
    assert len(off) == len(ut) + 1 and np.array_equal(np.diff(off), ut[:, 3] * ut[:, 5])
    assert len(task) == ns + P.scalars()["n_trsm"] and ptr[0] == 0 and ptr[-1] == len(ent)
    assert np.unique(task).size == task.size and task.min() == 0 and task.max() < len(ptr) - 1
    covered = [[] for _ in range(len(ut))]
    diag_piece = np.zeros(len(ptr) - 1, bool)
    for t in range(ns):
        w = fcol[t + 1] - fcol[t]
        diag_piece[task[t]:task[t] + (w + 31) // 32] = True
    for pc in range(len(ptr) - 1):
        es = ent[ptr[pc]:ptr[pc + 1]]
        if len(es) == 0:
            continue
        assert np.all(np.diff(es[:, 0]) > 0)  # update-tile order
        tgt = set(ut[es[:, 0], 1])
        assert len(tgt) == 1
        t = tgt.pop()
        Rt = rows[rowoff[t]:rowoff[t + 1]]
        w = fcol[t + 1] - fcol[t]
        pos = []
        for u, i0, i1 in es:
            s_, _, _, _, row0, rowlen = ut[u]
            assert 0 <= i0 < i1 <= rowlen
            g = rows[rowoff[s_] + row0 + i0: rowoff[s_] + row0 + i1]
            q = np.searchsorted(Rt, g)
            assert np.array_equal(Rt[q], g)
            pos.append(q)
            covered[u].append((i0, i1))
        pos = np.concatenate(pos)
        assert pos.max() - pos.min() < 32
        assert (pos.max() < w) == (pos.min() < w)  # never across the diagonal block's end
        if diag_piece[pc]:
            assert pos.max() < w and pos.min() // 32 == pos.max() // 32
    for u, c in enumerate(covered):
        c.sort()
        assert c[0][0] == 0 and c[-1][1] == ut[u, 5]
        assert all(a[1] == b_[0] for a, b_ in zip(c, c[1:]))
    # one gather task per piece that receives updates, on top of the static
    # order's tasks (which has no subtree tasks either)
    static = _plan(A, perm, deterministic=1, max_width=W).scalars()["factor_tasks"]
    assert P.scalars()["factor_tasks"] == static + int(np.count_nonzero(np.diff(ptr)))


@pytest.mark.parametrize("name,W", [("diff3d_8", 16), ("lap3d_12", 64), ("lap2d_24", 128)])
def test_fanin_reproduces_the_static_order_bitwise(name, W):
    """Fan-in aggregation adds each entry's updates in update-tile order, the
    order of the static (target, source) chains, so the two deterministic
    modes give bitwise the same factor and solution."""
    A, perm, b = gridgen.workload(name)
    B = gridgen.rhs_uniform(A.n, 2, seed=4)
    r1 = _plan(A, perm, deterministic=1, max_width=W).simulate(A.values, B, seed=3, want_pool=True)
    r2 = _plan(A, perm, deterministic=2, max_width=W).simulate(A.values, B, seed=5, want_pool=True)
    assert r1[0] == 0 and r2[0] == 0
    assert np.array_equal(r1[2], r2[2]) and np.array_equal(r1[1], r2[1])


@pytest.mark.parametrize("seed", range(4))
def test_fanin_on_random_spd_matrices(seed):
    """Fan-in mode on irregular patterns (random SPD matrices, random orderings,
    several panel widths): the simulated factor and solution are bitwise those
    of the static chains and meet the oracle's backward error."""
    import scipy.sparse as sp

    rng = np.random.default_rng(1300 + seed)
    n = int(rng.integers(50, 600))
    R = sp.random(n, n, density=float(rng.uniform(0.005, 0.03)), random_state=rng, format="csc")
    S = R + R.T
    S.data[:] = -np.abs(S.data)
    M = (S + sp.diags(np.asarray(np.abs(S).sum(axis=1)).ravel() + 1.0)).tocsc()
    L = sp.csc_matrix(sp.tril(M))
    L.sort_indices()
    A = gridgen.CscLower(n, L.indptr.astype(np.int64), L.indices.astype(np.int32), L.data.astype(np.float64))
    perm = rng.permutation(n)
    B = gridgen.rhs_uniform(n, 3, seed=seed)
    W = int(rng.choice([3, 16, 64, 128]))
    r1 = _plan(A, perm, deterministic=1, max_width=W).simulate(A.values, B, seed=1, want_pool=True)
    r2 = _plan(A, perm, deterministic=2, max_width=W).simulate(A.values, B, seed=2, want_pool=True)
    assert r1[0] == 0 and r2[0] == 0
    assert np.array_equal(r1[2], r2[2]) and np.array_equal(r1[1], r2[1])
    assert oracle.berr(A, r2[1], B) <= 1e-14


def test_fanin_matches_dynamic_to_rounding():
    """The fan-in factor equals the dynamic one up to rounding (only the order
    of the additions into each entry differs)."""
    A, perm, b = gridgen.workload("diff3d_10")
    _, _, L0 = _plan(A, perm).simulate(A.values, None, seed=1, want_pool=True)
    _, _, L2 = _plan(A, perm, deterministic=2).simulate(A.values, None, seed=1, want_pool=True)
    np.testing.assert_allclose(L2, L0, rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("name,W,depth", [("diff3d_8", 8, 1000), ("lap3d_12", 16, 1000), ("lap3d_12", 64, 3),
                                          ("lap2d_24", 4, 1000), ("lap2d_24", 8, -1)])
def test_w_panel_solve_protocol(name, W, depth):
    """The solves' W panels (W = L21 L11^{-1} kept for the panels near the root):
    their forward tiles are ready as soon as b_s is, their diagonal task runs
    after every forward tile of the panel has read b_s, their backward tiles
    after it, and the last backward tile releases the panel's readers.  Under
    random ready orders the simulated protocol runs exactly the tasks it
    should (the simulator checks every counter, and that the kept and pushed
    tasks are the non-seed tasks) and matches the oracle's solution."""
    A, perm, b = gridgen.workload(name)
    B = gridgen.rhs_uniform(A.n, 3, seed=W)
    P = _plan(A, perm, max_width=W, solve_w_depth=depth)
    f = oracle.OracleFactor.from_csc(A, P.get(hp.PERM))
    assert f.factor() == 0
    Xo = f.solve(B)
    for seed in range(4):
        rc, X, _ = P.simulate(A.values, B, seed=seed)
        assert rc == 0
        np.testing.assert_allclose(X, Xo, rtol=1e-11, atol=1e-13)
