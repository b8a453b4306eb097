"""Grid matrices in lower-triangular CSC form, plus seeded coefficients and RHS.

Conventions shared by every generator:

* Grid points are numbered in C order (axis 0 slowest): ``id = ravel(p, dims)``.
* The matrix is returned as the lower triangle of a symmetric matrix in CSC
  form: ``colptr`` (int64, length n+1), ``rowind`` (int32, sorted strictly
  increasing inside each column, diagonal first), ``values`` (float64).
* Dirichlet boundary with mesh width 1: a neighbour outside the grid is a ghost
  node whose coupling is kept on the diagonal and dropped off it.

The constant-coefficient stencils give the classic 2D 5-point (diagonal 4) and
3D 7-point (diagonal 6) Laplacians with off-diagonal -1.  The variable-coefficient
operators are weighted graph Laplacians plus ghost terms,
``A = sum_{edges uv} w_uv (e_u - e_v)(e_u - e_v)^T + sum_{ghosts} w_u e_u e_u^T``,
which is symmetric positive definite by construction whenever every weight is
positive and at least one ghost term exists.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp


@dataclass
class CscLower:
    """Lower triangle (diagonal included) of a symmetric matrix, CSC."""

    n: int
    colptr: np.ndarray  # int64[n+1]
    rowind: np.ndarray  # int32[nnz]
    values: np.ndarray  # float64[nnz]
    dims: tuple = ()
    kind: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.colptr[-1])

    def to_scipy_full(self) -> sp.csc_matrix:
        """Full symmetric matrix (for checks on the host only)."""
        L = sp.csc_matrix((self.values, self.rowind, self.colptr), shape=(self.n, self.n))
        D = sp.diags(L.diagonal())
        return (L + L.T - D).tocsc()


def _from_triplets(n, I, J, V, dims, kind, meta=None) -> CscLower:
    I = np.asarray(I, dtype=np.int64)
    J = np.asarray(J, dtype=np.int64)
    V = np.asarray(V, dtype=np.float64)
    lo = np.minimum(I, J)
    hi = np.maximum(I, J)
    M = sp.coo_matrix((V, (hi, lo)), shape=(n, n)).tocsc()
    M.sum_duplicates()
    M.sort_indices()
    return CscLower(
        n=n,
        colptr=M.indptr.astype(np.int64),
        rowind=M.indices.astype(np.int32),
        values=M.data.astype(np.float64),
        dims=tuple(dims),
        kind=kind,
        meta=dict(meta or {}),
    )


def _grid_ids(dims):
    return np.arange(int(np.prod(dims)), dtype=np.int64).reshape(dims)


def _neighbour_pairs(dims, offset):
    """(u, v) id pairs with v = u + offset, both inside the grid."""
    ids = _grid_ids(dims)
    src = [slice(None)] * len(dims)
    dst = [slice(None)] * len(dims)
    for a, d in enumerate(offset):
        if d > 0:
            src[a] = slice(0, dims[a] - d)
            dst[a] = slice(d, dims[a])
        elif d < 0:
            src[a] = slice(-d, dims[a])
            dst[a] = slice(0, dims[a] + d)
    return ids[tuple(src)].ravel(), ids[tuple(dst)].ravel()


def _half_offsets(ndim, full):
    """Stencil offsets with the first nonzero component positive (one per edge)."""
    out = []
    for off in itertools.product((-1, 0, 1), repeat=ndim):
        if not any(off):
            continue
        if not full and sum(abs(x) for x in off) != 1:
            continue
        first = next(x for x in off if x != 0)
        if first > 0:
            out.append(off)
    return out


def _laplacian(dims, shift, kind):
    ndim = len(dims)
    n = int(np.prod(dims))
    I = [np.arange(n)]
    J = [np.arange(n)]
    V = [np.full(n, 2.0 * ndim + shift)]
    for off in _half_offsets(ndim, full=False):
        u, v = _neighbour_pairs(dims, off)
        I.append(v)
        J.append(u)
        V.append(np.full(u.size, -1.0))
    return _from_triplets(n, np.concatenate(I), np.concatenate(J), np.concatenate(V),
                          dims, kind, {"shift": shift})


def laplacian_2d(nx: int, ny: int | None = None, shift: float = 0.0) -> CscLower:
    """2D 5-point Laplacian (diagonal 4 + shift, off-diagonal -1)."""
    ny = nx if ny is None else ny
    return _laplacian((nx, ny), shift, "lap2d5")


def laplacian_3d(nx: int, ny: int | None = None, nz: int | None = None,
                 shift: float = 0.0) -> CscLower:
    """3D 7-point Laplacian (diagonal 6 + shift, off-diagonal -1)."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    return _laplacian((nx, ny, nz), shift, "lap3d7")


def lognormal_kappa(dims, sigma: float, seed: int, clip: float = 2.303) -> np.ndarray:
    """Conductivity exp(sigma * clip(g, -clip, clip)), g iid N(0,1) per grid point.

    With sigma = 2 the values lie in [0.01, 100] (contrast 1e4); with sigma = 1
    in [0.1, 10] (contrast 1e2).  Drawn from ``default_rng(seed)``.
    """
    g = np.random.default_rng(seed).standard_normal(int(np.prod(dims)))
    return np.exp(sigma * np.clip(g, -clip, clip)).reshape(dims)


def _diffusion(dims, kappa, full_stencil, kind, meta):
    ndim = len(dims)
    n = int(np.prod(dims))
    k = np.asarray(kappa, dtype=np.float64).ravel()
    assert k.size == n and np.all(k > 0)
    diag = np.zeros(n)
    I, J, V = [], [], []
    for off in _half_offsets(ndim, full=full_stencil):
        s_off = 0.5 ** (sum(abs(x) for x in off) - 1)
        u, v = _neighbour_pairs(dims, off)
        w = s_off * 2.0 * k[u] * k[v] / (k[u] + k[v])
        I.append(v)
        J.append(u)
        V.append(-w)
        np.add.at(diag, u, w)
        np.add.at(diag, v, w)
    # Dirichlet ghosts: every stencil direction that leaves the grid.
    ids = _grid_ids(dims)
    for off in itertools.product((-1, 0, 1), repeat=ndim):
        if not any(off):
            continue
        if not full_stencil and sum(abs(x) for x in off) != 1:
            continue
        s_off = 0.5 ** (sum(abs(x) for x in off) - 1)
        outside = np.zeros(dims, dtype=bool)
        for a, d in enumerate(off):
            idx = [slice(None)] * ndim
            if d > 0:
                idx[a] = slice(dims[a] - d, dims[a])
                outside[tuple(idx)] = True
            elif d < 0:
                idx[a] = slice(0, -d)
                outside[tuple(idx)] = True
        u = ids[outside]
        np.add.at(diag, u, s_off * k[u])
    I.append(np.arange(n))
    J.append(np.arange(n))
    V.append(diag)
    return _from_triplets(n, np.concatenate(I), np.concatenate(J), np.concatenate(V),
                          dims, kind, meta)


def diffusion_3d_27pt(nx: int, sigma: float = 2.0, seed: int = 1,
                      ny: int | None = None, nz: int | None = None) -> CscLower:
    """3D 27-point variable-coefficient diffusion, SPD by construction.

    Edge weight ``s_off * 2 k_u k_v / (k_u + k_v)`` (harmonic mean), with
    ``s_off`` = 1 for faces, 1/2 for edges, 1/4 for corners; log-normal ``k``.
    """
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    dims = (nx, ny, nz)
    kappa = lognormal_kappa(dims, sigma, seed)
    return _diffusion(dims, kappa, True, "diff3d27", {"sigma": sigma, "seed": seed})


def neumann_laplacian_3d(nx: int, eps: float) -> CscLower:
    """3D 7-point graph Laplacian of the nx^3 grid (each diagonal entry the
    vertex's neighbour count: no Dirichlet boundary) plus eps * I: SPD with
    smallest eigenvalue eps (the constant vector), so kappa ~ 12 / eps --
    an ill-conditioned case for low-precision factors."""
    dims = (nx, nx, nx)
    n = nx ** 3
    I, J, V = [], [], []
    deg = np.zeros(n)
    for off in _half_offsets(3, full=False):
        u, v = _neighbour_pairs(dims, off)
        I.append(v)
        J.append(u)
        V.append(-np.ones(len(u)))
        np.add.at(deg, u, 1.0)
        np.add.at(deg, v, 1.0)
    I.append(np.arange(n))
    J.append(np.arange(n))
    V.append(deg + eps)
    return _from_triplets(n, np.concatenate(I), np.concatenate(J), np.concatenate(V), dims, "neumann3d",
                          {"eps": eps})


def diffusion_2d_5pt(nx: int, sigma: float = 1.0, seed: int = 1,
                     ny: int | None = None) -> CscLower:
    """2D 5-point variable-coefficient diffusion (harmonic-mean face weights)."""
    ny = nx if ny is None else ny
    dims = (nx, ny)
    kappa = lognormal_kappa(dims, sigma, seed)
    return _diffusion(dims, kappa, False, "diff2d5", {"sigma": sigma, "seed": seed})


def rhs_uniform(n: int, nrhs: int, seed: int = 0) -> np.ndarray:
    """n x nrhs column-major block, entries uniform in [-1, 1) from default_rng(seed)."""
    return np.asfortranarray(np.random.default_rng(seed).uniform(-1.0, 1.0, size=(nrhs, n)).T)


def batch_sides(count: int = 512, seed: int = 1234, lo: int = 16, hi: int = 128) -> np.ndarray:
    """Grid sides of the many-small-matrices batch, uniform integers in [lo, hi]."""
    return np.random.default_rng(seed).integers(lo, hi + 1, count)


def workload(name: str):
    """The named synthetic workloads: (matrix, perm, rhs) with the fixed seeds.

    ``lap2d_64``   2D 5-point 64x64 + 1e-2 I, one RHS, seed 0.
    ``lap3d_64``   3D 7-point 64^3, eight RHS, seed 0.
    ``diff3d_48``  3D 27-point diffusion 48^3, sigma 2, one RHS, seed 0.
    Smaller grids use the same recipes: ``lap2d_<s>``, ``lap3d_<s>``,
    ``diff3d_<s>``, ``diff2d_<s>``.
    """
    from .nd import geometric_nd

    kind, side = name.rsplit("_", 1)
    s = int(side)
    if kind == "lap2d":
        A = laplacian_2d(s, shift=1e-2 if s == 64 else 0.0)
        nrhs = 1
    elif kind == "lap3d":
        A = laplacian_3d(s)
        nrhs = 8
    elif kind == "diff3d":
        A = diffusion_3d_27pt(s, sigma=2.0, seed=1)
        nrhs = 1
    elif kind == "diff2d":
        A = diffusion_2d_5pt(s, sigma=1.0, seed=1)
        nrhs = 1
    else:
        raise ValueError(name)
    perm = geometric_nd(A.dims)
    b = rhs_uniform(A.n, nrhs, seed=0)
    return A, perm, b
