"""Helpers for the GPU parity tests: run the library through its C-ABI and the
oracle on the same seeded inputs."""
import numpy as np
import scipy.sparse as sp

import oracle
from paper_1608_00044_gb300 import spchol

# Backward-error bar of the FP64 path: ||b - A x|| / (||A|| ||x|| + ||b||) <= 1e-13.
BERR_FP64 = 1e-13


def gpu_factor_solve(A, perm, B, use_device=True, **opts):
    """Factor and solve with the GPU library.  Returns (rc, X, stats, handle)."""
    import torch

    o = spchol.default_options(**opts)
    h = spchol.analyze(A.n, A.colptr, A.rowind, perm, o)
    if use_device:
        vals = torch.from_numpy(np.ascontiguousarray(A.values)).cuda()
        rc = spchol.factorize(h, vals)
    else:
        rc = spchol.factorize(h, np.ascontiguousarray(A.values))
    X = None
    if rc == 0 and B is not None:
        Bf = np.asfortranarray(B, dtype=np.float64)
        if Bf.ndim == 1:
            Bf = Bf.reshape(-1, 1, order="F")
        nrhs = Bf.shape[1]
        if use_device:
            Bt = torch.from_numpy(np.ascontiguousarray(Bf.T)).cuda()  # (nrhs, n) row-major == n x nrhs col-major
            spchol.solve(h, Bt, A.n, nrhs)
            X = np.asfortranarray(Bt.cpu().numpy().T)
        else:
            X = Bf.copy(order="F")
            spchol.solve(h, X, A.n, nrhs)
    return rc, X, spchol.stats(h), h


def l_max_diff(h, A):
    """max |L_gpu - L_oracle| on the same permutation, and max |L_oracle|."""
    Lp, Li, Lx, perm = spchol.export_factor(h)
    n = A.n
    Lg = sp.csc_matrix((Lx, Li, Lp), shape=(n, n))
    f = oracle.OracleFactor.from_csc(A, perm)
    assert f.factor() == 0
    op, oi, ox = f.L()
    Lo = sp.csc_matrix((ox, oi, op), shape=(n, n))
    d = abs(Lg - Lo)
    return (d.max() if d.nnz else 0.0), abs(Lo).max()
