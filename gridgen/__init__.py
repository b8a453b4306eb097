"""Seeded synthetic inputs for the supernodal Cholesky library and its tests.

This package builds the symmetric positive definite grid matrices that stand in
for the paper's UF/SuiteSparse test matrices (Section V, Table I), the geometric
nested-dissection ordering that stands in for Scotch (Section V), and the seeded
right-hand sides.  It holds none of the factorization's arithmetic: no
elimination tree, no symbolic or numeric Cholesky step.  Both the CPU oracle's
tests and the GPU path read their inputs from here.
"""
from .grids import (
    CscLower,
    laplacian_2d,
    laplacian_3d,
    diffusion_2d_5pt,
    diffusion_3d_27pt,
    neumann_laplacian_3d,
    lognormal_kappa,
    rhs_uniform,
    batch_sides,
    workload,
)
from .nd import geometric_nd

__all__ = [
    "CscLower",
    "laplacian_2d",
    "laplacian_3d",
    "diffusion_2d_5pt",
    "diffusion_3d_27pt",
    "neumann_laplacian_3d",
    "lognormal_kappa",
    "rhs_uniform",
    "batch_sides",
    "workload",
    "geometric_nd",
]
