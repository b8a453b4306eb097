"""Geometric nested dissection of a box grid (stand-in for Scotch, Section V).

Recursive bisection: split the axis with the largest extent (the lowest axis
index on a tie) at the plane ``lo + size // 2``; number the left box, then the
right box, then the separator plane.  A box whose volume is at most 8 or whose
longest side is at most 2 is a leaf.  Points of a leaf or of a separator are
numbered in C order (axis 0 slowest).  On a 64^3 grid the top separator is the
64 x 64 plane x = 32.

The separator planes are full cuts for the 5-, 7- and 27-point stencils (no
stencil couples points two planes apart), so every subtree of the resulting
ordering is independent of its sibling.
"""
from __future__ import annotations

import numpy as np


def geometric_nd(dims, leaf_volume: int = 8, leaf_side: int = 2) -> np.ndarray:
    """Permutation ``perm`` (new -> old) of the grid points, int64."""
    dims = tuple(int(d) for d in dims)
    ids = np.arange(int(np.prod(dims)), dtype=np.int64).reshape(dims)
    out: list[np.ndarray] = []

    def emit(lo, hi):
        sl = tuple(slice(a, b) for a, b in zip(lo, hi))
        out.append(ids[sl].ravel())

    # Explicit stack of (lo, hi, stage): stage 0 = first visit, 1 = emit separator.
    stack = [(tuple(0 for _ in dims), dims, None)]
    while stack:
        lo, hi, sep = stack.pop()
        if sep is not None:
            emit(*sep)
            continue
        ext = [b - a for a, b in zip(lo, hi)]
        if int(np.prod(ext)) <= leaf_volume or max(ext) <= leaf_side:
            emit(lo, hi)
            continue
        ax = int(np.argmax(ext))
        cut = lo[ax] + ext[ax] // 2
        left_hi = list(hi)
        left_hi[ax] = cut
        right_lo = list(lo)
        right_lo[ax] = cut + 1
        sep_lo = list(lo)
        sep_lo[ax] = cut
        sep_hi = list(hi)
        sep_hi[ax] = cut + 1
        # LIFO: push in reverse of the numbering order (left, right, separator).
        stack.append((lo, hi, (tuple(sep_lo), tuple(sep_hi))))
        stack.append((tuple(right_lo), hi, None))
        stack.append((lo, tuple(left_hi), None))
    perm = np.concatenate(out)
    assert perm.size == ids.size
    return perm
