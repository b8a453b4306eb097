"""Decoder for the Fig. 1 fixture (the paper's worked example, Section II-B)."""
import math
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "fig1_structure.txt")


def _span(centre, size):
    # trunc toward zero of the drawing command's start and stop coordinates
    return range(math.trunc(centre - size / 2), math.trunc(centre + size / 2 - 1) + 1)


def load():
    """Return (n, A_pattern, fill, supernode column ranges, sn parent map)."""
    a_pat, fill, blocks, edges = set(), set(), {}, {}
    with open(GOLDEN) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if not line:
                continue
            kind, args = line[0], [float(x) for x in line[1:]]
            if kind == "dblk":
                label, size, c = int(args[0]), args[1], args[2]
                cols = list(_span(c, size))
                blocks[label] = (cols[0], cols[-1] + 1)
                for j in cols:
                    for i in cols:
                        if i >= j:
                            a_pat.add((i, j))
            elif kind in ("lublk", "flublk"):
                w, h, x, y = args
                target = a_pat if kind == "lublk" else fill
                for j in _span(x, w):
                    for i in _span(y, h):
                        target.add((i, j))
            elif kind == "edge":
                edges[int(args[0])] = int(args[1])
    n = max(i for i, _ in a_pat) + 1
    return n, a_pat, fill, blocks, edges


def spd_from_pattern(n, pattern):
    """Lower CSC with off-diagonal -1 and diagonal 2 + (row degree): SPD."""
    deg = np.zeros(n)
    for i, j in pattern:
        if i != j:
            deg[i] += 1
            deg[j] += 1
    entries = sorted((j, i) for i, j in pattern)
    colptr = np.zeros(n + 1, np.int64)
    rowind, vals = [], []
    for j, i in entries:
        colptr[j + 1] += 1
        rowind.append(i)
        vals.append(2.0 + deg[i] if i == j else -1.0)
    colptr = np.cumsum(colptr)
    return colptr, np.array(rowind, np.int32), np.array(vals, np.float64)
