"""CPU oracle for the supernodal Cholesky library (test infrastructure only).

Only the tests, the smoke check and the benchmark's CPU-baseline / reference leg
may import this package.  The library under ``paper_1608_00044_gb300`` never
does; the two share no code.  See ``spchol_oracle.c`` for what each routine
computes and which passage of the paper it follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spchol_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)
_f64p = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, so x86 and Arm agree)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.orc_analyze.restype = ctypes.c_void_p
            lib.orc_analyze.argtypes = [ctypes.c_int64, _i64p, _i32p, _f64p, _i64p]
            lib.orc_free.argtypes = [ctypes.c_void_p]
            lib.orc_nnzL.restype = ctypes.c_int64
            lib.orc_nnzL.argtypes = [ctypes.c_void_p]
            lib.orc_flops.restype = ctypes.c_double
            lib.orc_flops.argtypes = [ctypes.c_void_p]
            lib.orc_get_structure.argtypes = [ctypes.c_void_p, _i64p, _i64p]
            lib.orc_get_L.argtypes = [ctypes.c_void_p, _i64p, _i64p, _f64p]
            lib.orc_get_B.argtypes = [ctypes.c_void_p, _i64p, _i64p, _f64p]
            lib.orc_supernodes.restype = ctypes.c_int64
            lib.orc_supernodes.argtypes = [ctypes.c_void_p, _i64p]
            lib.orc_factor.restype = ctypes.c_int64
            lib.orc_factor.argtypes = [ctypes.c_void_p]
            lib.orc_solve.restype = ctypes.c_int
            lib.orc_solve.argtypes = [ctypes.c_void_p, _f64p, ctypes.c_int64, ctypes.c_int]
            lib.orc_berr.restype = ctypes.c_double
            lib.orc_berr.argtypes = [ctypes.c_int64, _i64p, _i32p, _f64p, _f64p, ctypes.c_int64,
                                     _f64p, ctypes.c_int64, ctypes.c_int]
            lib.orc_fact_err.restype = ctypes.c_double
            lib.orc_fact_err.argtypes = [ctypes.c_void_p]
            lib.orc_fact_err_csc.restype = ctypes.c_double
            lib.orc_fact_err_csc.argtypes = [ctypes.c_int64, _i64p, _i64p, _f64p, _i64p, _i64p, _f64p]
            _lib = lib
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


class OracleFactor:
    """Symbolic analysis (on construction) and numeric factor of P A P^T."""

    def __init__(self, n, colptr, rowind, values, perm=None):
        self._lib = _load()
        self.n = int(n)
        self.colptr = np.ascontiguousarray(colptr, dtype=np.int64)
        self.rowind = np.ascontiguousarray(rowind, dtype=np.int32)
        self.values = np.ascontiguousarray(values, dtype=np.float64)
        self.perm = None if perm is None else np.ascontiguousarray(perm, dtype=np.int64)
        h = self._lib.orc_analyze(self.n, _p(self.colptr, _i64p), _p(self.rowind, _i32p),
                                  _p(self.values, _f64p),
                                  None if self.perm is None else _p(self.perm, _i64p))
        if not h:
            raise ValueError("oracle: invalid matrix or permutation")
        self._h = ctypes.c_void_p(h)
        self.info = None

    @classmethod
    def from_csc(cls, A, perm=None):
        return cls(A.n, A.colptr, A.rowind, A.values, perm)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.orc_free(h)
            self._h = None

    # --- symbolic -------------------------------------------------------------
    @property
    def nnzL(self) -> int:
        return int(self._lib.orc_nnzL(self._h))

    @property
    def flops(self) -> float:
        """Sum of c_j^2 over columns, c_j the column count including the diagonal."""
        return float(self._lib.orc_flops(self._h))

    def structure(self):
        parent = np.empty(self.n, np.int64)
        cc = np.empty(self.n, np.int64)
        self._lib.orc_get_structure(self._h, _p(parent, _i64p), _p(cc, _i64p))
        return parent, cc

    def supernodes(self) -> np.ndarray:
        start = np.empty(self.n + 1, np.int64)
        ns = int(self._lib.orc_supernodes(self._h, _p(start, _i64p)))
        return start[: ns + 1].copy()

    def B(self):
        Bp = np.empty(self.n + 1, np.int64)
        self._lib.orc_get_B(self._h, _p(Bp, _i64p), None, None)
        nz = int(Bp[-1])
        Bi = np.empty(nz, np.int64)
        Bx = np.empty(nz, np.float64)
        self._lib.orc_get_B(self._h, None, _p(Bi, _i64p), _p(Bx, _f64p))
        return Bp, Bi, Bx

    def L(self):
        nz = self.nnzL
        Lp = np.empty(self.n + 1, np.int64)
        Li = np.empty(nz, np.int64)
        Lx = np.empty(nz, np.float64)
        self._lib.orc_get_L(self._h, _p(Lp, _i64p), _p(Li, _i64p), _p(Lx, _f64p))
        return Lp, Li, Lx

    # --- numeric --------------------------------------------------------------
    def factor(self) -> int:
        self.info = int(self._lib.orc_factor(self._h))
        return self.info

    def solve(self, B) -> np.ndarray:
        X = np.array(B, dtype=np.float64, order="F", copy=True)
        if X.ndim == 1:
            X = X.reshape(-1, 1, order="F")
        rc = self._lib.orc_solve(self._h, _p(X, _f64p), X.shape[0], X.shape[1])
        if rc != 0:
            raise RuntimeError("oracle: solve before a successful factor")
        return X

    def fact_err(self) -> float:
        return float(self._lib.orc_fact_err(self._h))


def berr(A, X, B) -> float:
    """Componentwise-free normwise backward error, max over right-hand sides."""
    lib = _load()
    X = np.asfortranarray(X, dtype=np.float64)
    B = np.asfortranarray(B, dtype=np.float64)
    if X.ndim == 1:
        X = X.reshape(-1, 1, order="F")
    if B.ndim == 1:
        B = B.reshape(-1, 1, order="F")
    colptr = np.ascontiguousarray(A.colptr, np.int64)
    rowind = np.ascontiguousarray(A.rowind, np.int32)
    values = np.ascontiguousarray(A.values, np.float64)
    return float(lib.orc_berr(A.n, _p(colptr, _i64p), _p(rowind, _i32p), _p(values, _f64p),
                              _p(X, _f64p), X.shape[0], _p(B, _f64p), B.shape[0], X.shape[1]))


def fact_err_csc(n, Lp, Li, Lx, Bp, Bi, Bx) -> float:
    """||L L^T - B||_F / ||B||_F for a lower CSC factor L and the lower CSC of a symmetric B.

    Rows ascending inside each column.  +inf when a product entry or an entry of
    B lies outside L's pattern.
    """
    lib = _load()
    arr = [np.ascontiguousarray(a, np.int64) for a in (Lp, Li)]
    lx = np.ascontiguousarray(Lx, np.float64)
    brr = [np.ascontiguousarray(a, np.int64) for a in (Bp, Bi)]
    bx = np.ascontiguousarray(Bx, np.float64)
    return float(lib.orc_fact_err_csc(int(n), _p(arr[0], _i64p), _p(arr[1], _i64p), _p(lx, _f64p),
                                      _p(brr[0], _i64p), _p(brr[1], _i64p), _p(bx, _f64p)))
