"""ctypes binding of libspchol_host (include/spchol_host.h): the host-only
symbolic plan and the task-protocol simulator.  No GPU needed."""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .spchol import Options, default_options_host

_HERE = os.path.dirname(os.path.abspath(__file__))
HOST_LIB_PATH = os.path.join(_HERE, "libspchol_host.so")

(PERM, COLCOUNT, ETREE, FCOL, NROWS, ROWOFF, ROWS, PARENT, DEPF, NTRSM, NU, UTASKS, NST, SCALARS, ADEST, NUHI, SUBLO,
 SUBHI, FANOFF, FANTASK, FANPTR, FANENT) = range(22)

_vp = ctypes.c_void_p
SIGNATURES = [
    ("spchol_plan_build", ctypes.c_int, [ctypes.c_int64, _vp, _vp, _vp, ctypes.POINTER(Options), ctypes.POINTER(_vp)]),
    ("spchol_plan_len", ctypes.c_int64, [_vp, ctypes.c_int]),
    ("spchol_plan_get", ctypes.c_int, [_vp, ctypes.c_int, _vp]),
    ("spchol_plan_flops", ctypes.c_double, [_vp]),
    ("spchol_plan_simulate", ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int64, ctypes.c_int, ctypes.c_uint64, _vp]),
    ("spchol_plan_pool_len", ctypes.c_int64, [_vp]),
    ("spchol_plan_destroy", None, [_vp]),
    ("spchol_order_nd", ctypes.c_int, [ctypes.c_int64, _vp, _vp, _vp]),
]
_lib = None


def load():
    global _lib
    if _lib is None:
        if not os.path.exists(HOST_LIB_PATH):
            raise RuntimeError("libspchol_host.so not built: run paper_1608_00044_gb300.build.build_host()")
        lib = ctypes.CDLL(HOST_LIB_PATH)
        for name, res, args in SIGNATURES:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def order_nd(n, colptr, rowind) -> np.ndarray:
    """spchol_order_nd from the host library (the same code as libspchol.so's)."""
    lib = load()
    colptr = np.ascontiguousarray(colptr, np.int64)
    rowind = np.ascontiguousarray(rowind, np.int32)
    perm = np.empty(max(int(n), 0), np.int64)
    rc = lib.spchol_order_nd(int(n), colptr.ctypes.data, rowind.ctypes.data, perm.ctypes.data if n > 0 else None)
    if rc != 0:
        raise ValueError(f"spchol_order_nd failed with code {rc}")
    return perm


class HostPlan:
    """Symbolic plan of P A P^T built on the host (same code as the GPU library's analyze)."""

    def __init__(self, n, colptr, rowind, perm=None, **options):
        lib = load()
        self._colptr = np.ascontiguousarray(colptr, np.int64)
        self._rowind = np.ascontiguousarray(rowind, np.int32)
        self._perm = None if perm is None else np.ascontiguousarray(perm, np.int64)
        self.opt = default_options_host(**options)
        h = ctypes.c_void_p()
        rc = lib.spchol_plan_build(int(n), self._colptr.ctypes.data, self._rowind.ctypes.data,
                                   None if self._perm is None else self._perm.ctypes.data,
                                   ctypes.byref(self.opt), ctypes.byref(h))
        if rc != 0:
            raise ValueError(f"spchol_plan_build failed with code {rc}")
        self._h = h
        self.n = int(n)

    def get(self, what: int) -> np.ndarray:
        lib = load()
        ln = lib.spchol_plan_len(self._h, what)
        out = np.empty(max(ln, 0), np.int64)
        if ln > 0:
            rc = lib.spchol_plan_get(self._h, what, out.ctypes.data)
            if rc != 0:
                raise ValueError(rc)
        return out

    @property
    def flops(self) -> float:
        return float(load().spchol_plan_flops(self._h))

    def scalars(self) -> dict:
        v = self.get(SCALARS)
        keys = ["n", "nnz_l", "ns", "factor_tasks", "solve_tasks", "max_w", "max_r", "nnz_l_stored", "n_trsm", "n_u",
                "n_hi_tasks", "n_sub"]
        return dict(zip(keys, (int(x) for x in v)))

    def simulate(self, values, B=None, seed=0, want_pool=False):
        """Run the task graph on the host in a seeded random ready order.  Returns (rc, X, pool)."""
        lib = load()
        vals = np.ascontiguousarray(values, np.float64)
        X = None
        nrhs, ldb, bp = 0, max(self.n, 1), None
        if B is not None:
            X = np.array(B, dtype=np.float64, order="F", copy=True)
            if X.ndim == 1:
                X = X.reshape(-1, 1, order="F")
            nrhs, ldb, bp = X.shape[1], X.shape[0], X.ctypes.data
        pool = np.empty(lib.spchol_plan_pool_len(self._h), np.float64) if want_pool else None
        rc = lib.spchol_plan_simulate(self._h, vals.ctypes.data, bp, ldb, nrhs, int(seed),
                                      None if pool is None else pool.ctypes.data)
        return rc, X, pool

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().spchol_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
