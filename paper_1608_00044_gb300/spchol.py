"""Thin ctypes binding of libspchol (include/spchol.h): argument marshalling only.

Every step of analyze / factorize / solve runs in the native library; this
module converts numpy arrays and torch tensors into pointers, passes the
current CUDA stream, and raises on non-zero return codes.  It fails loudly when
the compiled library is missing: there is no Python fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libspchol.so")

FP64, FP32, TF32, TF32X3, FP64_TC = 0, 1, 2, 3, 4
OK = 0
ENOMEM, ETIMEOUT, ESTATE, ENOCONV, ECUDA, EINTERNAL, ESCRATCH = -1001, -1002, -1003, -1004, -1005, -1006, -1007


class Options(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int),
        ("max_width", ctypes.c_int),
        ("relax_zeros", ctypes.c_int),
        ("tile_rows", ctypes.c_int),
        ("ctas_per_sm", ctypes.c_int),
        ("deterministic", ctypes.c_int),
        ("wait_budget_ns", ctypes.c_int64),
        ("ir_max_iter", ctypes.c_int),
        ("ir_tol", ctypes.c_double),
        ("fault_inject", ctypes.c_int),
        ("profile", ctypes.c_int),
        ("solve_tile_rows", ctypes.c_int),
        ("sched", ctypes.c_int),
        ("dev_alloc", ctypes.c_void_p),  # function pointers (DEV_ALLOC_FN / DEV_FREE_FN), NULL = the pool
        ("dev_free", ctypes.c_void_p),
        ("alloc_ctx", ctypes.c_void_p),
        ("solve_w_depth", ctypes.c_int),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64),
        ("nnz_a", ctypes.c_int64),
        ("nnz_l", ctypes.c_int64),
        ("nnz_l_stored", ctypes.c_int64),
        ("flops", ctypes.c_double),
        ("n_supernodes", ctypes.c_int64),
        ("n_tasks", ctypes.c_int64),
        ("max_width", ctypes.c_int64),
        ("max_rows", ctypes.c_int64),
        ("footprint_bytes", ctypes.c_int64),
        ("analyze_ms", ctypes.c_double),
        ("factor_ms", ctypes.c_double),
        ("solve_ms", ctypes.c_double),
        ("ir_iters", ctypes.c_int),
        ("berr", ctypes.c_double),
        ("precision", ctypes.c_int),
        ("factor_task_ms", ctypes.c_double * 3),
        ("factor_task_count", ctypes.c_int64 * 3),
        ("factor_wait_ms", ctypes.c_double),
        ("solve_task_ms", ctypes.c_double * 4),
        ("solve_wait_ms", ctypes.c_double),
        ("factor_tc_update_ms", ctypes.c_double),
        ("grid_factor", ctypes.c_int),
        ("grid_solve", ctypes.c_int),
        ("tma_staging", ctypes.c_int),
        ("n_subtrees", ctypes.c_int),
        ("factor_subtree_ms", ctypes.c_double),
        ("factor_subtree_count", ctypes.c_int64),
        ("ir_gmres_iters", ctypes.c_int),
        ("factor_gather_ms", ctypes.c_double * 3),
        ("factor_gather_batches", ctypes.c_int64),
        ("factor_gather_tiles", ctypes.c_int64),
        ("n_warp_subtrees", ctypes.c_int64),
    ]

    def as_dict(self):
        out = {}
        for k, _ in self._fields_:
            v = getattr(self, k)
            out[k] = list(v) if hasattr(v, "__len__") else v
        return out


class SpcholError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = int(code)
        detail = ""
        if code in (ECUDA, ENOMEM):
            detail = " [" + load().spchol_last_cuda_error().decode() + "]"
        super().__init__(f"{where}: {strerror(code)} (code {code}){detail}")


_lib = None

# (name, restype, argtypes) of every exported symbol declared in include/spchol.h
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
SIGNATURES = [
    ("spchol_default_options", None, [ctypes.POINTER(Options)]),
    ("spchol_analyze", ctypes.c_int, [_i64, _vp, _vp, _vp, ctypes.POINTER(Options), ctypes.POINTER(_vp)]),
    ("spchol_order_nd", ctypes.c_int, [_i64, _vp, _vp, _vp]),
    ("spchol_factorize", ctypes.c_int, [_vp, _vp, _vp]),
    ("spchol_factorize_enqueue", ctypes.c_int, [_vp, _vp, _vp]),
    ("spchol_factorize_status", ctypes.c_int, [_vp]),
    ("spchol_solve", ctypes.c_int, [_vp, _vp, _i64, ctypes.c_int, _vp]),
    ("spchol_solve_noalloc", ctypes.c_int, [_vp, _vp, _i64, ctypes.c_int, _vp]),
    ("spchol_stats_get", ctypes.c_int, [_vp, ctypes.POINTER(Stats)]),
    ("spchol_export_factor", ctypes.c_int, [_vp, ctypes.POINTER(_i64), _vp, _vp, _vp, _vp]),
    ("spchol_trace_get", ctypes.c_int, [_vp, ctypes.c_int, _vp, ctypes.POINTER(_i64)]),
    ("spchol_destroy", ctypes.c_int, [_vp]),
    ("spchol_strerror", ctypes.c_char_p, [ctypes.c_int]),
    ("spchol_last_cuda_error", ctypes.c_char_p, []),
    ("spchol_batch_analyze", ctypes.c_int, [ctypes.c_int, _vp, _vp, _vp, _vp, ctypes.POINTER(Options),
                                            ctypes.POINTER(_vp)]),
    ("spchol_batch_factorize", ctypes.c_int, [_vp, _vp, _vp]),
    ("spchol_batch_solve", ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    ("spchol_batch_info", ctypes.c_int, [_vp, _i64, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(_i64)]),
]


def load(path: str | None = None):
    """Load libspchol.so (built by ``paper_1608_00044_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libspchol.so not found at {p}: run paper_1608_00044_gb300.build.build() first")
    lib = ctypes.CDLL(p)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def strerror(code: int) -> str:
    return load().spchol_strerror(int(code)).decode()


def default_options(allocator=None, **kw) -> Options:
    """spchol_default_options, then the given fields.  allocator="torch" routes the
    handle's device memory through PyTorch's caching allocator (TorchAllocator)."""
    o = Options()
    load().spchol_default_options(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    if allocator == "torch":
        torch_allocator().install(o)
    elif allocator is not None:
        allocator.install(o)
    return o


def default_options_host(**kw) -> Options:
    """The defaults of include/spchol.h filled without loading the GPU library."""
    o = Options(precision=FP64, max_width=64, relax_zeros=4, tile_rows=0, ctas_per_sm=0, deterministic=0,
                wait_budget_ns=2_000_000_000, ir_max_iter=10, ir_tol=1e-12, fault_inject=0, profile=0, solve_tile_rows=0, sched=0,
                dev_alloc=None, dev_free=None, alloc_ctx=None, solve_w_depth=0)
    for k, v in kw.items():
        setattr(o, k, v)
    return o


# ------------------------------------------------------------------ device memory hook

DEV_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
DEV_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class TorchAllocator:
    """spchol_options.dev_alloc / dev_free served by PyTorch's caching allocator.

    The library asks for its device memory here instead of allocating it itself,
    so a handle's memory comes from (and returns to) the same cache as the
    caller's tensors: destroying a handle or growing a solve workspace never
    calls cudaFree, which would wait for every stream on the device.  A block
    is requested on the stream of the call that first uses it (the current
    stream when the library passes none).  The library releases a block only
    after its own work on it has completed, so returning it to the cache at once
    is safe.  One instance per process (``torch_allocator()``): the callbacks
    must outlive every handle that uses them.
    """

    def __init__(self):
        import torch

        self._torch = torch
        self._lock = threading.Lock()
        self.live = {}  # address -> bytes of the blocks the library holds
        self.failures = 0
        self._alloc_cb = DEV_ALLOC_FN(self._alloc)
        self._free_cb = DEV_FREE_FN(self._free)

    def _alloc(self, nbytes, stream, ctx):
        torch = self._torch
        try:
            dev = torch.cuda.current_device()  # the library makes the handle's device current
            st = int(stream) if stream else torch.cuda.current_stream(dev).cuda_stream
            p = int(torch.cuda.caching_allocator_alloc(int(nbytes), dev, st))
        except Exception:  # out of memory, or torch refused: the library returns SPCHOL_ENOMEM
            with self._lock:
                self.failures += 1
            return None
        with self._lock:
            self.live[p] = int(nbytes)
        return p

    def _free(self, ptr, nbytes, stream, ctx):
        with self._lock:
            self.live.pop(int(ptr), None)
        try:
            self._torch.cuda.caching_allocator_delete(int(ptr))
        except Exception:
            pass

    def held_bytes(self) -> int:
        with self._lock:
            return sum(self.live.values())

    def install(self, opt: Options) -> Options:
        opt.dev_alloc = ctypes.cast(self._alloc_cb, ctypes.c_void_p).value
        opt.dev_free = ctypes.cast(self._free_cb, ctypes.c_void_p).value
        opt.alloc_ctx = None
        return opt


_torch_alloc = None
_torch_alloc_lock = threading.Lock()


def torch_allocator() -> TorchAllocator:
    """The process-wide TorchAllocator (created on first use)."""
    global _torch_alloc
    with _torch_alloc_lock:
        if _torch_alloc is None:
            _torch_alloc = TorchAllocator()
        return _torch_alloc


# ------------------------------------------------------------------ marshalling


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x):
    """Address of a host numpy array or a torch tensor (host or device)."""
    if x is None:
        return None
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    if isinstance(x, int):
        return x
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream(stream):
    if stream is None:
        try:
            import torch

            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:  # pragma: no cover - torch missing
            pass
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def _host(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a


# ------------------------------------------------------------------ C-ABI mirrors


def analyze(n, colptr, rowind, perm=None, opt: Options | None = None):
    """spchol_analyze on host arrays.  Returns the handle (c_void_p)."""
    lib = load()
    colptr = _host(colptr, np.int64)
    rowind = _host(rowind, np.int32)
    perm = None if perm is None else _host(perm, np.int64)
    h = ctypes.c_void_p()
    rc = lib.spchol_analyze(int(n), colptr.ctypes.data, rowind.ctypes.data,
                            None if perm is None else perm.ctypes.data,
                            ctypes.byref(opt) if opt is not None else None, ctypes.byref(h))
    if rc != 0:
        raise SpcholError(rc, "spchol_analyze")
    return h


def order_nd(n, colptr, rowind) -> np.ndarray:
    """spchol_order_nd: a nested-dissection ordering (new -> old, int64) of a
    lower-triangle CSC pattern, for matrices that come without one."""
    lib = load()
    colptr = _host(colptr, np.int64)
    rowind = _host(rowind, np.int32)
    perm = np.empty(max(int(n), 0), np.int64)
    rc = lib.spchol_order_nd(int(n), colptr.ctypes.data, rowind.ctypes.data, perm.ctypes.data if n > 0 else None)
    if rc != 0:
        raise SpcholError(rc, "spchol_order_nd")
    return perm


def factorize(h, values, stream=None) -> int:
    """spchol_factorize; returns 0 or the positive non-SPD column; raises on errors."""
    if isinstance(values, np.ndarray):
        values = _host(values, np.float64)
    rc = load().spchol_factorize(h, _ptr(values), _stream(stream))
    if rc < 0:
        raise SpcholError(rc, "spchol_factorize")
    return rc


def factorize_enqueue(h, values, stream=None) -> None:
    """spchol_factorize_enqueue: queue the factorization (device values) without waiting."""
    rc = load().spchol_factorize_enqueue(h, _ptr(values), _stream(stream))
    if rc != 0:
        raise SpcholError(rc, "spchol_factorize_enqueue")


def factorize_status(h) -> int:
    """spchol_factorize_status: result of the last enqueued factorization, once its stream is done."""
    rc = load().spchol_factorize_status(h)
    if rc < 0:
        raise SpcholError(rc, "spchol_factorize_status")
    return rc


def solve(h, B, ldb=None, nrhs=None, stream=None) -> int:
    """spchol_solve in place on B (n x nrhs column-major: numpy F-order or a torch tensor whose
    transpose is contiguous, i.e. shape (nrhs, n) row-major)."""
    if nrhs is None or ldb is None:
        raise ValueError("give ldb and nrhs explicitly")
    rc = load().spchol_solve(h, _ptr(B), int(ldb), int(nrhs), _stream(stream))
    if rc != 0:
        raise SpcholError(rc, "spchol_solve")
    return rc


def solve_noalloc(h, B, ldb=None, nrhs=None, stream=None) -> int:
    """spchol_solve_noalloc: the solve without any device allocation, B in device memory."""
    if nrhs is None or ldb is None:
        raise ValueError("give ldb and nrhs explicitly")
    rc = load().spchol_solve_noalloc(h, _ptr(B), int(ldb), int(nrhs), _stream(stream))
    if rc != 0:
        raise SpcholError(rc, "spchol_solve_noalloc")
    return rc


def stats(h) -> dict:
    st = Stats()
    rc = load().spchol_stats_get(h, ctypes.byref(st))
    if rc != 0:
        raise SpcholError(rc, "spchol_stats_get")
    return st.as_dict()


def export_factor(h):
    """(Lp, Li, Lx, perm) of the resident factor, permuted ordering."""
    lib = load()
    nnz = ctypes.c_int64(0)
    st = stats(h)
    perm = np.empty(st["n"], np.int64)
    rc = lib.spchol_export_factor(h, ctypes.byref(nnz), None, None, None, perm.ctypes.data)
    if rc != 0:
        raise SpcholError(rc, "spchol_export_factor")
    Lp = np.empty(st["n"] + 1, np.int64)
    Li = np.empty(nnz.value, np.int64)
    Lx = np.empty(nnz.value, np.float64)
    rc = lib.spchol_export_factor(h, ctypes.byref(nnz), Lp.ctypes.data, Li.ctypes.data, Lx.ctypes.data, None)
    if rc != 0:
        raise SpcholError(rc, "spchol_export_factor")
    return Lp, Li[: nnz.value], Lx[: nnz.value], perm


def trace_get(h, which: int) -> np.ndarray:
    """(ntask, 2) start/end device-clock ns of each task of the last factorization (0) or solve (1)."""
    lib = load()
    cnt = ctypes.c_int64(0)
    rc = lib.spchol_trace_get(h, which, None, ctypes.byref(cnt))
    if rc != 0:
        raise SpcholError(rc, "spchol_trace_get")
    out = np.empty((cnt.value, 2), np.uint64)
    rc = lib.spchol_trace_get(h, which, out.ctypes.data, ctypes.byref(cnt))
    if rc != 0:
        raise SpcholError(rc, "spchol_trace_get")
    return out


def final_perm(h) -> np.ndarray:
    """The permutation (new -> old) the handle factors with: the given one refined by a postorder."""
    st = stats(h)
    perm = np.empty(st["n"], np.int64)
    nnz = ctypes.c_int64(0)
    rc = load().spchol_export_factor(h, ctypes.byref(nnz), None, None, None, perm.ctypes.data)
    if rc != 0:
        raise SpcholError(rc, "spchol_export_factor")
    return perm


def destroy(h):
    if h is not None and getattr(h, "value", None):
        load().spchol_destroy(h)
        h.value = None


def _ptr_array(items, ctype=ctypes.c_void_p):
    arr = (ctype * len(items))()
    for i, x in enumerate(items):
        arr[i] = _ptr(x) if ctype is ctypes.c_void_p else x
    return arr


def batch_analyze(ns, colptrs, rowinds, perms=None, opt: Options | None = None):
    lib = load()
    count = len(ns)
    colptrs = [_host(c, np.int64) for c in colptrs]
    rowinds = [_host(r, np.int32) for r in rowinds]
    perms_h = None if perms is None else [None if p is None else _host(p, np.int64) for p in perms]
    n_arr = (ctypes.c_int64 * count)(*[int(x) for x in ns])
    cp = _ptr_array(colptrs)
    ri = _ptr_array(rowinds)
    pm = None if perms_h is None else _ptr_array(perms_h)
    h = ctypes.c_void_p()
    rc = lib.spchol_batch_analyze(count, ctypes.addressof(n_arr), ctypes.addressof(cp), ctypes.addressof(ri),
                                  None if pm is None else ctypes.addressof(pm),
                                  ctypes.byref(opt) if opt is not None else None, ctypes.byref(h))
    if rc != 0:
        raise SpcholError(rc, "spchol_batch_analyze")
    h._keep = (colptrs, rowinds, perms_h)
    return h


def batch_factorize(h, values, stream=None) -> int:
    vals = [(_host(v, np.float64) if isinstance(v, np.ndarray) else v) for v in values]
    arr = _ptr_array(vals)
    rc = load().spchol_batch_factorize(h, ctypes.addressof(arr), _stream(stream))
    if rc < 0:
        raise SpcholError(rc, "spchol_batch_factorize")
    return rc


def batch_solve(h, Bs, ldbs, nrhss, stream=None) -> int:
    count = len(Bs)
    arr = _ptr_array(list(Bs))
    ld = (ctypes.c_int64 * count)(*[int(x) for x in ldbs])
    nr = (ctypes.c_int * count)(*[int(x) for x in nrhss])
    rc = load().spchol_batch_solve(h, ctypes.addressof(arr), ctypes.addressof(ld), ctypes.addressof(nr),
                                   _stream(stream))
    if rc != 0:
        raise SpcholError(rc, "spchol_batch_solve")
    return rc


def batch_info(h, k: int):
    m = ctypes.c_int(0)
    c = ctypes.c_int64(0)
    rc = load().spchol_batch_info(h, int(k), ctypes.byref(m), ctypes.byref(c))
    if rc != 0:
        raise SpcholError(rc, "spchol_batch_info")
    return m.value, c.value


# ------------------------------------------------------------------ convenience


class SparseCholesky:
    """analyze -> factorize -> solve for one matrix given as a lower CSC."""

    def __init__(self, n, colptr, rowind, perm=None, **options):
        self.opt = default_options(**options)
        self.h = analyze(n, colptr, rowind, perm, self.opt)
        self.n = int(n)

    def factorize(self, values, stream=None) -> int:
        return factorize(self.h, values, stream)

    def solve(self, B, stream=None):
        """Solve in place.  numpy: B is (n,) or (n, nrhs) Fortran order.  torch: B is a
        contiguous (nrhs, n) tensor (each row one right-hand side)."""
        if _is_torch(B):
            nrhs = 1 if B.dim() == 1 else B.shape[0]
            solve(self.h, B, self.n, nrhs, stream)
            return B
        if not (B.flags.f_contiguous and B.dtype == np.float64):
            raise ValueError("numpy B must be float64 and Fortran-contiguous")
        nrhs = 1 if B.ndim == 1 else B.shape[1]
        solve(self.h, B, self.n, nrhs, stream)
        return B

    def stats(self):
        return stats(self.h)

    def export_factor(self):
        return export_factor(self.h)

    def close(self):
        destroy(self.h)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
