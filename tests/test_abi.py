"""The C-ABI libraries load without a GPU and export every declared entry point."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1608_00044_gb300 import build, spchol

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = {
    "spchol.h": "libspchol.so",
    "spchol_host.h": "libspchol_host.so",
}


def _declared(header):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(spchol_[a-z0-9_]+)\s*\(", src)))


def test_build_produces_libraries():
    build.build()
    for lib in HEADERS.values():
        assert os.path.exists(os.path.join(ROOT, "paper_1608_00044_gb300", lib))


@pytest.mark.parametrize("header", sorted(HEADERS))
def test_every_declared_symbol_is_exported(header):
    build.build()
    lib = ctypes.CDLL(os.path.join(ROOT, "paper_1608_00044_gb300", HEADERS[header]))
    names = _declared(header)
    assert len(names) >= 7
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    names = set(_declared("spchol.h"))
    bound = {n for n, _, _ in spchol.SIGNATURES}
    assert names == bound


def test_strerror_and_defaults_without_gpu():
    build.build()
    assert "wait budget" in spchol.strerror(spchol.ETIMEOUT)
    assert "not positive definite" in spchol.strerror(7)
    assert "invalid argument" in spchol.strerror(-3)
    o = spchol.default_options()
    assert (o.precision, o.max_width, o.relax_zeros, o.ir_max_iter) == (spchol.FP64, 64, 4, 10)
    assert o.wait_budget_ns == 2_000_000_000 and o.fault_inject == 0
    host = spchol.default_options_host()
    for f, _ in spchol.Options._fields_:
        assert getattr(o, f) == getattr(host, f), f


def test_analyze_argument_checks_precede_device_work():
    build.build()
    lib = spchol.load()
    h = ctypes.c_void_p()
    bad_opt = spchol.default_options(max_width=0)
    cp = np.array([0, 1], np.int64)
    ri = np.array([0], np.int32)
    assert lib.spchol_analyze(1, cp.ctypes.data, ri.ctypes.data, None, ctypes.byref(bad_opt), ctypes.byref(h)) == -5
    assert lib.spchol_analyze(1, cp.ctypes.data, ri.ctypes.data, None, None, None) == -6
    # the schedule switch and the allocator hook pair are checked with the options
    for bad in (spchol.default_options(sched=2), spchol.default_options(sched=-1)):
        assert lib.spchol_analyze(1, cp.ctypes.data, ri.ctypes.data, None, ctypes.byref(bad), ctypes.byref(h)) == -5
    cb = spchol.DEV_ALLOC_FN(lambda n, s, c: None)
    half = spchol.default_options()
    half.dev_alloc = ctypes.cast(cb, ctypes.c_void_p).value  # dev_free left NULL
    assert lib.spchol_analyze(1, cp.ctypes.data, ri.ctypes.data, None, ctypes.byref(half), ctypes.byref(h)) == -5


def test_no_cpu_fallback_in_the_product_library():
    """The GPU library has no host numeric path: without a device, analyze fails
    loudly instead of computing anything."""
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    lib = spchol.load()
    h = ctypes.c_void_p()
    cp = np.array([0, 1], np.int64)
    ri = np.array([0], np.int32)
    assert lib.spchol_analyze(1, cp.ctypes.data, ri.ctypes.data, None, None, ctypes.byref(h)) == spchol.ECUDA
