"""Compile libspchol.so in place for sm_103a (nvcc, no cmake).

Translation units are compiled in parallel, then linked with the static CUDA
runtime, so the library depends only on the driver.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libspchol.so")
HOST_LIB = os.path.join(HERE, "libspchol_host.so")
HOST_SOURCES = ["symbolic.cpp", "hostsim.cpp", "ordering.cpp"]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["api.cu", "factor.cu", "solve.cu", "mixed.cu", "symbolic.cpp", "ordering.cpp"]  # peak_probe.cu is a separate program


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found")
    return cand


def _flags():
    return ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"),
            "-I", CSRC]


def _compile(src: str) -> str:
    obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
    path = os.path.join(CSRC, src)
    cmd = [_nvcc(), *ARCH, *_flags(), "-c", path, "-o", obj]
    if src.endswith(".cpp"):
        cmd = [_nvcc(), *_flags(), "-x", "c++", "-c", path, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return obj


def _stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "spchol.h")]
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build_host(force: bool = False) -> str:
    """Host-only library (symbolic analysis + task-protocol simulator), plain g++."""
    if not force and not _stale(HOST_LIB):
        return HOST_LIB
    cxx = shutil.which("g++") or "g++"
    tmp = HOST_LIB + f".{os.getpid()}.tmp"
    cmd = [cxx, "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off", "-I", os.path.join(ROOT, "include"),
           "-I", CSRC, "-o", tmp] + [os.path.join(CSRC, s) for s in HOST_SOURCES]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"host build failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, HOST_LIB)
    return HOST_LIB


PROBE = os.path.join(BUILD, "peak_probe")


def build_probe() -> str:
    """Arithmetic-throughput probe used for the roofline denominators."""
    src = os.path.join(CSRC, "peak_probe.cu")
    if not os.path.exists(PROBE) or os.path.getmtime(PROBE) < os.path.getmtime(src):
        os.makedirs(BUILD, exist_ok=True)
        subprocess.check_call([_nvcc(), *ARCH, "-O3", "-o", PROBE, src])
    return PROBE


def build(force: bool = False, verbose: bool = False) -> str:
    build_host(force)
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    srcs = [s for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]
    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(_compile, srcs))
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [_nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    if verbose:
        print("built", LIB, file=sys.stderr)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
