"""Build and load the oracle's C library (liboracle.so).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the timed
CPU baseline, never by the CUDA path.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csrc", "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (-O2, OpenMP, portable flags only)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    compile_to(_SRC, tmp)
    os.replace(tmp, _LIB)
    return _LIB


def compile_to(src: str, out: str) -> None:
    """gcc -O2 with OpenMP into the shared library ``out``; no contraction of
    a * b + c into fused multiply-adds, so every machine rounds each operation
    as written."""
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-o", out, src, "-lm"]
    subprocess.run(cmd, check=True)


def bind(path: str):
    """Load a compiled oracle.c from ``path`` and declare its signatures."""
    L = ctypes.CDLL(path)
    i32p = ctypes.POINTER(ctypes.c_int32)
    f64p = ctypes.POINTER(ctypes.c_double)
    L.oracle_series.argtypes = [ctypes.c_int32, i32p, i32p, i32p, ctypes.c_int32,
                                ctypes.c_int32, i32p, f64p, f64p, f64p, ctypes.c_int32]
    L.oracle_series.restype = ctypes.c_int
    L.oracle_cg.argtypes = [ctypes.c_int32, i32p, i32p, ctypes.c_int32, i32p, i32p,
                            ctypes.c_double, ctypes.c_int32, f64p, i32p, ctypes.c_int32]
    L.oracle_cg.restype = ctypes.c_int
    L.oracle_cg_block.argtypes = L.oracle_cg.argtypes
    L.oracle_cg_block.restype = ctypes.c_int
    L.oracle_series_terms.argtypes = [ctypes.c_int32, i32p, i32p, ctypes.c_int32, ctypes.c_int32, i32p,
                                      ctypes.POINTER(ctypes.c_int64), f64p, ctypes.c_int32]
    L.oracle_series_terms.restype = ctypes.c_int
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = bind(_LIB)
    return _lib


def ptr(a, ctype):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def default_threads() -> int:
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
