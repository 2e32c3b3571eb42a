"""Build and load the oracle's C loops (test infrastructure only).

gcc -O2 -fopenmp, IEEE semantics (no -ffast-math), no machine-specific flags,
so the same source gives the same results on x86_64 and aarch64.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "_oracle_loops.c")
_LIB = os.path.join(_HERE, "_oracle_loops.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle loops into oracle/_oracle_loops.so."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            I64 = ctypes.c_int64
            L.orc_direct_type2.argtypes = [ctypes.c_int, P, P, P, I64, P, P]
            L.orc_direct_type1.argtypes = [ctypes.c_int, P, P, I64, P, P, P]
            L.orc_interp.argtypes = [ctypes.c_int, P, P, I64, P, ctypes.c_int, ctypes.c_double, P]
            L.orc_spread.argtypes = [ctypes.c_int, P, I64, P, P, ctypes.c_int, ctypes.c_double, P]
            for f in (L.orc_direct_type2, L.orc_direct_type1, L.orc_interp, L.orc_spread):
                f.restype = None
            L.orc_set_threads.argtypes = [ctypes.c_int]
            L.orc_set_threads.restype = None
            L.orc_max_threads.argtypes = []
            L.orc_max_threads.restype = ctypes.c_int
            _lib = L
    return _lib


def ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def i64arr(v):
    return np.ascontiguousarray(np.asarray(v, dtype=np.int64))


def f64arr(v):
    return np.ascontiguousarray(np.asarray(v, dtype=np.float64))


def set_threads(n: int):
    """Limit OpenMP threads for subsequent oracle calls."""
    lib().orc_set_threads(int(n))


def max_threads() -> int:
    return int(lib().orc_max_threads())
