"""ctypes loader for the oracle's C direct-sum translation (m2l.c).

TEST INFRASTRUCTURE: used only by the oracle's matrix-free solve.  ``build()`` compiles the shared
object next to the source with gcc and OpenMP.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "m2l.c")
_LIB = os.path.join(_HERE, "_m2l.so")
_lib = None


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", _LIB, _SRC, "-lm"])
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.oracle_m2l_apply.restype = None
        lib.oracle_m2l_apply.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_void_p, ctypes.c_void_p]
        _lib = lib
    return _lib


def apply(xy, k, p, d, alpha, beta):
    """T beta (all pairs, three images) by direct summation in C."""
    lib = _load()
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    b = np.ascontiguousarray(beta, dtype=np.complex128)
    out = np.empty_like(b)
    lib.oracle_m2l_apply(int(xy.shape[0]), int(p), xy.ctypes.data, float(k), float(d),
                         float(np.real(alpha)), float(np.imag(alpha)), b.ctypes.data, out.ctypes.data)
    return out
