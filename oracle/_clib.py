"""ORACLE — test infrastructure only.

Builds and loads the oracle's C part (``legendre.c``) with gcc and exposes it
through ctypes.  Nothing here is shared with the GPU library.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "legendre.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle.so")
_lib = None


def build(force=False):
    """Compile legendre.c into oracle/_build/liboracle.so (gcc, OpenMP, FP64).

    -ffp-contract=off keeps the arithmetic the same on x86-64 and aarch64.
    """
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           "-std=c11", "-Wall", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        L.oracle_legendre_column.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_double, dp, dp, ip]
        L.oracle_legendre_column.restype = None
        for name in ("oracle_legendre_inverse", "oracle_legendre_forward"):
            f = getattr(L, name)
            f.argtypes = [ctypes.c_int, dp, ctypes.c_int, dp, dp, dp, ctypes.c_int, ip, dp]
            f.restype = None
        _lib = L
    return _lib


def dptr(a):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def iptr(a):
    assert a.dtype == np.int32 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
