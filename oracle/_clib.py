"""Build and load the oracle's C Wilson operator (test infrastructure only)."""

from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wilson.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liborc.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile wilson.c with gcc into oracle/_build/liborc.so."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.orc_wilson.restype = None
        _lib.orc_wilson.argtypes = [
            ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
            ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
        _lib.orc_gamma.restype = None
        _lib.orc_gamma.argtypes = [ctypes.c_int, ctypes.c_void_p]
    return _lib


def wilson(U: np.ndarray, dims, bc, M0: float, v: np.ndarray, dag: bool) -> np.ndarray:
    """Apply D_W(-M0) (or its adjoint) to every 4D field stacked in ``v``."""
    U = np.ascontiguousarray(U, dtype=np.complex128)
    v = np.ascontiguousarray(v, dtype=np.complex128)
    V = int(np.prod(dims))
    assert v.size % (V * 12) == 0
    nf = v.size // (V * 12)
    out = np.empty_like(v)
    d = (ctypes.c_int * 4)(*[int(x) for x in dims])
    b = (ctypes.c_int * 4)(*[int(x) for x in bc])
    lib().orc_wilson(U.ctypes.data, d, b, float(M0), int(bool(dag)), int(nf),
                     v.ctypes.data, out.ctypes.data)
    return out


def gamma_table(mu: int) -> np.ndarray:
    out = np.zeros((4, 4), dtype=np.complex128)
    lib().orc_gamma(int(mu), out.ctypes.data)
    return out
