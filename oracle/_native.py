"""Builds and loads the oracle's plain-C helper (``jacobi.c``) with gcc.

Test infrastructure only. The shared object is written next to the source and
rebuilt whenever the source is newer.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "jacobi.c")
_LIB = os.path.join(_HERE, "_oracle_jacobi.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``jacobi.c`` into ``_oracle_jacobi.so`` (portable flags only)."""
    with _lock:
        stale = (not os.path.exists(_LIB)
                 or os.path.getmtime(_LIB) < os.path.getmtime(_SRC))
        if force or stale:
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.oracle_jacobi_eigh.restype = ctypes.c_int
        lib.oracle_jacobi_eigh.argtypes = [
            ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
            ctypes.c_int, ctypes.c_double]
        _lib = lib
    return _lib


def jacobi_eigh(a: np.ndarray, max_sweeps: int = 100, rel_tol: float = 1e-15):
    """Eigen-decomposition of a symmetric FP64 matrix by cyclic Jacobi rotations.

    Returns (w, V) with eigenvalues sorted ascending and V[:, k] the k-th eigenvector.
    """
    a = np.array(a, dtype=np.float64, order="C", copy=True)
    n = a.shape[0]
    vec = np.zeros((n, n), dtype=np.float64)
    w = np.zeros(n, dtype=np.float64)
    sweeps = _load().oracle_jacobi_eigh(n, a.ctypes.data, vec.ctypes.data, w.ctypes.data,
                                        max_sweeps, rel_tol)
    if sweeps < 0:
        raise RuntimeError("Jacobi iteration did not converge")
    order = np.argsort(w, kind="stable")
    return w[order], vec[:, order]
