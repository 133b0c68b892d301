"""FP64 direct sum (the PPM of Sec. 4.1) -- TEST INFRASTRUCTURE ONLY.

psi(x_i)   = sum_j q_j G(x_i, y_j),  G = (1/4pi) log(d^2/4)        (Eq. SUM, GRE_FUN)
alpha(x_i) = sum_j q_j P_x(x_i - y_j) / (2 pi d^2)                  (Eq. ALP_PSI)

A pair with d^2 == 0 is skipped (self-interaction when targets == sources).
The arithmetic lives in direct.c; this module only marshals arrays.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.oracle_direct.argtypes = [dp, dp, ctypes.c_int64, dp, ctypes.c_int64, dp, dp, dp]
        lib.oracle_direct.restype = ctypes.c_int64
        lib.oracle_threads.argtypes = []
        lib.oracle_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def direct_sum(src, q, tgt, want=("psi", "alpha")):
    """Return a dict with 'psi' [M], 'alpha' [M,2] (e_theta, e_phi),
    'alpha3' [M,3] (tangent 3-vector) as requested, plus 'skipped'."""
    lib = _load()
    src = np.ascontiguousarray(src, dtype=np.float64).reshape(-1, 3)
    tgt = np.ascontiguousarray(tgt, dtype=np.float64).reshape(-1, 3)
    q = np.ascontiguousarray(q, dtype=np.float64).reshape(-1)
    if q.shape[0] != src.shape[0]:
        raise ValueError("q and src differ in length")
    M = tgt.shape[0]
    out = {}
    psi = np.empty(M) if "psi" in want else None
    a2 = np.empty((M, 2)) if "alpha" in want else None
    a3 = np.empty((M, 3)) if "alpha3" in want else None
    out["skipped"] = int(lib.oracle_direct(_ptr(src), _ptr(q), src.shape[0], _ptr(tgt), M,
                                           _ptr(psi), _ptr(a2), _ptr(a3)))
    if psi is not None:
        out["psi"] = psi
    if a2 is not None:
        out["alpha"] = a2
    if a3 is not None:
        out["alpha3"] = a3
    return out


def threads() -> int:
    return int(_load().oracle_threads())
