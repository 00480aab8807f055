"""Build and load the oracle's plain-C part (ic0.c) with gcc; ctypes bindings."""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ic0.c")
_LIB = os.path.join(_HERE, "_build", "liboracle_ic0.so")
_handle = None


def build(force: bool = False) -> str:
    """Compile ic0.c into oracle/_build/liboracle_ic0.so (portable flags: x86_64 and aarch64)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _handle
    if _handle is None:
        build()
        h = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        h.oracle_ic0_factor.argtypes = [ctypes.c_int64, P, P, P, P]
        h.oracle_ic0_factor.restype = ctypes.c_int
        h.oracle_ic0_solve.argtypes = [ctypes.c_int64, P, P, P, P, P]
        h.oracle_ic0_solve.restype = None
        _handle = h
    return _handle


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def ic0_factor(indptr: np.ndarray, indices: np.ndarray, data: np.ndarray):
    """IC(0) of a lower-triangular CSR (ascending columns, diagonal last). Returns (L, status)."""
    indptr = np.ascontiguousarray(indptr, dtype=np.int64)
    indices = np.ascontiguousarray(indices, dtype=np.int32)
    data = np.ascontiguousarray(data, dtype=np.float64)
    L = np.zeros_like(data)
    st = lib().oracle_ic0_factor(len(indptr) - 1, _ptr(indptr), _ptr(indices), _ptr(data), _ptr(L))
    return L, int(st)


def ic0_solve(indptr: np.ndarray, indices: np.ndarray, L: np.ndarray, r: np.ndarray) -> np.ndarray:
    r = np.ascontiguousarray(r, dtype=np.float64)
    z = np.empty_like(r)
    lib().oracle_ic0_solve(len(indptr) - 1, _ptr(indptr), _ptr(indices), _ptr(L), _ptr(r), _ptr(z))
    return z
