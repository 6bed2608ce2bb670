"""Loads (building on first use) the oracle's plain C kernel loops.

TEST INFRASTRUCTURE ONLY.  The library is compiled from
``oracle/csrc/oracle_kernel.c`` with gcc and OpenMP; nothing in the CUDA
path links it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csrc", "oracle_kernel.c")
_OUT = os.path.join(_HERE, "csrc", "liboracle_kernel.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle's C file into a shared library next to it."""
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i64 = ctypes.c_int64
            L.okrr_kernel_matrix.argtypes = [P, i64, P, i64, ctypes.c_int, ctypes.c_double, P]
            L.okrr_kernel_matrix.restype = None
            L.okrr_sqdist_matrix.argtypes = [P, i64, P, i64, ctypes.c_int, P]
            L.okrr_sqdist_matrix.restype = None
            L.okrr_kernel_product.argtypes = [P, i64, P, i64, ctypes.c_int, ctypes.c_double,
                                              P, ctypes.c_int, P, P, P, i64, P, P]
            L.okrr_kernel_product.restype = None
            L.okrr_num_threads.restype = ctypes.c_int
            _lib = L
    return _lib


def ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)
