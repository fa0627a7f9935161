"""Builds and loads the oracle's plain-C parts (symbolic analysis, sparse Cholesky).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline load this; the product path never does.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["symbolic.c", "chol.c"]
LIB = os.path.join(HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    srcs = [os.path.join(HERE, s) for s in SOURCES]
    newest = max(os.path.getmtime(s) for s in srcs)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < newest:
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp] + srcs + ["-lm"])
        os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(LIB)
            P = ctypes.c_void_p
            L.osym_analyze.restype = P
            L.osym_analyze.argtypes = [ctypes.c_int, P, P]
            L.osym_analyze_relaxed.restype = P
            L.osym_analyze_relaxed.argtypes = [ctypes.c_int, P, P, ctypes.c_int, ctypes.c_int]
            L.osym_sizes.argtypes = [P, P, P]
            L.osym_export.argtypes = [P] * 7
            L.osym_free.argtypes = [P]
            L.ochol_factor.restype = ctypes.c_int
            L.ochol_factor.argtypes = [ctypes.c_int, P, P, P, P, P, P, P]
            L.ochol_solve.argtypes = [ctypes.c_int, P, P, P, P]
            _lib = L
    return _lib


def ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)
