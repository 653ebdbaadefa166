"""Loader for the oracle's C loops (oracle/csrc/oracle.c).

Test infrastructure only.  ``build()`` compiles the C file with gcc into
``oracle/_oracle.so`` (OpenMP, -O2, no fast-math, no FMA contraction so that
x86 and Arm hosts round the same way).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csrc", "oracle.c")
_SO = os.path.join(_HERE, "_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle's C loops; returns the path of the shared library."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    tmp = _SO + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


_D = ctypes.POINTER(ctypes.c_double)
_I64 = ctypes.POINTER(ctypes.c_int64)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            i64, i32, dbl = ctypes.c_int64, ctypes.c_int, ctypes.c_double
            L.o1_direct.restype = i64
            L.o1_direct.argtypes = [i32, i64, _D, _D, _D, i64, _I64, _D, _D]
            L.o1_grad_x.restype = None
            L.o1_grad_x.argtypes = [i32, i64, _D, _D, _D, _D, i64, _I64, _D]
            L.o1_grad_f.restype = None
            L.o1_grad_f.argtypes = [i32, i64, _D, _D, i64, _I64, _D]
            L.o1_grad_fq.restype = None
            L.o1_grad_fq.argtypes = [i64, _D, _D, _D, _D, i64, _I64, _D, _D]
            L.o_kernel_full.restype = None
            L.o_kernel_full.argtypes = [i32, i64, _D, _D]
            L.o_kernel_real.restype = None
            L.o_kernel_real.argtypes = [i32, i64, _D, dbl, _D]
            L.o_kernel_real_grad.restype = i32
            L.o_kernel_real_grad.argtypes = [i32, i64, _D, dbl, _D]
            L.o2_real.restype = i64
            L.o2_real.argtypes = [i32, i64, _D, _D, _D, i64, _I64, _D, dbl, dbl, _D]
            L.o2_real_T.restype = None
            L.o2_real_T.argtypes = [i32, i64, _D, _D, i64, _I64, dbl, dbl, _D]
            L.o2_real_grad_x.restype = i32
            L.o2_real_grad_x.argtypes = [i32, i64, _D, _D, _D, i64, _I64, dbl, dbl, _D]
            L.o2_spread.restype = i32
            L.o2_spread.argtypes = [i64, _D, i32, _D, i32, i32, dbl, _D, dbl, dbl, _D]
            L.o2_gather.restype = i32
            L.o2_gather.argtypes = [i64, _D, i32, _D, i32, i32, dbl, _D, dbl, dbl, _D]
            L.o2_gather_grad.restype = i32
            L.o2_gather_grad.argtypes = [i64, _D, i32, _D, _D, _D, _D, i32, i32, dbl, _D, dbl,
                                         dbl, _D]
            _lib = L
    return _lib


def dptr(a: np.ndarray | None):
    if a is None:
        return ctypes.cast(None, _D)
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def iptr(a: np.ndarray | None):
    if a is None:
        return ctypes.cast(None, _I64)
    assert a.dtype == np.int64 and a.flags.c_contiguous
    return a.ctypes.data_as(_I64)


def f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))
