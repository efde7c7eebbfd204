"""The paper's own CPU method (Algorithms 1-3 as parallel counting sorts, and
Top-K-sadilla), restated in C++/OpenMP so that the bench can time it on the
host cores beside the GPU path, for context.

Bench and test infrastructure: it shares no code with the CUDA library and
is not the oracle either (the tests check it against the oracle). Nothing in
the product package imports it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qsd_cpu_method.cpp")
_LIB = os.path.join(_HERE, "libqsd_cpu_method.so")
_lib = None


def build(force: bool = False) -> str:
    """Compiles qsd_cpu_method.cpp (OpenMP) with g++ into a shared library."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["g++", "-O2", "-std=c++17", "-fopenmp", "-shared", "-fPIC",
                        _SRC, "-o", tmp], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        i64, p = ctypes.c_int64, ctypes.c_void_p
        L.qsd_cpu_method_transpose_topk.argtypes = [ctypes.c_int, i64, p, i64, p, ctypes.c_int, p,
                                                    p, p, ctypes.c_int, ctypes.c_int, p, i64, p]
        L.qsd_cpu_method_transpose_topk.restype = ctypes.c_int
        L.qsd_cpu_method_threads.argtypes = [ctypes.c_int]
        L.qsd_cpu_method_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def transpose(coords: np.ndarray, vals, dims, sigma, tau=None, threads: int = 0,
              top_k: int = 0):
    """The paper's method on the host cores (Algorithm 3's calls as counting
    sorts, parallel as in Section 3.2; top_k > 0: Top-K-sadilla, Section
    3.6). coords: int32 (r, nnz); vals: 1-D 4- or 8-byte items or None.
    Returns (out_coords, out_vals)."""
    L = _load()
    coords = np.ascontiguousarray(coords, dtype=np.int32)
    r, nnz = coords.shape
    tau = list(range(r)) if tau is None else list(tau)
    out_c = np.empty_like(coords)
    vb = 0 if vals is None else vals.dtype.itemsize
    v_in = None if vals is None else np.ascontiguousarray(vals)
    out_v = None if vals is None else np.empty_like(v_in)
    d = np.ascontiguousarray(dims, dtype=np.int64)
    rc = L.qsd_cpu_method_transpose_topk(
        r, nnz, _ptr(coords), nnz, None if v_in is None else _ptr(v_in), vb, _ptr(d),
        _ptr(np.ascontiguousarray(tau, dtype=np.int32)),
        _ptr(np.ascontiguousarray(sigma, dtype=np.int32)), int(top_k), int(threads), _ptr(out_c),
        nnz, None if out_v is None else _ptr(out_v))
    if rc != 0:
        raise ValueError("cpu method rejected its arguments")
    return out_c, out_v


def threads(n: int = 0) -> int:
    """Threads the method runs with (n = 0: all host cores)."""
    return int(_load().qsd_cpu_method_threads(int(n)))
