"""Reference oracle for sparse COO tensor transposition (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the bench's CPU-baseline leg
use this package. It shares no code with the CUDA library: the transposition
oracle is ``qsd_oracle.cpp`` (a stable sort under the target-order
lexicographic comparator, Section 2), the planner oracle is ``plan.py``
(Algorithm 3 and an exhaustive search, Sections 3.4-3.5), ``partial_sort``
holds Algorithms 1 and 2 as literal loops and ``csf`` the CSF levels.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qsd_oracle.cpp")
_LIB_PATH = os.path.join(_HERE, "libqsd_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compiles the C++ oracle with g++ into oracle/libqsd_oracle.so."""
    if force or not os.path.exists(_LIB_PATH) or (
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC",
                        _SRC, "-o", tmp], check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        i64, p = ctypes.c_int64, ctypes.c_void_p
        L.qsd_oracle_permutation.argtypes = [ctypes.c_int, i64, p, i64, p, p]
        L.qsd_oracle_permutation.restype = ctypes.c_int
        L.qsd_oracle_transpose.argtypes = [ctypes.c_int, i64, p, i64, p,
                                           ctypes.c_int, p, p, i64, p]
        L.qsd_oracle_transpose.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def transpose(coords: np.ndarray, vals: np.ndarray | None, sigma):
    """Stable sigma-lexicographic re-sort of a COO tensor.

    coords: int32 array of shape (r, nnz) (one row per mode); vals: 1-D array
    of 4- or 8-byte items or None. Returns (out_coords, out_vals).
    """
    coords = np.ascontiguousarray(coords, dtype=np.int32)
    r, nnz = coords.shape
    sig = np.ascontiguousarray(sigma, dtype=np.int32)
    out_c = np.empty_like(coords)
    vb = 0 if vals is None else vals.dtype.itemsize
    v_in = None if vals is None else np.ascontiguousarray(vals)
    out_v = None if vals is None else np.empty_like(v_in)
    rc = lib().qsd_oracle_transpose(
        r, nnz, _ptr(coords), nnz, None if v_in is None else _ptr(v_in), vb,
        _ptr(sig), _ptr(out_c), nnz, None if out_v is None else _ptr(out_v))
    if rc != 0:
        raise ValueError("oracle rejected its arguments")
    return out_c, out_v


def permutation(coords: np.ndarray, sigma) -> np.ndarray:
    """Input index of each output entry of the stable sigma-lexicographic sort."""
    coords = np.ascontiguousarray(coords, dtype=np.int32)
    r, nnz = coords.shape
    sig = np.ascontiguousarray(sigma, dtype=np.int32)
    perm = np.empty(nnz, dtype=np.int64)
    rc = lib().qsd_oracle_permutation(r, nnz, _ptr(coords), nnz, _ptr(sig),
                                      _ptr(perm))
    if rc != 0:
        raise ValueError("oracle rejected its arguments")
    return perm


def rank_under(coords: np.ndarray, sigma, entry) -> tuple:
    """(#entries strictly less than `entry`, #entries equal to it) under the
    sigma-lexicographic order of Section 2, counted directly over all entries.

    For a transposition this fixes where `entry` lands: a stable sort places
    the entries equal to it at positions [less, less + equal). Plain numpy,
    O(r * nnz) per call; used to check single output positions of tensors too
    large for the full oracle.
    """
    coords = np.asarray(coords)
    nnz = coords.shape[1]
    lt = np.zeros(nnz, dtype=bool)
    eq = np.ones(nnz, dtype=bool)
    for m in sigma:
        col = coords[m]
        v = entry[m]
        lt |= eq & (col < v)
        eq &= col == v
    return int(lt.sum()), int(eq.sum())
