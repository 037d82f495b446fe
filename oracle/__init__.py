"""CPU FP64 oracle for the continuous box Gauss transform (paper eq. (bgt)).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only callers.  The GPU product path never
imports this package, and this package imports nothing from the product.

``box_fgt`` evaluates u(x) = int_B G(x-y; delta) sigma~(y) dy at the Gauss-Legendre
nodes of chosen target leaves, where sigma~ is the per-leaf tensor Lagrange
interpolant of the node values (the density the paper's Algorithm 4 takes as
input).  The arithmetic lives in ``oracle.c``; see its header comment.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into _oracle.so with gcc (portable flags only)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-pthread", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_box_fgt.restype = ctypes.c_int
            lib.oracle_box_fgt.argtypes = [
                ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_long,
                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                ctypes.c_long, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
            lib.oracle_box_fgt_boxes.restype = ctypes.c_int
            lib.oracle_box_fgt_boxes.argtypes = [
                ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_long,
                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                ctypes.c_long, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
            lib.oracle_point_fgt.restype = ctypes.c_int
            lib.oracle_point_fgt.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_long, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_long, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_int]
            lib.oracle_gauss_legendre.restype = ctypes.c_int
            lib.oracle_gauss_legendre.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
            lib.oracle_default_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def default_threads() -> int:
    return int(_load().oracle_default_threads())


def gauss_legendre(n: int):
    """The oracle's own n-point Gauss-Legendre rule on [-1, 1] (ascending)."""
    x = np.zeros(n)
    w = np.zeros(n)
    if _load().oracle_gauss_legendre(n, x.ctypes.data, w.ctypes.data) != 0:
        raise ValueError("bad n")
    return x, w


def box_fgt(d, p, delta, periodic, leaf_level, leaf_coord, sigma, targets=None, threads=0):
    """u[len(targets), p**d] at the nodes of the target leaves (default: all leaves).

    leaf_level: int32 [n_leaves]; leaf_coord: int32 [n_leaves, d] (box index at its
    level); sigma: float64 [n_leaves, p**d], node index j_1 (x_1) fastest.
    """
    lev = np.ascontiguousarray(leaf_level, dtype=np.int32)
    crd = np.ascontiguousarray(leaf_coord, dtype=np.int32).reshape(-1)
    sig = np.ascontiguousarray(sigma, dtype=np.float64).reshape(len(lev), p ** d)
    if targets is None:
        targets = np.arange(len(lev))
    tg = np.ascontiguousarray(targets, dtype=np.int64)
    u = np.zeros((len(tg), p ** d))
    rc = _load().oracle_box_fgt(int(d), int(p), float(delta), int(bool(periodic)), len(lev),
                                lev.ctypes.data, crd.ctypes.data, sig.ctypes.data,
                                len(tg), tg.ctypes.data, u.ctypes.data, int(threads))
    if rc != 0:
        raise RuntimeError(f"oracle_box_fgt failed ({rc})")
    return u


def box_fgt_boxes(d, p, delta, periodic, leaf_level, leaf_coord, sigma, tgt_level, tgt_coord, threads=0):
    """u[n_boxes, p**d] at the nodes of target boxes given by their own level and coordinates
    (for example the leaves of an output tree that refines or coarsens the source tree)."""
    lev = np.ascontiguousarray(leaf_level, dtype=np.int32)
    crd = np.ascontiguousarray(leaf_coord, dtype=np.int32).reshape(-1)
    sig = np.ascontiguousarray(sigma, dtype=np.float64).reshape(len(lev), p ** d)
    tl = np.ascontiguousarray(tgt_level, dtype=np.int32)
    tc = np.ascontiguousarray(tgt_coord, dtype=np.int32).reshape(-1)
    u = np.zeros((len(tl), p ** d))
    rc = _load().oracle_box_fgt_boxes(int(d), int(p), float(delta), int(bool(periodic)), len(lev),
                                      lev.ctypes.data, crd.ctypes.data, sig.ctypes.data,
                                      len(tl), tl.ctypes.data, tc.ctypes.data, u.ctypes.data, int(threads))
    if rc != 0:
        raise RuntimeError(f"oracle_box_fgt_boxes failed ({rc})")
    return u


def point_fgt(d, delta, src, q, tgt, threads=0):
    """u[i] = sum_j exp(-|x_i - y_j|^2/delta) q_j (the discrete Gauss transform, summed directly)."""
    y = np.ascontiguousarray(src, dtype=np.float64).reshape(-1, d)
    w = np.ascontiguousarray(q, dtype=np.float64).reshape(-1)
    x = np.ascontiguousarray(tgt, dtype=np.float64).reshape(-1, d)
    u = np.zeros(len(x))
    rc = _load().oracle_point_fgt(int(d), float(delta), len(y), y.ctypes.data, w.ctypes.data, len(x),
                                  x.ctypes.data, u.ctypes.data, int(threads))
    if rc != 0:
        raise RuntimeError("oracle_point_fgt failed")
    return u
