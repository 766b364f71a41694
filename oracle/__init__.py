"""Plain CPU oracle for Vietoris-Rips barcodes over Z/2.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library and never imports it; the product path never imports
this.

The arithmetic lives in ``vr_oracle.c`` (plain C, compiled with
``-O2 -ffp-contract=off`` so that every float operation rounds once, as the
single-precision distance formula requires).  This module only marshals
arguments and filters results.  Function-by-function citations of the
dissertation (arXiv 2502.05063) are in the C file; in short:

* ``plain``    -- Algorithm 2 on the full Z/2 boundary matrix of the Rips
                  complex ordered as in Sec. 5.1.4 (the definition).
* ``cohom``    -- Algorithm 12 on the implicit coboundary matrix (Sec. 5.2.1,
                  5.2.8), clearing of Sec. 5.2.3 behind a flag.
* ``apparent`` -- Def 5.3.4 applied literally.
* ``brute``    -- persistent Betti numbers from Z/2 ranks (see brute.py).

Parity pins: every function here is pinned by tests in
``tests/test_oracle_*.py`` against values the paper prints (Figs 4.1/4.2,
5.1, 5.5, 5.6), closed forms (Thm 5.4.2), textbook routines (Kruskal's MST,
scipy's MST) and brute force on small inputs.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vr_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

PAIR_DTYPE = np.dtype([("dim", "<i4"), ("pad", "<i4"), ("birth", "<f8"), ("death", "<f8"),
                       ("birth_cidx", "<i8"), ("death_cidx", "<i8")])


def build(force: bool = False) -> str:
    """Compile vr_oracle.c into liboracle.so next to it (gcc, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.POINTER
            c_i64, c_i32, c_dbl = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
            lib.or_distances_f32.argtypes = [ctypes.c_void_p, c_i64, c_i32, ctypes.c_void_p]
            lib.or_distances_f64.argtypes = [ctypes.c_void_p, c_i64, c_i32, ctypes.c_void_p]
            lib.or_enclosing_radius.argtypes = [ctypes.c_void_p, c_i64]
            lib.or_enclosing_radius.restype = c_dbl
            lib.or_plain.argtypes = [ctypes.c_void_p, c_i64, c_i32, c_dbl, P(ctypes.c_void_p)]
            lib.or_plain.restype = c_i64
            lib.or_cohom.argtypes = [ctypes.c_void_p, c_i64, c_i32, c_dbl, c_i32,
                                     P(ctypes.c_void_p), ctypes.c_void_p]
            lib.or_cohom.restype = c_i64
            lib.or_apparent.argtypes = [ctypes.c_void_p, c_i64, c_i32, c_dbl, P(ctypes.c_void_p)]
            lib.or_apparent.restype = c_i64
            lib.or_reduce_explicit.argtypes = [c_i64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
            lib.or_reduce_explicit.restype = c_i64
            lib.or_simplex_vertices.argtypes = [ctypes.c_uint64, c_i32, c_i64, ctypes.c_void_p]
            lib.or_simplex_vertices.restype = c_i32
            lib.or_simplex_index.argtypes = [ctypes.c_void_p, c_i32, c_i64]
            lib.or_simplex_index.restype = ctypes.c_uint64
            lib.or_critical_edge.argtypes = [ctypes.c_void_p, c_i64, ctypes.c_uint64, c_i32, ctypes.c_void_p]
            lib.or_critical_edge.restype = c_i32
            lib.or_free.argtypes = [ctypes.c_void_p]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def distances_f32(pts: np.ndarray) -> np.ndarray:
    """Condensed lower triangle of the float32 distance formula."""
    pts = np.ascontiguousarray(pts, dtype=np.float32)
    n, dim = pts.shape
    out = np.zeros(n * (n - 1) // 2, dtype=np.float32)
    _load().or_distances_f32(_ptr(pts), n, dim, _ptr(out))
    return out


def distances_f64(pts: np.ndarray) -> np.ndarray:
    pts = np.ascontiguousarray(pts, dtype=np.float64)
    n, dim = pts.shape
    out = np.zeros(n * (n - 1) // 2, dtype=np.float64)
    _load().or_distances_f64(_ptr(pts), n, dim, _ptr(out))
    return out


def enclosing_radius(D: np.ndarray, n: int) -> float:
    D = np.ascontiguousarray(D, dtype=np.float64)
    return float(_load().or_enclosing_radius(_ptr(D), n))


def _take_pairs(ptr, count) -> np.ndarray:
    if count < 0:
        raise RuntimeError("oracle failed (%d)" % count)
    if count == 0:
        if ptr.value:
            _load().or_free(ptr)
        return np.zeros(0, dtype=PAIR_DTYPE)
    buf = (ctypes.c_char * (count * PAIR_DTYPE.itemsize)).from_address(ptr.value)
    arr = np.frombuffer(bytes(buf), dtype=PAIR_DTYPE).copy()
    _load().or_free(ptr)
    return arr


def plain(D: np.ndarray, n: int, dmax: int, threshold: float = np.inf) -> np.ndarray:
    """All pairs (incl. zero-length and essential) by Algorithm 2."""
    D = np.ascontiguousarray(D, dtype=np.float64)
    out = ctypes.c_void_p()
    c = _load().or_plain(_ptr(D), n, dmax, float(threshold), ctypes.byref(out))
    return _take_pairs(out, c)


def cohom(D: np.ndarray, n: int, dmax: int, threshold: float = np.inf, clearing: bool = False):
    """All pairs by the oblivious dual reduction (Algorithm 12).

    Returns (pairs, stats) with stats[p] = (columns, additions, pairs, essential)."""
    D = np.ascontiguousarray(D, dtype=np.float64)
    out = ctypes.c_void_p()
    stats = np.zeros(4 * (dmax + 1), dtype=np.int64)
    c = _load().or_cohom(_ptr(D), n, dmax, float(threshold), int(bool(clearing)),
                         ctypes.byref(out), _ptr(stats))
    return _take_pairs(out, c), stats.reshape(dmax + 1, 4)


def apparent(D: np.ndarray, n: int, p: int, threshold: float = np.inf) -> np.ndarray:
    """(s, t) combinatorial indices of the dimension-(p, p+1) apparent pairs (Def 5.3.4)."""
    D = np.ascontiguousarray(D, dtype=np.float64)
    out = ctypes.c_void_p()
    c = _load().or_apparent(_ptr(D), n, p, float(threshold), ctypes.byref(out))
    if c < 0:
        raise RuntimeError("oracle failed")
    if c == 0:
        return np.zeros((0, 2), dtype=np.uint64)
    buf = (ctypes.c_char * (16 * c)).from_address(out.value)
    arr = np.frombuffer(bytes(buf), dtype=np.uint64).reshape(c, 2).copy()
    _load().or_free(out)
    return arr


def reduce_explicit(columns) -> np.ndarray:
    """Algorithm 2 on an explicit Z/2 matrix given as a list of row lists."""
    N = len(columns)
    colptr = np.zeros(N + 1, dtype=np.int64)
    rows = []
    for j, c in enumerate(columns):
        rows.extend(sorted(c))
        colptr[j + 1] = len(rows)
    rows = np.asarray(rows if rows else [0], dtype=np.int64)
    low = np.zeros(max(N, 1), dtype=np.int64)
    if _load().or_reduce_explicit(N, _ptr(colptr), _ptr(rows), _ptr(low)) != 0:
        raise RuntimeError("oracle failed")
    return low[:N]


def simplex_vertices(cidx: int, q: int, n: int) -> list:
    v = np.zeros(q + 1, dtype=np.int32)
    if _load().or_simplex_vertices(int(cidx), q, n, _ptr(v)) != 0:
        raise RuntimeError("oracle failed")
    return [int(x) for x in v]


def simplex_index(vertices, n: int) -> int:
    v = np.ascontiguousarray(sorted(vertices), dtype=np.int32)
    return int(_load().or_simplex_index(_ptr(v), len(v) - 1, n))


def critical_edge(D: np.ndarray, n: int, cidx: int, q: int):
    D = np.ascontiguousarray(D, dtype=np.float64)
    uv = np.zeros(2, dtype=np.int32)
    if _load().or_critical_edge(_ptr(D), n, int(cidx), q, _ptr(uv)) != 0:
        raise RuntimeError("oracle failed")
    return int(uv[0]), int(uv[1])


def diagram(pairs: np.ndarray, dmax: int, keep_zero: bool = False):
    """Per-dimension list of (birth, death, birth_cidx, death_cidx) rows, sorted.

    Zero-length pairs (death == birth) are dropped unless keep_zero; the sort
    key is (birth, death, birth_cidx)."""
    res = []
    for p in range(dmax + 1):
        sel = pairs[pairs["dim"] == p]
        if not keep_zero:
            sel = sel[sel["death"] > sel["birth"]]
        order = np.lexsort((sel["birth_cidx"], sel["death"], sel["birth"]))
        res.append(sel[order])
    return res
