"""CPU oracle for maximal all-ones square detection — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
(and its ``--impl reference`` arm) may import this package.  The CUDA library
never uses it.  The C routines and their parity status are described in
``oracle.h``; this file is ctypes marshalling plus ``erode`` and ``unpack``
conveniences.

Results are ``(side, row, col)`` tuples: the largest all-ones square side and
the bottom-right corner of the first such square in row-major order
(``(0, -1, -1)`` when there is none).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")

_i64 = ctypes.c_int64
_vp = ctypes.c_void_p


class _Result(ctypes.Structure):
    _fields_ = [("side", ctypes.c_int32), ("row", ctypes.c_int32), ("col", ctypes.c_int32),
                ("status", ctypes.c_int32)]


class _Cube(ctypes.Structure):
    _fields_ = [("side", ctypes.c_int32), ("slice", ctypes.c_int32), ("row", ctypes.c_int32),
                ("col", ctypes.c_int32)]


def build(force: bool = False) -> str:
    srcs = [os.path.join(_HERE, f) for f in ("oracle.c", "oracle.h")]
    if force or not os.path.exists(_SO) or any(os.path.getmtime(s) > os.path.getmtime(_SO)
                                               for s in srcs):
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-o", _SO, srcs[0]])
    return _SO


_lib = None


def _l():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        for name in ("oracle_dp", "oracle_freq_dpmap"):
            f = getattr(lib, name)
            f.restype = ctypes.c_int
            f.argtypes = [_vp, _i64, _i64, _i64, _vp, _i64, ctypes.POINTER(_Result)]
        for name in ("oracle_dp_rows", "oracle_freq", "oracle_brute"):
            f = getattr(lib, name)
            f.restype = ctypes.c_int
            f.argtypes = [_vp, _i64, _i64, _i64, ctypes.POINTER(_Result)]
        lib.oracle_all_max.restype = ctypes.c_int
        lib.oracle_all_max.argtypes = [_vp, _i64, _i64, _i64, _vp, _i64,
                                       ctypes.POINTER(_i64), ctypes.POINTER(_Result)]
        lib.oracle_cube.restype = ctypes.c_int
        lib.oracle_cube.argtypes = [_vp, _i64, _i64, _i64, _i64, _i64, ctypes.POINTER(_Cube)]
        lib.oracle_erode.restype = ctypes.c_int
        lib.oracle_erode.argtypes = [_vp, _i64, _i64, _i64, _i64, _vp, _i64]
        _lib = lib
    return _lib


def _mat(a: np.ndarray, n: int | None):
    a = np.asarray(a)
    if a.ndim != 2:
        raise ValueError("expected a 2-D matrix")
    if a.dtype != np.uint8 or not a.flags.c_contiguous:
        a = np.ascontiguousarray(a, dtype=np.uint8)
    m = a.shape[0]
    n = a.shape[1] if n is None else n
    ld = max(a.shape[1], 1)
    if m == 0 or n == 0:
        a = np.zeros((max(m, 1), max(ld, 1)), dtype=np.uint8)
    return a, m, n, ld


def _tuple(r: _Result):
    return (int(r.side), int(r.row), int(r.col))


def _check(rc: int, name: str):
    if rc != 0:
        raise MemoryError(f"{name}: allocation failed")


def dp(a: np.ndarray, n: int | None = None, want_map: bool = True):
    """Textbook DP (Eq. 1).  Returns ((side, row, col), dp map or None)."""
    a, m, n, ld = _mat(a, n)
    res = _Result()
    if want_map and m > 0 and n > 0:
        out = np.zeros((m, n), dtype=np.int32)
        _check(_l().oracle_dp(a.ctypes.data, m, n, ld, out.ctypes.data, n, ctypes.byref(res)),
               "oracle_dp")
        return _tuple(res), out
    _check(_l().oracle_dp(a.ctypes.data, m, n, ld, None, 0, ctypes.byref(res)), "oracle_dp")
    return _tuple(res), (np.zeros((m, n), dtype=np.int32) if want_map else None)


def dp_rows(a: np.ndarray, n: int | None = None):
    """O(n)-space DP (Sec. 4.9 baseline).  Returns (side, row, col)."""
    a, m, n, ld = _mat(a, n)
    res = _Result()
    _check(_l().oracle_dp_rows(a.ctypes.data, m, n, ld, ctypes.byref(res)), "oracle_dp_rows")
    return _tuple(res)


def freq(a: np.ndarray, n: int | None = None):
    """The paper's Algorithm 1 (side instead of area) with its last validation."""
    a, m, n, ld = _mat(a, n)
    res = _Result()
    _check(_l().oracle_freq(a.ctypes.data, m, n, ld, ctypes.byref(res)), "oracle_freq")
    return _tuple(res)


def freq_dpmap(a: np.ndarray, n: int | None = None):
    """DP map from the frequency array.  Returns ((side, row, col), dp map)."""
    a, m, n, ld = _mat(a, n)
    res = _Result()
    out = np.zeros((m, n), dtype=np.int32)
    dst = out.ctypes.data if (m > 0 and n > 0) else None
    _check(_l().oracle_freq_dpmap(a.ctypes.data, m, n, ld, dst, n, ctypes.byref(res)),
           "oracle_freq_dpmap")
    return _tuple(res), out


def brute(a: np.ndarray, n: int | None = None):
    a, m, n, ld = _mat(a, n)
    res = _Result()
    _check(_l().oracle_brute(a.ctypes.data, m, n, ld, ctypes.byref(res)), "oracle_brute")
    return _tuple(res)


def all_max(a: np.ndarray, n: int | None = None):
    """Every bottom-right corner of a largest all-ones square, row-major.
    Returns ((side, row, col), int32 array of shape (count, 2))."""
    a, m, n, ld = _mat(a, n)
    res = _Result()
    cnt = _i64(0)
    _check(_l().oracle_all_max(a.ctypes.data, m, n, ld, None, 0, ctypes.byref(cnt),
                               ctypes.byref(res)), "oracle_all_max")
    out = np.zeros((max(cnt.value, 1), 2), dtype=np.int32)
    if cnt.value:
        _check(_l().oracle_all_max(a.ctypes.data, m, n, ld, out.ctypes.data, cnt.value,
                                   ctypes.byref(cnt), ctypes.byref(res)), "oracle_all_max")
    return _tuple(res), out[:cnt.value]


def cube(v: np.ndarray):
    """Largest all-ones cube of a (d, m, n) volume: (side, slice, row, col) of
    the first corner, in (z, i, j) order, of a largest cube."""
    v = np.ascontiguousarray(np.asarray(v), dtype=np.uint8)
    if v.ndim != 3:
        raise ValueError("expected a 3-D volume")
    d, m, n = v.shape
    res = _Cube()
    buf = v if v.size else np.zeros(1, dtype=np.uint8)
    _check(_l().oracle_cube(buf.ctypes.data, d, m, n, max(n, 1), max(m * n, 1),
                            ctypes.byref(res)), "oracle_cube")
    return (int(res.side), int(res.slice), int(res.row), int(res.col))


def erode(a: np.ndarray, t: int, n: int | None = None) -> np.ndarray:
    """uint8 map of bottom-right corners of all-ones t x t squares."""
    a, m, n, ld = _mat(a, n)
    out = np.zeros((m, n), dtype=np.uint8)
    if m > 0 and n > 0:
        _check(_l().oracle_erode(a.ctypes.data, m, n, ld, t, out.ctypes.data, n), "oracle_erode")
    return out


def unpack(words: np.ndarray, m: int, n: int) -> np.ndarray:
    """MS_BITS32 rows -> uint8 0/1 (bit b of word w is column 32*w+b; padding ignored)."""
    w = np.ascontiguousarray(words, dtype=np.uint32)
    if m == 0 or n == 0:
        return np.zeros((m, n), dtype=np.uint8)
    bits = np.unpackbits(w.view(np.uint8).reshape(m, -1), axis=1, bitorder="little")
    return np.ascontiguousarray(bits[:, :n])
