"""Seeded synthetic 0/1 matrices shared by the oracle side and the CUDA side.

This module draws inputs only; it contains none of the maximal-square
arithmetic.  The generator definition (counter-style SplitMix64, Bernoulli by a
24-bit threshold, planted squares, the MS_BITS32 packing) is in ``msgen.h``.

Host functions use ``libmsgen.so`` (gcc); ``fill_u8_dev`` and friends use
``libmsgen_dev.so`` (nvcc) and take raw device pointers plus a CUDA stream.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_HOST_SO = os.path.join(_HERE, "libmsgen.so")
_DEV_SO = os.path.join(_HERE, "libmsgen_dev.so")

_i64 = ctypes.c_int64
_u64 = ctypes.c_uint64
_u32 = ctypes.c_uint32
_vp = ctypes.c_void_p


def _stale(target: str, *sources: str) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(os.path.join(_HERE, s)) > t for s in sources)


def build_host(force: bool = False) -> str:
    if force or _stale(_HOST_SO, "msgen.c", "msgen.h"):
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-o", _HOST_SO,
                               os.path.join(_HERE, "msgen.c")])
    return _HOST_SO


def build_dev(force: bool = False) -> str:
    if force or _stale(_DEV_SO, "msgen_dev.cu"):
        subprocess.check_call(["nvcc", "-O3", "-shared", "-Xcompiler", "-fPIC",
                               "-gencode", "arch=compute_103a,code=sm_103a",
                               "-o", _DEV_SO, os.path.join(_HERE, "msgen_dev.cu")])
    return _DEV_SO


_host = None
_dev = None


def _lib():
    global _host
    if _host is None:
        lib = ctypes.CDLL(build_host())
        lib.msgen_mix64.restype = _u64
        lib.msgen_mix64.argtypes = [_u64]
        lib.msgen_draw.restype = _u64
        lib.msgen_draw.argtypes = [_u64, _u64]
        lib.msgen_thr24.restype = _u32
        lib.msgen_thr24.argtypes = [ctypes.c_double]
        lib.msgen_fill_u8.argtypes = [_vp, _i64, _i64, _i64, _u64, _u32]
        lib.msgen_fill_u8_rows.argtypes = [_vp, _i64, _i64, _i64, _i64, _u64, _u32]
        lib.msgen_plant_pos.argtypes = [_u64, _i64, _i64, _i64, ctypes.POINTER(_i64),
                                        ctypes.POINTER(_i64)]
        lib.msgen_plant_u8.argtypes = [_vp, _i64, _i64, _i64, _i64]
        lib.msgen_pack_bits.argtypes = [_vp, _i64, _i64, _i64, _vp, _i64, ctypes.c_int]
        lib.msgen_unpack_bits.argtypes = [_vp, _i64, _i64, _i64, _vp, _i64]
        _host = lib
    return _host


def _dlib():
    global _dev
    if _dev is None:
        lib = ctypes.CDLL(build_dev())
        lib.msgen_fill_u8_dev.argtypes = [_vp, _i64, _i64, _i64, _u64, _u32, _vp]
        lib.msgen_fill_bits_dev.argtypes = [_vp, _i64, _i64, _i64, _u64, _u32, ctypes.c_int, _vp]
        lib.msgen_plant_u8_dev.argtypes = [_vp, _i64, _i64, _i64, _i64, _vp]
        lib.msgen_plant_bits_dev.argtypes = [_vp, _i64, _i64, _i64, _i64, _vp]
        _dev = lib
    return _dev


def mix64(z: int) -> int:
    return int(_lib().msgen_mix64(z))


def draw(seed: int, k: int) -> int:
    return int(_lib().msgen_draw(seed, k))


def thr24(p: float) -> int:
    return int(_lib().msgen_thr24(p))


def bernoulli_u8(m: int, n: int, p: float, seed: int, ld: int | None = None,
                 threads: int = 1) -> np.ndarray:
    """m x n uint8 0/1 matrix (as an m x ld array whose first n columns are the cells).
    threads > 1 fills disjoint row ranges concurrently (same cells)."""
    ld = n if ld is None else ld
    out = np.zeros((m, max(ld, 1)), dtype=np.uint8)
    if m <= 0 or n <= 0:
        return out
    t = thr24(p)
    if threads <= 1 or m < 2 * threads:
        _lib().msgen_fill_u8(out.ctypes.data, m, n, ld, seed, t)
        return out
    import concurrent.futures as cf
    lib, base = _lib(), out.ctypes.data
    step = (m + threads - 1) // threads
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:  # ctypes drops the GIL
        list(ex.map(lambda r0: lib.msgen_fill_u8_rows(base + r0 * ld, r0, min(m, r0 + step),
                                                      n, ld, seed, t),
                    range(0, m, step)))
    return out


def config_u8(spec: dict, threads: int = 1) -> np.ndarray:
    """The uint8 matrix of a workload recipe (see ``gen.configs``): Bernoulli
    cells plus the planted square, if any."""
    a = bernoulli_u8(spec["m"], spec["n"], spec["p"], spec["seed"], threads=threads)
    if spec.get("plant"):
        r, c = plant_pos(spec["seed"], spec["m"], spec["n"], spec["plant"])
        a[r:r + spec["plant"], c:c + spec["plant"]] = 1
    return a


def plant_pos(seed: int, m: int, n: int, s: int) -> tuple[int, int]:
    r, c = _i64(), _i64()
    _lib().msgen_plant_pos(seed, m, n, s, ctypes.byref(r), ctypes.byref(c))
    return int(r.value), int(c.value)


def plant_u8(a: np.ndarray, r: int, c: int, s: int) -> None:
    assert a.dtype == np.uint8 and a.flags.c_contiguous
    a[r:r + s, c:c + s] = 1


def pack_bits(a: np.ndarray, n: int, ldw: int | None = None, pad_value: int = 0) -> np.ndarray:
    """Pack the first n columns of a C-contiguous uint8 matrix into MS_BITS32 rows."""
    a = np.ascontiguousarray(a, dtype=np.uint8)
    m = a.shape[0]
    ldw = (n + 31) // 32 if ldw is None else ldw
    out = np.zeros((m, max(ldw, 1)), dtype=np.uint32)
    if m > 0 and ldw > 0:
        _lib().msgen_pack_bits(a.ctypes.data, m, n, a.shape[1], out.ctypes.data, ldw,
                               int(pad_value))
    return out


def unpack_bits(w: np.ndarray, m: int, n: int) -> np.ndarray:
    w = np.ascontiguousarray(w, dtype=np.uint32)
    out = np.zeros((m, max(n, 1)), dtype=np.uint8)
    if m > 0 and n > 0:
        _lib().msgen_unpack_bits(w.ctypes.data, m, n, w.shape[1], out.ctypes.data, out.shape[1])
    return out[:, :n]


# ---- device-side fills (raw device pointers, stream handle as int) ----

def fill_u8_dev(ptr: int, m: int, n: int, ld: int, p: float, seed: int, stream: int = 0) -> None:
    rc = _dlib().msgen_fill_u8_dev(ptr, m, n, ld, seed, thr24(p), stream)
    if rc:
        raise RuntimeError(f"msgen_fill_u8_dev failed: cuda error {rc}")


def fill_bits_dev(ptr: int, m: int, n: int, ldw: int, p: float, seed: int, pad_value: int = 0,
                  stream: int = 0) -> None:
    rc = _dlib().msgen_fill_bits_dev(ptr, m, n, ldw, seed, thr24(p), int(pad_value), stream)
    if rc:
        raise RuntimeError(f"msgen_fill_bits_dev failed: cuda error {rc}")


def plant_u8_dev(ptr: int, ld: int, r: int, c: int, s: int, stream: int = 0) -> None:
    rc = _dlib().msgen_plant_u8_dev(ptr, ld, r, c, s, stream)
    if rc:
        raise RuntimeError(f"msgen_plant_u8_dev failed: cuda error {rc}")


def plant_bits_dev(ptr: int, ldw: int, r: int, c: int, s: int, stream: int = 0) -> None:
    rc = _dlib().msgen_plant_bits_dev(ptr, ldw, r, c, s, stream)
    if rc:
        raise RuntimeError(f"msgen_plant_bits_dev failed: cuda error {rc}")
