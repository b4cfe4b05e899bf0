"""Maximal all-ones square detection on GB300: Python binding of libms.

Argument marshalling only.  Every step of the computation runs in the CUDA
kernels of ``libms.so`` (built from ``csrc/``); PyTorch supplies device
memory and streams.  There is no CPU fallback: if the library is missing or
was built for another machine, importing the binding raises.

Results are int32 device tensors ``[side, row, col, status]``: the largest
all-ones square side, the bottom-right corner of the first such square in
row-major order (-1, -1 when side == 0) and an ``ms_status`` code.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Iterable, Sequence

_HERE = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_HERE)
LIB_PATH = os.path.join(_HERE, "libms.so")
_SOURCES = [os.path.join(_HERE, "csrc", f) for f in ("ms.cu", "ms_noalloc.cu", "ms_serve.cu",
                                                      "ms_cube.cu", "ms_kernels.cuh",
                                                      "ms_device.cuh", "ms_bits.cuh",
                                                      "ms_bitile.cuh")]
_UNITS = [os.path.join(_HERE, "csrc", f) for f in ("ms.cu", "ms_noalloc.cu", "ms_serve.cu",
                                                    "ms_cube.cu")]
_HEADER = os.path.join(_ROOT, "include", "ms.h")

MS_U8 = 0
MS_BITS32 = 1
STATUS = {0: "MS_OK", 1: "MS_ERR_INVALID", 2: "MS_ERR_OOM", 3: "MS_ERR_CUDA",
          4: "MS_ERR_TIMEOUT", 5: "MS_ERR_BUDGET", 6: "MS_ERR_UNSUPPORTED",
          7: "MS_ERR_CANCELLED"}

NVCC_FLAGS = ["-O3", "-std=c++17", "-shared", "-Xcompiler", "-fPIC",
              "-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo", "--threads", "4"]


class MSError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {STATUS.get(code, code)}")
        self.code = code


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libms.so in-tree for sm_103a (nvcc cross-compiles without a GPU)."""
    srcs = [p for p in _SOURCES + [_HEADER] if os.path.exists(p)]
    stale = force or not os.path.exists(LIB_PATH) or any(
        os.path.getmtime(p) > os.path.getmtime(LIB_PATH) for p in srcs)
    if stale:
        cmd = ["nvcc", *NVCC_FLAGS, "-o", LIB_PATH, *_UNITS]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        subprocess.check_call(cmd)
    return LIB_PATH


class _Volume(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("d", ctypes.c_int64), ("m", ctypes.c_int64),
                ("n", ctypes.c_int64), ("ld", ctypes.c_int64), ("ld_slice", ctypes.c_int64),
                ("fmt", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class _Matrix(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("m", ctypes.c_int64), ("n", ctypes.c_int64),
                ("ld", ctypes.c_int64), ("fmt", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class _Tuning(ctypes.Structure):
    _fields_ = [("band_rows", ctypes.c_int32), ("packed_path", ctypes.c_int32),
                ("test_hold_carries", ctypes.c_int32), ("lane_cols", ctypes.c_int32),
                ("tile_kind", ctypes.c_int32), ("reserved", ctypes.c_int32 * 3)]


class Profile(ctypes.Structure):
    _fields_ = [("tile_launches", ctypes.c_int64), ("tile_ms", ctypes.c_double),
                ("fixup_launches", ctypes.c_int64), ("fixup_ms", ctypes.c_double),
                ("other_launches", ctypes.c_int64), ("other_ms", ctypes.c_double),
                ("untimed_launches", ctypes.c_int64), ("bit_tile_launches", ctypes.c_int64)]


class _Result(ctypes.Structure):
    _fields_ = [("side", ctypes.c_int32), ("row", ctypes.c_int32), ("col", ctypes.c_int32),
                ("status", ctypes.c_int32)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("memory_budget_bytes", ctypes.c_size_t), ("streams", ctypes.c_int32),
                ("max_batch", ctypes.c_int32), ("test_fail_batch", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 3)]


class Completion(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("result", _Result), ("t_submit", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_launch", ctypes.c_double),
                ("t_done", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("batches", ctypes.c_int64), ("peak_bytes", ctypes.c_int64),
                ("peak_inflight", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("host_batch_s", ctypes.c_double), ("host_copy_s", ctypes.c_double)]


_lib = None

EXPORTS = ("ms_create", "ms_destroy", "ms_max_square", "ms_dp_map", "ms_all_max_squares",
           "ms_max_cube", "ms_batch",
           "ms_status_string", "ms_set_tuning", "ms_get_tuning", "ms_profile_start",
           "ms_profile_stop", "ms_autotune", "ms_max_square_noalloc", "ms_server_create",
           "ms_server_submit", "ms_server_poll", "ms_server_cancel", "ms_server_wait_all",
           "ms_server_stats_get",
           "ms_server_destroy", "ms_server_now")


def lib():
    """Load libms.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libms.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i64 = ctypes.c_void_p, ctypes.c_int64
        L.ms_create.restype = ctypes.c_int
        L.ms_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_size_t]
        L.ms_destroy.restype = ctypes.c_int
        L.ms_destroy.argtypes = [vp]
        L.ms_max_square.restype = ctypes.c_int
        L.ms_max_square.argtypes = [vp, ctypes.POINTER(_Matrix), vp, vp]
        L.ms_dp_map.restype = ctypes.c_int
        L.ms_dp_map.argtypes = [vp, ctypes.POINTER(_Matrix), vp, i64, vp, vp]
        L.ms_max_cube.restype = ctypes.c_int
        L.ms_max_cube.argtypes = [vp, ctypes.POINTER(_Volume), vp, vp]
        L.ms_all_max_squares.restype = ctypes.c_int
        L.ms_all_max_squares.argtypes = [vp, ctypes.POINTER(_Matrix), vp, i64, vp, vp, vp]
        L.ms_batch.restype = ctypes.c_int
        L.ms_batch.argtypes = [vp, ctypes.POINTER(_Matrix), ctypes.c_int32, vp, vp]
        L.ms_status_string.restype = ctypes.c_char_p
        L.ms_status_string.argtypes = [ctypes.c_int]
        L.ms_set_tuning.restype = ctypes.c_int
        L.ms_set_tuning.argtypes = [vp, ctypes.POINTER(_Tuning)]
        L.ms_get_tuning.restype = ctypes.c_int
        L.ms_get_tuning.argtypes = [vp, ctypes.POINTER(_Tuning)]
        L.ms_server_create.restype = ctypes.c_int
        L.ms_server_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int,
                                       ctypes.POINTER(ServerConfig)]
        L.ms_server_submit.restype = ctypes.c_int
        L.ms_server_submit.argtypes = [vp, ctypes.POINTER(_Matrix), ctypes.c_double,
                                       ctypes.POINTER(ctypes.c_uint64)]
        L.ms_server_poll.restype = ctypes.c_int
        L.ms_server_poll.argtypes = [vp, ctypes.POINTER(Completion), ctypes.c_int32,
                                     ctypes.POINTER(ctypes.c_int32)]
        L.ms_server_wait_all.restype = ctypes.c_int
        L.ms_server_wait_all.argtypes = [vp]
        L.ms_server_cancel.restype = ctypes.c_int
        L.ms_server_cancel.argtypes = [vp, ctypes.c_uint64]
        L.ms_server_stats_get.restype = ctypes.c_int
        L.ms_server_stats_get.argtypes = [vp, ctypes.POINTER(ServerStats)]
        L.ms_server_destroy.restype = ctypes.c_int
        L.ms_server_destroy.argtypes = [vp]
        L.ms_server_now.restype = ctypes.c_double
        L.ms_server_now.argtypes = []
        L.ms_autotune.restype = ctypes.c_int
        L.ms_autotune.argtypes = [vp, ctypes.POINTER(_Matrix), ctypes.c_int32, vp, vp,
                                  ctypes.POINTER(_Tuning)]
        L.ms_profile_start.restype = ctypes.c_int
        L.ms_profile_start.argtypes = [vp, ctypes.c_int32]
        L.ms_profile_stop.restype = ctypes.c_int
        L.ms_profile_stop.argtypes = [vp, ctypes.POINTER(Profile)]
        _lib = L
    return _lib


def _check(code: int, what: str) -> None:
    if code != 0:
        raise MSError(code, what)


def describe(x, n: int | None = None, fmt: int | None = None) -> _Matrix:
    """ms_matrix for a 2-D CUDA tensor: uint8 cells (MS_U8) or 32-bit words of
    packed bits (MS_BITS32, n = number of columns required)."""
    import torch
    if x.dim() != 2 or x.stride(1) != 1:
        raise ValueError("expected a 2-D tensor with unit column stride")
    if fmt is None:
        fmt = MS_U8 if x.dtype == torch.uint8 else MS_BITS32
    if fmt == MS_U8:
        if x.dtype != torch.uint8:
            raise ValueError("MS_U8 expects a uint8 tensor")
        n = x.shape[1] if n is None else n
    else:
        if x.dtype not in (torch.int32, torch.uint32):
            raise ValueError("MS_BITS32 expects an int32/uint32 tensor of packed words")
        if n is None:
            raise ValueError("MS_BITS32 needs the column count n")
    ld = x.stride(0) if x.shape[0] > 1 else max(x.shape[1], 1)
    return _Matrix(x.data_ptr(), x.shape[0], n, ld, fmt, 0)


def _stream_ptr(stream) -> int | None:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream or None


class MaxSquare:
    """A libms context on one device."""

    def __init__(self, device: int = 0, workspace_budget: int = 0):
        self.device = device
        h = ctypes.c_void_p()
        _check(lib().ms_create(ctypes.byref(h), device, workspace_budget), "ms_create")
        self._h = h

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().ms_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_tuning(self, band_rows: int = 0, packed_path: int = 0,
                   test_hold_carries: int = 0, lane_cols: int = 0, tile_kind: int = 0) -> None:
        t = _Tuning(band_rows, packed_path, test_hold_carries, lane_cols, tile_kind)
        _check(lib().ms_set_tuning(self._h, ctypes.byref(t)), "ms_set_tuning")

    def profile_start(self, max_launches: int = 1 << 20) -> None:
        _check(lib().ms_profile_start(self._h, max_launches), "ms_profile_start")

    def profile_stop(self) -> Profile:
        p = Profile()
        _check(lib().ms_profile_stop(self._h, ctypes.byref(p)), "ms_profile_stop")
        return p

    def autotune(self, mats: Sequence, stream=None) -> dict:
        """Time candidate tunings on these matrices (one: the ms_max_square path;
        several: ms_batch) and cache the fastest for their workload class."""
        import torch
        descs = (_Matrix * len(mats))()
        dev = None
        for i, item in enumerate(mats):
            descs[i] = describe(*item) if isinstance(item, tuple) else describe(item)
            dev = (item[0] if isinstance(item, tuple) else item).device
        out = torch.empty((len(mats), 4), dtype=torch.int32, device=dev)
        t = _Tuning()
        _check(lib().ms_autotune(self._h, descs, len(mats), out.data_ptr(), _stream_ptr(stream),
                                 ctypes.byref(t)), "ms_autotune")
        return {"band_rows": t.band_rows, "packed_path": t.packed_path,
                "lane_cols": t.lane_cols, "tile_kind": t.tile_kind}

    def get_tuning(self) -> dict:
        t = _Tuning()
        _check(lib().ms_get_tuning(self._h, ctypes.byref(t)), "ms_get_tuning")
        return {"band_rows": t.band_rows, "packed_path": t.packed_path,
                "lane_cols": t.lane_cols, "tile_kind": t.tile_kind}

    def max_square(self, x, n: int | None = None, fmt: int | None = None, out=None, stream=None):
        import torch
        desc = describe(x, n, fmt)
        if out is None:
            out = torch.empty(4, dtype=torch.int32, device=x.device)
        _check(lib().ms_max_square(self._h, ctypes.byref(desc), out.data_ptr(),
                                   _stream_ptr(stream)), "ms_max_square")
        return out

    def max_cube(self, v, stream=None):
        """Largest all-ones cube of a (d, m, n) uint8 CUDA tensor with unit
        column stride.  Returns an int32 tensor [side, slice, row, col,
        status, 0] (the call waits for the stream)."""
        import torch
        if v.dim() != 3 or v.dtype != torch.uint8 or (v.numel() and v.stride(2) != 1):
            raise ValueError("expected a 3-D uint8 tensor with unit column stride")
        d, m, n = v.shape
        desc = _Volume(v.data_ptr() if v.numel() else None, d, m, n,
                       v.stride(1) if m > 1 else max(n, 1),
                       v.stride(0) if d > 1 else max(m * (v.stride(1) if m > 1 else n), 1),
                       MS_U8, 0)
        out = torch.empty(6, dtype=torch.int32, device=v.device)
        _check(lib().ms_max_cube(self._h, ctypes.byref(desc), out.data_ptr(),
                                 _stream_ptr(stream)), "ms_max_cube")
        return out

    def all_max_squares(self, x, n: int | None = None, fmt: int | None = None,
                        capacity: int = 1024, stream=None):
        """Every bottom-right corner of a largest all-ones square.  Returns
        (result tensor [side, row, col, status], int32 (count, 2) corners, in
        unspecified order).  Calls again with room for all of them when the
        first capacity was too small."""
        import torch
        desc = describe(x, n, fmt)
        out = torch.empty(4, dtype=torch.int32, device=x.device)
        count = torch.zeros(1, dtype=torch.int64, device=x.device)
        while True:
            corners = torch.empty((max(capacity, 1), 2), dtype=torch.int32, device=x.device)
            _check(lib().ms_all_max_squares(self._h, ctypes.byref(desc), corners.data_ptr(),
                                            capacity, count.data_ptr(), out.data_ptr(),
                                            _stream_ptr(stream)), "ms_all_max_squares")
            c = int(count.item())
            if c <= capacity:
                return out, corners[:c]
            capacity = c

    def dp_map(self, x, n: int | None = None, fmt: int | None = None, dp=None, out=None,
               stream=None):
        import torch
        desc = describe(x, n, fmt)
        if dp is None:
            dp = torch.empty((desc.m, desc.n), dtype=torch.int32, device=x.device)
        if out is None:
            out = torch.empty(4, dtype=torch.int32, device=x.device)
        ld_dp = dp.stride(0) if dp.dim() == 2 and dp.shape[0] > 1 else max(desc.n, 1)
        _check(lib().ms_dp_map(self._h, ctypes.byref(desc), dp.data_ptr(), ld_dp, out.data_ptr(),
                               _stream_ptr(stream)), "ms_dp_map")
        return dp, out

    def batch(self, mats: Sequence, out=None, stream=None):
        """mats: tensors (uint8) or (tensor, n) / (tensor, n, fmt) tuples."""
        import torch
        descs = (_Matrix * max(len(mats), 1))()
        dev = None
        for i, item in enumerate(mats):
            if isinstance(item, tuple):
                descs[i] = describe(*item)
                dev = item[0].device
            else:
                descs[i] = describe(item)
                dev = item.device
        if out is None:
            out = torch.empty((len(mats), 4), dtype=torch.int32,
                              device=dev if dev is not None else f"cuda:{self.device}")
        _check(lib().ms_batch(self._h, descs, len(mats), out.data_ptr(), _stream_ptr(stream)),
               "ms_batch")
        return out

    def batch_descs(self, descs, count: int, out, stream=None):
        """ms_batch on a prepared ctypes array of ms_matrix (no per-call marshalling)."""
        _check(lib().ms_batch(self._h, descs, count, out.data_ptr(), _stream_ptr(stream)),
               "ms_batch")
        return out


def status_string(code: int) -> str:
    return lib().ms_status_string(code).decode()


def host_describe(a, n: int | None = None, fmt: int | None = None) -> _Matrix:
    """ms_matrix for a 2-D host (numpy or CPU torch) array: uint8 cells or packed words."""
    import numpy as np
    arr = a.numpy() if hasattr(a, "numpy") else a
    if arr.ndim != 2 or arr.strides[1] != arr.itemsize:
        raise ValueError("expected a 2-D array with unit column stride")
    if fmt is None:
        fmt = MS_U8 if arr.dtype == np.uint8 else MS_BITS32
    if fmt == MS_U8:
        n = arr.shape[1] if n is None else n
    elif n is None:
        raise ValueError("MS_BITS32 needs the column count n")
    ld = arr.strides[0] // arr.itemsize if arr.shape[0] > 1 else max(arr.shape[1], 1)
    return _Matrix(arr.ctypes.data, arr.shape[0], n, ld, fmt, 0)


class Server:
    """The libms request server (admission by memory budget, continuous batching)."""

    def __init__(self, device: int = 0, memory_budget: int = 16 << 30, streams: int = 2,
                 max_batch: int = 512, test_fail_batch: int = 0):
        cfg = ServerConfig(memory_budget, streams, max_batch, test_fail_batch)
        h = ctypes.c_void_p()
        _check(lib().ms_server_create(ctypes.byref(h), device, ctypes.byref(cfg)),
               "ms_server_create")
        self._h = h
        self._keep = {}
        self._rid = ctypes.c_uint64()

    def submit(self, a, n: int | None = None, fmt: int | None = None, t_arrival: float = -1.0,
               keep=None) -> int:
        """Submit a host matrix; it must stay alive until its completion is polled
        (pass keep= to have the server object hold a reference)."""
        desc = host_describe(a, n, fmt)
        rid = ctypes.c_uint64()
        _check(lib().ms_server_submit(self._h, ctypes.byref(desc), t_arrival, ctypes.byref(rid)),
               "ms_server_submit")
        self._keep[rid.value] = a if keep is None else keep
        return rid.value

    def submit_desc(self, desc: "_Matrix", t_arrival: float = -1.0) -> int:
        """Submit a prebuilt descriptor (from host_describe) whose host memory
        the caller keeps alive until completion: the low-overhead path for
        load generators."""
        rid = self._rid
        _check(lib().ms_server_submit(self._h, ctypes.byref(desc), t_arrival, ctypes.byref(rid)),
               "ms_server_submit")
        return rid.value

    def poll(self, max_n: int = 4096) -> list:
        buf = (Completion * max_n)()
        n = ctypes.c_int32()
        _check(lib().ms_server_poll(self._h, buf, max_n, ctypes.byref(n)), "ms_server_poll")
        out = []
        for k in range(n.value):
            c = buf[k]
            self._keep.pop(c.id, None)
            out.append({"id": c.id, "result": [c.result.side, c.result.row, c.result.col,
                                               c.result.status],
                        "t_submit": c.t_submit, "t_admit": c.t_admit, "t_launch": c.t_launch,
                        "t_done": c.t_done})
        return out

    def cancel(self, rid: int) -> int:
        """Withdraw a request still waiting for admission; returns the status
        code (0: cancelled, 1: unknown or already admitted)."""
        return lib().ms_server_cancel(self._h, rid)

    def wait_all(self) -> None:
        _check(lib().ms_server_wait_all(self._h), "ms_server_wait_all")

    def stats(self) -> dict:
        st = ServerStats()
        _check(lib().ms_server_stats_get(self._h, ctypes.byref(st)), "ms_server_stats_get")
        return {k: getattr(st, k) for k in ("submitted", "completed", "batches", "peak_bytes",
                                            "peak_inflight", "host_batch_s", "host_copy_s")}

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().ms_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def now() -> float:
    return lib().ms_server_now()
