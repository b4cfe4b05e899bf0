"""The C-ABI library builds, loads without a GPU and exports every symbol that
include/*.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for fn in os.listdir(inc):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(inc, fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(?:ms_status|const char\s*\*|void|int)\s+(ms_\w+)\s*\(", src):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def libms():
    import paper_2503_18974_gb300 as ms
    ms.build()
    return ctypes.CDLL(ms.LIB_PATH)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("ms_create", "ms_max_square", "ms_dp_map", "ms_batch", "ms_destroy",
                     "ms_status_string"):
        assert required in names


def test_library_exports_every_declared_symbol(libms):
    missing = [n for n in sorted(declared_functions()) if not hasattr(libms, n)]
    assert not missing, missing


def test_status_strings_without_gpu(libms):
    libms.ms_status_string.restype = ctypes.c_char_p
    assert libms.ms_status_string(0) == b"MS_OK"
    assert b"TIMEOUT" in libms.ms_status_string(4)
    assert libms.ms_status_string(99) == b"unknown ms_status"


def test_null_arguments_rejected_without_gpu(libms):
    # argument checks run before any device call
    libms.ms_max_square.restype = ctypes.c_int
    libms.ms_max_square.argtypes = [ctypes.c_void_p] * 4
    assert libms.ms_max_square(None, None, None, None) == 1
    libms.ms_destroy.restype = ctypes.c_int
    libms.ms_destroy.argtypes = [ctypes.c_void_p]
    assert libms.ms_destroy(None) == 1
    libms.ms_all_max_squares.restype = ctypes.c_int
    libms.ms_all_max_squares.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int64] + \
        [ctypes.c_void_p] * 3
    assert libms.ms_all_max_squares(None, None, None, 0, None, None, None) == 1


def test_python_binding_imports_and_fails_loudly_without_library(tmp_path, monkeypatch):
    import paper_2503_18974_gb300 as ms
    monkeypatch.setattr(ms, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(ms, "_lib", None)
    with pytest.raises(ImportError):
        ms.lib()
