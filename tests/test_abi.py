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


def test_binding_structures_match_the_header(tmp_path):
    """Every structure the binding passes across the C ABI has the header's
    size and field offsets (compiled from include/ms.h with the host C
    compiler, so that an edit of one side without the other fails here)."""
    import shutil
    import subprocess

    import paper_2503_18974_gb300 as ms
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    pairs = {"ms_matrix": ms._Matrix, "ms_result": ms._Result, "ms_tuning": ms._Tuning,
             "ms_profile": ms.Profile, "ms_server_config": ms.ServerConfig,
             "ms_server_completion": ms.Completion, "ms_server_stats": ms.ServerStats,
             "ms_volume": ms._Volume}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "ms.h"', "int main(void) {"]
    for cname, py in pairs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "abi.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "abi"
    subprocess.check_call([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                           str(exe)])
    got = {}
    for line in subprocess.check_output([str(exe)], text=True).splitlines():
        cname, key, val = line.split()
        got[(cname, key)] = int(val)
    for cname, py in pairs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)
