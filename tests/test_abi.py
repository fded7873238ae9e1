"""CPU-side checks of the C ABI: the library builds, loads without a GPU, exports
every symbol include/dctplus.h declares, and rejects bad arguments on the host."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2409_08970_gb300 import build, _lib
    build.build()
    return _lib.load()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "dctplus.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dctplus_\w+)\s*\(", text)))


def test_header_declarations_are_exported(lib):
    names = declared_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name
    from paper_2409_08970_gb300 import _lib
    assert sorted(_lib.EXPORTS) == names


def test_exports_via_nm(lib):
    from paper_2409_08970_gb300 import _lib
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.LIB_PATH], capture_output=True,
                         text=True).stdout
    for name in declared_functions():
        assert re.search(rf"\bT {name}\b", out), name


def test_status_strings(lib):
    for code in range(9):
        s = lib.dctplus_status_string(code)
        assert s and s != b"unknown status"
    assert lib.dctplus_status_string(99) == b"unknown status"


def _has_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def test_plan_argument_errors_before_any_device_work(lib):
    from paper_2409_08970_gb300 import _lib
    h = ctypes.c_void_p()
    v = np.zeros(8)
    ptr = v.ctypes.data
    assert lib.dctplus_plan(None, 8, ptr, 1.0, None) == _lib.ERR_INVALID_ARG
    assert lib.dctplus_plan(ctypes.byref(h), 1, ptr, 1.0, None) == _lib.ERR_INVALID_ARG
    assert lib.dctplus_plan(ctypes.byref(h), 16385, ptr, 1.0, None) == _lib.ERR_INVALID_ARG
    assert lib.dctplus_plan(ctypes.byref(h), 8, None, 1.0, None) == _lib.ERR_INVALID_ARG
    assert lib.dctplus_plan(ctypes.byref(h), 8, ptr, float("nan"), None) == _lib.ERR_INVALID_ARG
    v[3] = float("inf")
    assert lib.dctplus_plan(ctypes.byref(h), 8, ptr, 1.0, None) == _lib.ERR_INVALID_ARG
    bad = _lib.Opts(7, 0, 0, -1)
    v[3] = 0.0
    assert lib.dctplus_plan(ctypes.byref(h), 8, ptr, 1.0, ctypes.byref(bad)) == _lib.ERR_INVALID_ARG
    assert h.value is None


def test_execute_argument_errors(lib):
    from paper_2409_08970_gb300 import _lib
    assert lib.dctplus_execute(None, 0, None, 8, None, 8, 1, None) == _lib.ERR_INVALID_ARG
    assert lib.dctplus_execute_host(None, 0, None, None, 1, None) == _lib.ERR_INVALID_ARG
    assert lib.dctplus_group_create(None, 1, None) == _lib.ERR_INVALID_ARG
    g = ctypes.c_void_p()
    assert lib.dctplus_group_create(ctypes.byref(g), 0, None) == _lib.ERR_INVALID_ARG
    assert lib.dctplus_execute_group(None, None, None, None, 0, None) == _lib.ERR_INVALID_ARG
    assert lib.dctplus_plan_size(None) == -1


@pytest.mark.skipif(_has_gpu(), reason="checks the no-device path")
def test_no_device_is_reported(lib):
    from paper_2409_08970_gb300 import _lib
    h = ctypes.c_void_p()
    v = np.zeros(8)
    v[0] = 1
    assert lib.dctplus_plan(ctypes.byref(h), 8, v.ctypes.data, 1.0, None) == _lib.ERR_NO_DEVICE


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    import paper_2409_08970_gb300._lib as L
    monkeypatch.setattr(L, "_lib", None)
    monkeypatch.setattr(L, "LIB_PATH", str(tmp_path / "absent.so"))
    with pytest.raises(RuntimeError, match="missing"):
        L.load()


def test_product_never_imports_oracle():
    pkg = os.path.join(ROOT, "paper_2409_08970_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle\b", src, re.M), f
                assert "synthetic" not in re.findall(r"^\s*(?:from|import)\s+(\w+)", src, re.M), f
    for dirpath, _, files in os.walk(os.path.join(ROOT, "oracle")):
        for f in files:
            if f.endswith(".py"):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+paper_2409_08970_gb300\b", src, re.M), f
