"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/tsvdm.h declares; host-side argument checks that need no GPU."""
import ctypes
import os
import re

import pytest

from paper_2605_16058_gb300 import build, native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "tsvdm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tsvdm_[a-z_0-9]+)\s*\(", src)))


def test_library_builds_and_exports_every_declared_symbol():
    path = build.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(native.SIGNATURES), set(names) ^ set(native.SIGNATURES)


def test_host_argument_checks_need_no_gpu():
    L = native.lib()
    h = ctypes.c_void_p()
    assert L.tsvdm_plan_create(0, 4, 4, native.F32, native.P_FP32, 1, None, ctypes.byref(h)) == native.EINVAL
    assert L.tsvdm_plan_create(4, 4, 4, native.F64, native.P_FP32, 1, None, ctypes.byref(h)) == native.ENOTSUP
    assert L.tsvdm_plan_create(4, 4, 4, 7, native.P_FP32, 1, None, ctypes.byref(h)) == native.EINVAL
    assert L.tsvdm_plan_create(4, 4, 4, native.F32, native.P_FP32, 1, None, None) == native.EINVAL
    assert L.tsvdm_fixed_rank(None, None, None, 1, None, None, None, 0, None) == native.EINVAL
    assert L.tsvdm_plan_destroy(None) == native.EINVAL
    assert L.tsvdm_adam(0, native.F32, None, None, None, None, 1, 1e-3, 0.9, 0.999, 1e-8, None) == native.EINVAL
    assert L.tsvdm_strerror(native.ECAPACITY).decode() == "output capacity below the total rank"


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(native, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(native, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        native.lib()
