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


def test_newer_entry_points_check_arguments_before_any_device_work():
    """Engine choice, warm start, Jacobi settings, data-driven transform, d-way plans,
    batches and the allocation-free selection reject bad arguments on the host."""
    L = native.lib()
    h = ctypes.c_void_p()
    assert L.tsvdm_plan_set_engine(None, native.JACOBI_TC) == native.EINVAL
    assert L.tsvdm_plan_set_warm_start(None, 1) == native.EINVAL
    assert L.tsvdm_plan_set_jacobi(None, 0.0, 10) == native.EINVAL
    assert L.tsvdm_data_transform(None, None, None) == native.EINVAL
    assert L.tsvdm_transform(None, None, None, 0, None) == native.EINVAL
    assert L.tsvdm_tolerance(None, None, None, 0.1, None, None, None, None, None, 0, None,
                             None) == native.EINVAL
    assert L.tsvdm_reconstruct(None, None, None, None, None, 1, None, None) == native.EINVAL
    assert L.tsvdm_backward(None, None, None, 1, None, None, None, 1.0, None, None,
                            None) == native.EINVAL
    # d-way plans: order 3..8, every mode positive
    for dims in [(4, 4), (2,) * 9, (4, 4, 0), (4, 4, 3, -1)]:
        arr = (ctypes.c_int64 * len(dims))(*dims)
        assert L.tsvdm_plan_create_dway(len(dims), arr, native.F32, native.P_FP32, 1, None,
                                        ctypes.byref(h)) == native.EINVAL, dims
    assert L.tsvdm_plan_create_dway(3, None, native.F32, native.P_FP32, 1, None,
                                    ctypes.byref(h)) == native.EINVAL
    b = ctypes.c_void_p()
    desc = native.BatchDesc(8, 8, 4, 0, 2, 0.0)
    assert L.tsvdm_batch_create(None, 1, native.F32, native.P_FP32, None,
                                ctypes.byref(b)) == native.EINVAL
    assert L.tsvdm_batch_create(ctypes.byref(desc), 0, native.F32, native.P_FP32, None,
                                ctypes.byref(b)) == native.EINVAL
    assert L.tsvdm_batch_create(ctypes.byref(desc), 1, native.F64, native.P_FP32, None,
                                ctypes.byref(b)) == native.ENOTSUP
    assert L.tsvdm_batch_graph_kernels(None, None) == native.EINVAL
    # allocation-free selection: eps in (0, 1) and the size limit are checked first (the
    # host buffers below are never read)
    sig = (ctypes.c_float * 4)()
    rk = (ctypes.c_int32 * 4)()
    off = (ctypes.c_int64 * 5)()
    vp = lambda a: ctypes.cast(a, ctypes.c_void_p)
    for eps in (0.0, 1.0, 1.5, -0.1):
        assert L.tsvdm_select_ranks_noalloc(vp(sig), 4, 1, eps, vp(rk), vp(off), None,
                                            None) == native.EINVAL, eps
    assert L.tsvdm_select_ranks_noalloc(None, 4, 1, 0.1, vp(rk), vp(off), None,
                                        None) == native.EINVAL
    assert L.tsvdm_select_ranks_noalloc(vp(sig), 1024, 300, 0.1, vp(rk), vp(off), None,
                                        None) == native.ESCRATCH


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(native, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(native, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        native.lib()
