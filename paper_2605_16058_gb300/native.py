"""ctypes binding of libtsvdm.so (include/tsvdm.h), same names as the C entry points.

Argument marshalling only: tensors are passed by data pointer, every computation runs in
the library's CUDA kernels.  Loading fails loudly when the library has not been built
(there is no CPU fallback).  PyTorch is used for device memory and streams.
"""
from __future__ import annotations

import ctypes
import math
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libtsvdm.so")

OK, EINVAL, ENOTORTHO, ENOCONV, ENONFINITE, ETIMEOUT, ENOMEM, ECAPACITY, ECUDA, ENOTSUP, ESCRATCH = range(11)
F32, F64 = 0, 1
P_FP64, P_FP32, P_TF32, P_BF16X3 = 0, 1, 2, 3
PRECISIONS = {"fp64": P_FP64, "fp32": P_FP32, "tf32": P_TF32, "bf16x3": P_BF16X3}
JACOBI_AUTO, JACOBI_FMA, JACOBI_TC = 0, 1, 2
ENGINES = {"auto": JACOBI_AUTO, "fma": JACOBI_FMA, "tc": JACOBI_TC}
ANGLE_FP64, ANGLE_FP32 = 0, 1
ANGLES = {"fp64": ANGLE_FP64, "fp32": ANGLE_FP32}

# every symbol include/tsvdm.h declares, with (restype, argtypes)
_i64, _i32, _dbl, _vp = ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
_pi64, _pdbl = ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)
SIGNATURES = {
    "tsvdm_plan_create": (_i32, [_i64, _i64, _i64, _i32, _i32, _i32, _vp, ctypes.POINTER(_vp)]),
    "tsvdm_plan_destroy": (_i32, [_vp]),
    "tsvdm_plan_create_dway": (_i32, [_i32, ctypes.POINTER(_i64), _i32, _i32, _i32, _vp,
                                      ctypes.POINTER(_vp)]),
    "tsvdm_plan_set_jacobi": (_i32, [_vp, _dbl, _i32]),
    "tsvdm_plan_set_tuning": (_i32, [_vp, _i32, _i32, _i32, _i32, _i32, _i32]),
    "tsvdm_plan_set_engine": (_i32, [_vp, _i32]),
    "tsvdm_plan_set_warm_start": (_i32, [_vp, _i32]),
    "tsvdm_plan_set_angle_precision": (_i32, [_vp, _i32]),
    "tsvdm_plan_set_wait_limit": (_i32, [_vp, _i64]),
    "tsvdm_plan_set_vectors": (_i32, [_vp, _i32]),
    "tsvdm_plan_set_transform": (_i32, [_vp, _i32]),
    "tsvdm_probe_peak": (_i32, [_i32, _i64, _vp, _pdbl]),
    "tsvdm_data_transform": (_i32, [_vp, _vp, _vp]),
    "tsvdm_transform": (_i32, [_vp, _vp, _vp, _i32, _vp]),
    "tsvdm_fixed_rank": (_i32, [_vp, _vp, _vp, _i64, _vp, _vp, _vp, _i32, _pdbl]),
    "tsvdm_tolerance": (_i32, [_vp, _vp, _vp, _dbl, _vp, _vp, _vp, _vp, _vp, _i64, _pi64, _pdbl]),
    "tsvdm_tolerance_pack": (_i32, [_vp, _vp, _vp, _vp, _i64]),
    "tsvdm_reconstruct": (_i32, [_vp, _vp, _vp, _vp, _vp, _i64, _vp, _vp]),
    "tsvdm_backward": (_i32, [_vp, _vp, _vp, _i64, _vp, _vp, _vp, _dbl, _vp, _vp, _vp]),
    "tsvdm_last_status": (_i32, [_vp]),
    "tsvdm_plan_stats": (_i32, [_vp, _pi64, _pi64]),
    "tsvdm_strerror": (ctypes.c_char_p, [_i32]),
    "tsvdm_cayley": (_i32, [_i64, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "tsvdm_cayley_backward": (_i32, [_i64, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "tsvdm_plan_profile": (_i32, [_vp, _i32]),
    "tsvdm_plan_profile_read": (_i32, [_vp, ctypes.POINTER(ctypes.c_float), _pi64]),
    "tsvdm_batch_create": (_i32, [_vp, _i32, _i32, _i32, _vp, ctypes.POINTER(_vp)]),
    "tsvdm_batch_destroy": (_i32, [_vp]),
    "tsvdm_batch_run": (_i32, [_vp, _vp]),
    "tsvdm_batch_capture": (_i32, [_vp, _vp]),
    "tsvdm_batch_launch": (_i32, [_vp]),
    "tsvdm_batch_tune": (_i32, [_vp, _vp, ctypes.POINTER(ctypes.c_int)]),
    "tsvdm_batch_status": (_i32, [_vp, _pi64, _pi64]),
    "tsvdm_batch_graph_kernels": (_i32, [_vp, _pi64]),
    "tsvdm_select_ranks_noalloc": (_i32, [_vp, _i64, _i64, _dbl, _vp, _vp, _vp, _vp]),
    "tsvdm_adam": (_i32, [_i64, _i32, _vp, _vp, _vp, _vp, _i64, _dbl, _dbl, _dbl, _dbl, _vp]),
}

_lock = threading.Lock()
_lib = None


class TsvdmError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = status
        msg = lib().tsvdm_strerror(status).decode() if _lib is not None else str(status)
        super().__init__("%s: %s (status %d)" % (where, msg, status))


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError("libtsvdm.so is not built (run __graft_entry__.build() or "
                                   "python paper_2605_16058_gb300/build.py)")
            h = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(h, name)
                f.restype = res
                f.argtypes = args
            _lib = h
    return _lib


def check(status, where):
    if status != OK:
        raise TsvdmError(status, where)
    return status


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


# ---------------------------------------------------------------- thin wrappers
def tsvdm_plan_create(n1, n2, n3, dtype, prec, m_is_orthogonal, stream=None):
    h = ctypes.c_void_p()
    check(lib().tsvdm_plan_create(n1, n2, n3, dtype, prec, int(bool(m_is_orthogonal)),
                                  _stream(stream), ctypes.byref(h)), "tsvdm_plan_create")
    return h


def tsvdm_plan_create_dway(dims, dtype, prec, m_is_orthogonal, stream=None):
    h = ctypes.c_void_p()
    arr = (ctypes.c_int64 * max(len(dims), 1))(*[int(d) for d in dims])
    check(lib().tsvdm_plan_create_dway(len(dims), arr, dtype, prec, int(bool(m_is_orthogonal)),
                                       _stream(stream), ctypes.byref(h)),
          "tsvdm_plan_create_dway")
    return h


def tsvdm_plan_destroy(plan):
    return lib().tsvdm_plan_destroy(plan)


def tsvdm_plan_set_jacobi(plan, tol, max_sweeps):
    return check(lib().tsvdm_plan_set_jacobi(plan, float(tol), int(max_sweeps)),
                 "tsvdm_plan_set_jacobi")


def tsvdm_plan_set_tuning(plan, block_width=0, cluster_size=0, clusters=0, stages=0, ordering=0,
                          inner_sweeps=0):
    return check(lib().tsvdm_plan_set_tuning(plan, int(block_width), int(cluster_size),
                                             int(clusters), int(stages), int(ordering),
                                             int(inner_sweeps)),
                 "tsvdm_plan_set_tuning")


def tsvdm_plan_set_engine(plan, engine):
    e = ENGINES[engine] if isinstance(engine, str) else int(engine)
    return check(lib().tsvdm_plan_set_engine(plan, e), "tsvdm_plan_set_engine")


def tsvdm_plan_set_warm_start(plan, enable):
    return check(lib().tsvdm_plan_set_warm_start(plan, int(bool(enable))),
                 "tsvdm_plan_set_warm_start")


def tsvdm_plan_set_angle_precision(plan, angles):
    a = ANGLES[angles] if isinstance(angles, str) else int(angles)
    return check(lib().tsvdm_plan_set_angle_precision(plan, a), "tsvdm_plan_set_angle_precision")


VECTORS_ACCUMULATE, VECTORS_SECOND_PASS = 0, 1
VECTORS = {"accumulate": VECTORS_ACCUMULATE, "second_pass": VECTORS_SECOND_PASS}


def tsvdm_plan_set_vectors(plan, mode):
    m = VECTORS[mode] if isinstance(mode, str) else int(mode)
    return check(lib().tsvdm_plan_set_vectors(plan, m), "tsvdm_plan_set_vectors")


TRANSFORM_DENSE, TRANSFORM_DCT2 = 0, 1
TRANSFORMS = {"dense": TRANSFORM_DENSE, "dct2": TRANSFORM_DCT2}


def tsvdm_plan_set_transform(plan, kind):
    k = TRANSFORMS[kind] if isinstance(kind, str) else int(kind)
    return check(lib().tsvdm_plan_set_transform(plan, k), "tsvdm_plan_set_transform")


def tsvdm_plan_set_wait_limit(plan, polls):
    return check(lib().tsvdm_plan_set_wait_limit(plan, int(polls)), "tsvdm_plan_set_wait_limit")


PROBE_FP32_FMA, PROBE_TF32_MMA, PROBE_BF16_MMA, PROBE_FP64_FMA = 0, 1, 2, 3


def tsvdm_probe_peak(unit, iters, stream=None):
    """Measured TFLOP/s of one unit (see include/tsvdm.h)."""
    out = ctypes.c_double(math.nan)
    check(lib().tsvdm_probe_peak(int(unit), int(iters), _stream(stream), ctypes.byref(out)),
          "tsvdm_probe_peak")
    return out.value


def tsvdm_data_transform(plan, X, M):
    return check(lib().tsvdm_data_transform(plan, _ptr(X), _ptr(M)), "tsvdm_data_transform")


def tsvdm_transform(plan, X, M, inverse, Y):
    return check(lib().tsvdm_transform(plan, _ptr(X), _ptr(M), int(inverse), _ptr(Y)),
                 "tsvdm_transform")


def tsvdm_fixed_rank(plan, X, M, k, U, S, V, original_domain=0, want_rel_err=True,
                     raise_on_error=True):
    err = ctypes.c_double(math.nan)
    st = lib().tsvdm_fixed_rank(plan, _ptr(X), _ptr(M), int(k), _ptr(U), _ptr(S), _ptr(V),
                                int(original_domain), ctypes.byref(err) if want_rel_err else None)
    if raise_on_error:
        check(st, "tsvdm_fixed_rank")
    return (err.value if want_rel_err else None), st


def tsvdm_tolerance(plan, X, M, eps, ranks, offsets, U, S, V, capacity, want_rel_err=True,
                    raise_on_error=True):
    tot = ctypes.c_int64(0)
    err = ctypes.c_double(math.nan)
    st = lib().tsvdm_tolerance(plan, _ptr(X), _ptr(M), float(eps), _ptr(ranks), _ptr(offsets),
                               _ptr(U), _ptr(S), _ptr(V), int(capacity), ctypes.byref(tot),
                               ctypes.byref(err) if want_rel_err else None)
    if raise_on_error and st not in (OK, ECAPACITY):
        check(st, "tsvdm_tolerance")
    return tot.value, (err.value if want_rel_err else None), st


def tsvdm_tolerance_pack(plan, U, S, V, capacity):
    return check(lib().tsvdm_tolerance_pack(plan, _ptr(U), _ptr(S), _ptr(V), int(capacity)),
                 "tsvdm_tolerance_pack")


def tsvdm_reconstruct(plan, U, S, V, offsets, k, M, Xk):
    return check(lib().tsvdm_reconstruct(plan, _ptr(U), _ptr(S), _ptr(V), _ptr(offsets), int(k),
                                         _ptr(M), _ptr(Xk)), "tsvdm_reconstruct")


def tsvdm_backward(plan, X, M, k, U, S, V, dL, dX, dM, loss=None):
    """loss: None, a 1-element float64 CUDA tensor (written without synchronising), or
    'host' to return the value."""
    if isinstance(loss, str):
        out = ctypes.c_double(math.nan)
        check(lib().tsvdm_backward(plan, _ptr(X), _ptr(M), int(k), _ptr(U), _ptr(S), _ptr(V),
                                   float(dL), _ptr(dX), _ptr(dM), ctypes.byref(out)),
              "tsvdm_backward")
        return out.value
    check(lib().tsvdm_backward(plan, _ptr(X), _ptr(M), int(k), _ptr(U), _ptr(S), _ptr(V),
                               float(dL), _ptr(dX), _ptr(dM), _ptr(loss)), "tsvdm_backward")
    return None


def tsvdm_last_status(plan):
    return lib().tsvdm_last_status(plan)


def tsvdm_plan_stats(plan):
    a, b = ctypes.c_int64(0), ctypes.c_int64(0)
    check(lib().tsvdm_plan_stats(plan, ctypes.byref(a), ctypes.byref(b)), "tsvdm_plan_stats")
    return a.value, b.value


STAGES = ("ttm", "transpose", "jacobi", "finalize", "select", "emit", "other")


def tsvdm_plan_profile(plan, enable):
    return check(lib().tsvdm_plan_profile(plan, int(enable)), "tsvdm_plan_profile")


def tsvdm_plan_profile_read(plan):
    ms = (ctypes.c_float * len(STAGES))()
    n = ctypes.c_int64(0)
    check(lib().tsvdm_plan_profile_read(plan, ms, ctypes.byref(n)), "tsvdm_plan_profile_read")
    return dict(zip(STAGES, [float(x) for x in ms])), n.value


class BatchDesc(ctypes.Structure):
    _fields_ = [("n1", ctypes.c_int64), ("n2", ctypes.c_int64), ("n3", ctypes.c_int64),
                ("mode", ctypes.c_int), ("k", ctypes.c_int64), ("eps", ctypes.c_double)]


class BatchIO(ctypes.Structure):
    _fields_ = [("X", _vp), ("M", _vp), ("U", _vp), ("S", _vp), ("V", _vp),
                ("ranks", _vp), ("offsets", _vp), ("rel_err", _vp)]


def tsvdm_batch_create(descs, dtype, prec, stream=None):
    arr = (BatchDesc * len(descs))(*descs)
    h = ctypes.c_void_p()
    check(lib().tsvdm_batch_create(arr, len(descs), dtype, prec, _stream(stream),
                                   ctypes.byref(h)), "tsvdm_batch_create")
    return h


def _io_array(ios):
    return (BatchIO * len(ios))(*ios)


def tsvdm_batch_run(b, ios):
    return check(lib().tsvdm_batch_run(b, _io_array(ios)), "tsvdm_batch_run")


def tsvdm_batch_capture(b, ios):
    return check(lib().tsvdm_batch_capture(b, _io_array(ios)), "tsvdm_batch_capture")


def tsvdm_batch_launch(b):
    return check(lib().tsvdm_batch_launch(b), "tsvdm_batch_launch")


def tsvdm_batch_tune(b, ios):
    ch = (ctypes.c_int * 4)()
    check(lib().tsvdm_batch_tune(b, _io_array(ios), ch), "tsvdm_batch_tune")
    return dict(width=ch[0], cluster=ch[1], stages=ch[2], jacobi_ms=ch[3] / 1000.0)


def tsvdm_batch_status(b):
    a, c = ctypes.c_int64(0), ctypes.c_int64(0)
    st = lib().tsvdm_batch_status(b, ctypes.byref(a), ctypes.byref(c))
    return st, a.value, c.value


def tsvdm_batch_graph_kernels(b):
    k = ctypes.c_int64(0)
    check(lib().tsvdm_batch_graph_kernels(b, ctypes.byref(k)), "tsvdm_batch_graph_kernels")
    return k.value


def tsvdm_batch_destroy(b):
    return lib().tsvdm_batch_destroy(b)


def tsvdm_cayley(n, dtype, A, M0, M, Z, Q, work, stream=None):
    return check(lib().tsvdm_cayley(int(n), dtype, _ptr(A), _ptr(M0), _ptr(M), _ptr(Z), _ptr(Q),
                                    _ptr(work), _stream(stream)), "tsvdm_cayley")


def tsvdm_cayley_backward(n, dtype, M0, Z, Q, dM, dA, work, stream=None):
    return check(lib().tsvdm_cayley_backward(int(n), dtype, _ptr(M0), _ptr(Z), _ptr(Q), _ptr(dM),
                                             _ptr(dA), _ptr(work), _stream(stream)),
                 "tsvdm_cayley_backward")


def tsvdm_adam(count, dtype, param, grad, m1, m2, step, lr, beta1=0.9, beta2=0.999, eps=1e-8,
               stream=None):
    return check(lib().tsvdm_adam(int(count), dtype, _ptr(param), _ptr(grad), _ptr(m1), _ptr(m2),
                                  int(step), float(lr), float(beta1), float(beta2), float(eps),
                                  _stream(stream)), "tsvdm_adam")
