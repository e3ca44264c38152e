"""Thin Python binding of libse1p's C ABI (include/se1p.h).

Argument marshalling only: every step of the evaluation runs in the CUDA
library.  Functions carry the C names; device arrays are torch CUDA tensors
(float64, contiguous) whose data pointers are handed to the library, and the
stream is the caller's current torch stream unless one is given.

The shared library is built in-tree by ``paper_1611_09538_gb300.build.build()``.
If it is missing, every call raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libse1p.so")

SE1P_FP64 = 0
SE1P_MIXED = 1
SE1P_FLAG_TRIPLY_PERIODIC = 1  # params.flags: the triply periodic comparison method (SE3P)

STATUS = {
    0: "SE1P_OK", 1: "SE1P_ERR_INVALID_ARG", 2: "SE1P_ERR_NOT_NEUTRAL", 3: "SE1P_ERR_OUT_OF_BOX",
    4: "SE1P_ERR_ALLOC", 5: "SE1P_ERR_CUDA", 6: "SE1P_ERR_TIMEOUT", 7: "SE1P_ERR_NAN",
    8: "SE1P_ERR_CAPACITY",
}

# every symbol include/se1p.h declares
EXPORTS = (
    "se1p_plan_create", "se1p_plan_destroy", "se1p_plan_get_info", "se1p_eval", "se1p_eval_host",
    "se1p_eval_vjp",
    "se1p_spread", "se1p_fourier", "se1p_gather", "se1p_real_space", "se1p_plan_set_profiling",
    "se1p_plan_stage_times", "se1p_plan_sync_status", "se1p_real_space_noalloc", "se1p_status_string",
    "se1p_autotune", "se1p_batch_create", "se1p_batch_destroy", "se1p_batch_eval", "se1p_batch_sync_status",
    "se1p_batch_plan", "se1p_measure_fma_peak",
)

STAGES = ("pack", "spread", "fourier", "gather", "real", "final")


class SE1PError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {STATUS.get(code, code)}")


class se1p_params(ctypes.Structure):
    _fields_ = [
        ("L", ctypes.c_double * 3), ("xi", ctypes.c_double), ("M", ctypes.c_int * 3), ("P", ctypes.c_int),
        ("Mt", ctypes.c_int), ("n0", ctypes.c_int), ("nI", ctypes.c_int), ("nl", ctypes.c_int),
        ("s0", ctypes.c_double), ("sl", ctypes.c_double), ("rc", ctypes.c_double), ("tol", ctypes.c_double),
        ("precision", ctypes.c_int), ("flags", ctypes.c_int),
    ]


class se1p_plan_info(ctypes.Structure):
    _fields_ = [
        ("Mt", ctypes.c_int), ("M3", ctypes.c_int), ("n0", ctypes.c_int), ("nI", ctypes.c_int),
        ("nl", ctypes.c_int), ("n_I_modes", ctypes.c_int), ("P", ctypes.c_int), ("precision", ctypes.c_int),
        ("h", ctypes.c_double), ("hz", ctypes.c_double), ("eta", ctypes.c_double), ("etaz", ctypes.c_double),
        ("R", ctypes.c_double), ("cells", ctypes.c_int * 3), ("features", ctypes.c_int),
        ("workspace_bytes", ctypes.c_size_t),
    ]


class se1p_tune_request(ctypes.Structure):
    _fields_ = [
        ("L", ctypes.c_double * 3), ("xi", ctypes.c_double), ("Q", ctypes.c_double), ("n", ctypes.c_int),
        ("tol", ctypes.c_double), ("precision", ctypes.c_int),
    ]


_lib = None


def load(path: str | None = None):
    """Load libse1p.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libse1p.so not found at {p}; build it with "
                           "paper_1611_09538_gb300.build.build() (needs nvcc)")
    lib = ctypes.CDLL(p)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.se1p_plan_create.argtypes = [ctypes.POINTER(se1p_params), i, ctypes.POINTER(vp)]
    lib.se1p_plan_destroy.argtypes = [vp]
    lib.se1p_plan_get_info.argtypes = [vp, ctypes.POINTER(se1p_plan_info)]
    lib.se1p_eval.argtypes = [vp, i, vp, vp, vp, vp, vp, vp]
    lib.se1p_eval_host.argtypes = [vp, i, vp, vp, vp, vp, vp, vp]
    lib.se1p_eval_vjp.argtypes = [vp, i, vp, vp, vp, vp, vp, vp]
    lib.se1p_spread.argtypes = [vp, i, vp, vp, vp, vp]
    lib.se1p_fourier.argtypes = [vp, vp, vp, vp]
    lib.se1p_gather.argtypes = [vp, i, vp, vp, vp, vp, vp, vp]
    lib.se1p_real_space.argtypes = [vp, i, vp, vp, vp, vp, vp]
    lib.se1p_plan_set_profiling.argtypes = [vp, i]
    lib.se1p_plan_stage_times.argtypes = [vp, ctypes.POINTER(d), ctypes.POINTER(i)]
    lib.se1p_plan_sync_status.argtypes = [vp, vp]
    lib.se1p_real_space_noalloc.argtypes = [ctypes.POINTER(se1p_params), i, vp, vp, vp, vp, vp]
    lib.se1p_status_string.argtypes = [i]
    lib.se1p_status_string.restype = ctypes.c_char_p
    lib.se1p_autotune.argtypes = [ctypes.POINTER(se1p_tune_request), ctypes.POINTER(se1p_params)]
    lib.se1p_batch_create.argtypes = [i, ctypes.POINTER(se1p_params), ctypes.POINTER(i), ctypes.POINTER(vp)]
    lib.se1p_batch_destroy.argtypes = [vp]
    lib.se1p_batch_eval.argtypes = [vp, ctypes.POINTER(i), vp, vp, vp, vp, vp, vp]
    lib.se1p_batch_sync_status.argtypes = [vp, vp]
    lib.se1p_batch_plan.argtypes = [vp, i]
    lib.se1p_batch_plan.restype = vp
    lib.se1p_measure_fma_peak.argtypes = [i, ctypes.POINTER(d), ctypes.POINTER(i)]
    for name in EXPORTS:
        if name not in ("se1p_status_string", "se1p_batch_plan"):
            getattr(lib, name).restype = i
    _lib = lib
    return lib


def _check(code: int, where: str):
    if code != 0:
        raise SE1PError(code, where)


def _ptr(t):
    """Data pointer of a contiguous float64 tensor / numpy array, or None."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        if not t.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return t.data_ptr()
    return t.ctypes.data  # numpy (host entry points)


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def make_params(L, xi, M, P, *, Mt=0, n0=0, nI=0, nl=-1, s0=0.0, sl=0.0, rc=0.0, tol=0.0,
                precision=SE1P_FP64, flags=0) -> se1p_params:
    prm = se1p_params()
    prm.L[:] = [float(v) for v in L]
    prm.xi = float(xi)
    prm.M[:] = [int(v) for v in M]
    prm.P = int(P)
    prm.Mt, prm.n0, prm.nI, prm.nl = int(Mt), int(n0), int(nI), int(nl)
    prm.s0, prm.sl, prm.rc, prm.tol = float(s0), float(sl), float(rc if rc is not None else 0.0), float(tol)
    prm.precision = int(precision)
    prm.flags = int(flags)
    return prm


# ------------------------------------------------------------------ C-named entry points

def se1p_plan_create(params: se1p_params, n_max: int) -> int:
    lib = load()
    h = ctypes.c_void_p()
    _check(lib.se1p_plan_create(ctypes.byref(params), int(n_max), ctypes.byref(h)), "se1p_plan_create")
    return h.value


def se1p_plan_destroy(plan: int) -> None:
    _check(load().se1p_plan_destroy(plan), "se1p_plan_destroy")


def se1p_plan_get_info(plan: int) -> se1p_plan_info:
    info = se1p_plan_info()
    _check(load().se1p_plan_get_info(plan, ctypes.byref(info)), "se1p_plan_get_info")
    return info


def se1p_eval(plan, n, x, q, phi=None, force=None, energy=None, stream=None) -> None:
    _check(load().se1p_eval(plan, int(n), _ptr(x), _ptr(q), _ptr(phi), _ptr(force), _ptr(energy),
                            _stream(stream)), "se1p_eval")


def se1p_eval_host(plan, n, x, q, phi=None, force=None, energy=None, stream=None) -> None:
    _check(load().se1p_eval_host(plan, int(n), _ptr(x), _ptr(q), _ptr(phi), _ptr(force), _ptr(energy),
                                 _stream(stream)), "se1p_eval_host")


def se1p_eval_vjp(plan, n, x, q, v_phi, grad_x=None, grad_q=None, stream=None) -> None:
    _check(load().se1p_eval_vjp(plan, int(n), _ptr(x), _ptr(q), _ptr(v_phi), _ptr(grad_x), _ptr(grad_q),
                                _stream(stream)), "se1p_eval_vjp")


def se1p_spread(plan, n, x, q, grid, stream=None) -> None:
    _check(load().se1p_spread(plan, int(n), _ptr(x), _ptr(q), _ptr(grid), _stream(stream)), "se1p_spread")


def se1p_fourier(plan, grid_in, grid_out, stream=None) -> None:
    _check(load().se1p_fourier(plan, _ptr(grid_in), _ptr(grid_out), _stream(stream)), "se1p_fourier")


def se1p_gather(plan, n, x, q, grid, phi=None, force=None, stream=None) -> None:
    _check(load().se1p_gather(plan, int(n), _ptr(x), _ptr(q), _ptr(grid), _ptr(phi), _ptr(force),
                              _stream(stream)), "se1p_gather")


def se1p_real_space(plan, n, x, q, phi=None, force=None, stream=None) -> None:
    _check(load().se1p_real_space(plan, int(n), _ptr(x), _ptr(q), _ptr(phi), _ptr(force), _stream(stream)),
           "se1p_real_space")


def se1p_plan_set_profiling(plan, enable) -> None:
    """enable: False/0 off, True/1 on, 2 on with the stages run in sequence (times alone)."""
    _check(load().se1p_plan_set_profiling(plan, int(enable)), "se1p_plan_set_profiling")


def se1p_plan_stage_times(plan) -> tuple[dict, int]:
    """Summed per-stage milliseconds over the recorded evaluations, and their count."""
    ms = (ctypes.c_double * len(STAGES))()
    n = ctypes.c_int()
    _check(load().se1p_plan_stage_times(plan, ms, ctypes.byref(n)), "se1p_plan_stage_times")
    return dict(zip(STAGES, list(ms))), n.value


def se1p_plan_sync_status(plan, stream=None) -> int:
    """Synchronise and return (not raise) the device status code."""
    return int(load().se1p_plan_sync_status(plan, _stream(stream)))


def se1p_real_space_noalloc(params: se1p_params, n, x, q, phi, force, stream=None) -> None:
    """Real-space sum without any device allocation (scratch in a static device array;
    n <= 16384; concurrent calls must be serialised by the caller)."""
    _check(load().se1p_real_space_noalloc(ctypes.byref(params), int(n), _ptr(x), _ptr(q), _ptr(phi),
                                          _ptr(force), _stream(stream)), "se1p_real_space_noalloc")


def se1p_measure_fma_peak(precision) -> tuple[float, int]:
    """Measured FMA throughput (TFLOP/s, FP32 for SE1P_MIXED, FP64 for SE1P_FP64) of the
    current device and its multiprocessor count."""
    tf = ctypes.c_double()
    sms = ctypes.c_int()
    _check(load().se1p_measure_fma_peak(int(precision), ctypes.byref(tf), ctypes.byref(sms)),
           "se1p_measure_fma_peak")
    return tf.value, sms.value


def se1p_status_string(code: int) -> str:
    return load().se1p_status_string(int(code)).decode()


def se1p_autotune(L, xi, Q, n, tol, precision=SE1P_FP64) -> se1p_params:
    req = se1p_tune_request()
    req.L[:] = [float(v) for v in L]
    req.xi, req.Q, req.n, req.tol, req.precision = float(xi), float(Q), int(n), float(tol), int(precision)
    out = se1p_params()
    _check(load().se1p_autotune(ctypes.byref(req), ctypes.byref(out)), "se1p_autotune")
    return out


def se1p_batch_create(params_list, n_max_list) -> int:
    count = len(params_list)
    arr = (se1p_params * count)(*params_list)
    nm = (ctypes.c_int * count)(*[int(v) for v in n_max_list])
    h = ctypes.c_void_p()
    _check(load().se1p_batch_create(count, arr, nm, ctypes.byref(h)), "se1p_batch_create")
    return h.value


def se1p_batch_destroy(batch) -> None:
    _check(load().se1p_batch_destroy(batch), "se1p_batch_destroy")


def se1p_batch_eval(batch, offsets, x, q, phi=None, force=None, energy=None, stream=None) -> None:
    off = (ctypes.c_int * len(offsets))(*[int(v) for v in offsets])
    _check(load().se1p_batch_eval(batch, off, _ptr(x), _ptr(q), _ptr(phi), _ptr(force), _ptr(energy),
                                  _stream(stream)), "se1p_batch_eval")


def se1p_batch_sync_status(batch, stream=None) -> int:
    return int(load().se1p_batch_sync_status(batch, _stream(stream)))


def se1p_batch_plan(batch, i: int) -> int:
    return load().se1p_batch_plan(batch, int(i))


# ------------------------------------------------------------------ convenience wrapper

@dataclass
class Result:
    phi: object
    force: object
    energy: object


class Plan:
    """Owns one C plan; evaluates torch CUDA tensors (x [n,3], q [n], float64)."""

    def __init__(self, L, xi, M, P, n_max, **kw):
        """L, xi, M, P as in se1p_params; keywords as make_params."""
        self.params = make_params(L, xi, M, P, **kw)
        self.handle = se1p_plan_create(self.params, n_max)
        self.n_max = n_max

    @classmethod
    def from_params(cls, params: se1p_params, n_max):
        """A plan from a filled se1p_params (e.g. the result of se1p_autotune)."""
        self = cls.__new__(cls)
        self.params = params
        self.handle = se1p_plan_create(params, n_max)
        self.n_max = n_max
        return self

    @property
    def info(self) -> se1p_plan_info:
        return se1p_plan_info_copy(se1p_plan_get_info(self.handle))

    def grid_shape(self):
        i = se1p_plan_get_info(self.handle)
        return (i.M3, i.Mt, i.Mt)

    def eval(self, x, q, stream=None, check=True) -> Result:
        import torch
        n = x.shape[0]
        phi = torch.empty(n, dtype=torch.float64, device=x.device)
        force = torch.empty((n, 3), dtype=torch.float64, device=x.device)
        energy = torch.empty(1, dtype=torch.float64, device=x.device)
        se1p_eval(self.handle, n, x, q, phi, force, energy, stream)
        if check:
            _check(se1p_plan_sync_status(self.handle, stream), "se1p_eval (device status)")
        return Result(phi, force, energy)

    def close(self):
        if getattr(self, "handle", None):
            se1p_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass


def se1p_plan_info_copy(info: se1p_plan_info) -> dict:
    return {k: (list(getattr(info, k)) if k == "cells" else getattr(info, k)) for k, _ in info._fields_}
