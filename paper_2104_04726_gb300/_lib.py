"""ctypes loader of the in-tree CUDA library (`_build/libmes.so`).

Argument marshalling only.  Loading fails loudly when the library has not
been built: there is no fallback implementation of any entry point.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libmes.so")

STATUS = {
    0: "MES_OK",
    1: "MES_ERR_INVALID_ARG",
    2: "MES_ERR_RANK",
    3: "MES_ERR_OOM",
    4: "MES_ERR_CUDA",
    5: "MES_ERR_TIMEOUT",
    6: "MES_ERR_NONFINITE",
    7: "MES_ERR_NOT_IMPLEMENTED",
}

# Entry points declared in include/mes.h, with their ctypes signatures.
_c = ctypes
_p = _c.c_void_p
_i64p = _c.POINTER(_c.c_int64)
SIGNATURES = {
    "mes_last_error": (_c.c_char_p, []),
    "mes_version": (_c.c_char_p, []),
    "mes_colour_convert": (_c.c_int, [_p, _c.c_int64, _c.c_int64, _c.c_int64, _c.c_int, _c.c_float,
                                      _p, _p, _p]),
    "mes_colour_invert": (_c.c_int, [_p, _c.c_int64, _c.c_int64, _c.c_int64, _c.c_int, _c.c_float,
                                     _p, _p, _p, _p, _p]),
    "mes_tucker_als": (_c.c_int, [_p, _c.c_int, _i64p, _i64p, _c.c_int, _c.c_double, _p,
                                  _c.POINTER(_p), _p, _p, _p]),
    "mes_tucker_als_workspace_size": (_c.c_int, [_c.c_int, _i64p, _i64p, _p, _c.POINTER(_c.c_size_t)]),
    "mes_reconstruct": (_c.c_int, [_p, _c.POINTER(_p), _c.c_int, _i64p, _i64p, _p, _p, _p, _c.c_int, _p]),
    "mes_quantize_core": (_c.c_int, [_p, _c.c_int, _i64p, _c.c_int, _p, _p, _c.c_int, _p]),
    "mes_dequantize_core": (_c.c_int, [_p, _p, _c.c_int, _i64p, _p, _p]),
    "mes_quantize_core_noalloc": (_c.c_int, [_p, _c.c_int, _i64p, _c.c_int, _p, _p, _p]),
    "mes_gemm_selftest": (_c.c_int, [_c.c_int, _p, _p, _p, _c.c_int64, _c.c_int64, _c.c_int64, _c.c_int, _p]),
    "mes_solve_selftest": (_c.c_int, [_p, _c.c_int, _p, _c.c_int64, _p, _p, _p, _p, _p]),
    "mes_batch_create": (_c.c_int, [_c.c_int, _c.POINTER(_p)]),
    "mes_batch_run": (_c.c_int, [_p, _p, _c.c_int, _c.POINTER(_c.c_int), _p]),
    "mes_batch_capture": (_c.c_int, [_p, _p, _c.c_int, _p]),
    "mes_batch_launch": (_c.c_int, [_p, _p]),
    "mes_batch_destroy": (_c.c_int, [_p]),
    "mes_serve_create": (_c.c_int, [_c.c_size_t, _c.c_int, _c.POINTER(_p)]),
    "mes_serve_submit": (_c.c_int, [_p, _p, _c.POINTER(_c.c_uint64)]),
    "mes_serve_poll": (_c.c_int, [_p, _c.c_uint64, _c.POINTER(_c.c_int), _c.POINTER(_c.c_int),
                                  _c.POINTER(_c.c_double)]),
    "mes_serve_wait": (_c.c_int, [_p, _c.c_uint64, _c.c_double, _c.POINTER(_c.c_int), _c.POINTER(_c.c_double)]),
    "mes_serve_get_stats": (_c.c_int, [_p, _p]),
    "mes_serve_destroy": (_c.c_int, [_p]),
    "mes_profile_enable": (None, [_c.c_int]),
    "mes_profile_count": (_c.c_int, []),
    "mes_profile_get": (_c.c_int, [_c.c_int, _c.c_char_p, _c.c_int, _i64p, _c.POINTER(_c.c_double),
                                   _c.POINTER(_c.c_double), _c.POINTER(_c.c_double)]),
}


class MesAlsOpts(ctypes.Structure):
    """Mirror of `mes_als_opts` in include/mes.h."""
    _fields_ = [
        ("precision", ctypes.c_int),
        ("init_iters", ctypes.c_int),
        ("inner_iters", ctypes.c_int),
        ("seed", ctypes.c_uint64),
        ("init_factors", ctypes.POINTER(ctypes.c_void_p)),
        ("iters_done", ctypes.c_void_p),
        ("fit_history", ctypes.c_void_p),
        ("canonical", ctypes.c_int),
        ("init", ctypes.c_int),
        ("reconstruction", ctypes.c_void_p),
        ("status", ctypes.c_void_p),
        ("wait_ns", ctypes.c_int64),
        ("concurrency", ctypes.c_int),
    ]


class MesProblem(ctypes.Structure):
    """Mirror of `mes_problem` in include/mes.h."""
    _fields_ = [
        ("rgb8", ctypes.c_void_p),
        ("space", ctypes.c_int),
        ("gamma", ctypes.c_float),
        ("X", ctypes.c_void_p),
        ("N", ctypes.c_int),
        ("dims", ctypes.c_int64 * 8),
        ("ranks", ctypes.c_int64 * 8),
        ("max_iters", ctypes.c_int),
        ("tol", ctypes.c_double),
        ("opts", MesAlsOpts),
        ("core", ctypes.c_void_p),
        ("factors", ctypes.c_void_p * 8),
        ("fit", ctypes.c_void_p),
        ("quant_bits", ctypes.c_int),
        ("q", ctypes.c_void_p),
        ("scales", ctypes.c_void_p),
    ]


class MesServeStats(ctypes.Structure):
    """Mirror of `mes_serve_stats` in include/mes.h."""
    _fields_ = [
        ("submitted", ctypes.c_uint64),
        ("completed", ctypes.c_uint64),
        ("failed", ctypes.c_uint64),
        ("queued", ctypes.c_uint64),
        ("running", ctypes.c_uint64),
        ("p50_ms", ctypes.c_double),
        ("p99_ms", ctypes.c_double),
        ("max_ms", ctypes.c_double),
        ("mean_ms", ctypes.c_double),
        ("first_admit_s", ctypes.c_double),
        ("last_done_s", ctypes.c_double),
        ("hbm_in_use", ctypes.c_size_t),
        ("hbm_peak", ctypes.c_size_t),
    ]


class MesError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        self.status = status
        self.name = STATUS.get(status, str(status))
        super().__init__(f"{where}: {self.name}: {msg}")


_lib = None


def load(path: str = LIB_PATH):
    """Load the library (once) and attach the signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(
            f"CUDA library not built ({path} missing); run `python -m paper_2104_04726_gb300.build`")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(status: int, where: str) -> None:
    if status != 0:
        msg = load().mes_last_error().decode(errors="replace")
        raise MesError(status, where, msg)
