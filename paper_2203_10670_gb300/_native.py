"""ctypes view of libfcfs (include/fcfs.h): structures, entry points, codes.

Argument marshalling only.  Loading fails loudly when the library has not
been built; there is no fallback implementation anywhere in this package.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfcfs.so")

# fcfs_status
FCFS_OK = 0
FCFS_ERR_ARG = -1
FCFS_ERR_KERNEL_TOO_SMALL = -2
FCFS_ERR_UNSUPPORTED = -3
FCFS_ERR_CUDA = -4
FCFS_ERR_NOMEM = -5
FCFS_ERR_TIMEOUT = -6
FCFS_ERR_BUSY = -7
# fcfs_method
FCFS_NEAREST, FCFS_BILINEAR, FCFS_BICUBIC = 0, 1, 2
# fcfs_pad
FCFS_PAD_REPLICATE, FCFS_PAD_CONSTANT, FCFS_PAD_REFLECT = 0, 1, 2
# fcfs_align
FCFS_ALIGN_PAPER, FCFS_ALIGN_HALF_PIXEL, FCFS_ALIGN_FLOOR = 0, 1, 2
FCFS_ACT_NONE, FCFS_ACT_RELU, FCFS_ACT_LEAKY_RELU, FCFS_ACT_CLAMP = 0, 1, 2, 3
# fcfs_dtype
FCFS_F32, FCFS_BF16, FCFS_U8 = 0, 1, 2
FCFS_MAX_R = 64
FCFS_MAX_TAPS = 9


class fcfs_axis(ctypes.Structure):
    _fields_ = [("r", ctypes.c_int), ("s", ctypes.c_int), ("K", ctypes.c_int), ("method", ctypes.c_int),
                ("w", ctypes.c_void_p), ("w_per_channel", ctypes.c_int)]


class fcfs_desc(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("n", ctypes.c_longlong), ("c", ctypes.c_longlong),
                ("in_shape", ctypes.c_longlong * 3), ("out_shape", ctypes.c_longlong * 3),
                ("dtype_in", ctypes.c_int), ("dtype_out", ctypes.c_int), ("pad", ctypes.c_int),
                ("pad_value", ctypes.c_float), ("align", ctypes.c_int), ("axis", fcfs_axis * 3),
                ("cubic_a", ctypes.c_float), ("w2d", ctypes.c_void_p), ("w2d_per_channel", ctypes.c_int),
                ("antialias", ctypes.c_int)]


class fcfs_epilogue(ctypes.Structure):
    _fields_ = [("c_out", ctypes.c_int), ("mix", ctypes.c_void_p), ("bias", ctypes.c_void_p), ("act", ctypes.c_int),
                ("alpha", ctypes.c_float), ("lo", ctypes.c_float), ("hi", ctypes.c_float)]


class fcfs_serve_config(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_inflight", ctypes.c_int),
                ("out_dtype", ctypes.c_int), ("tile_budget_per_step", ctypes.c_int),
                ("timeout_ms", ctypes.c_int), ("auto_release", ctypes.c_int)]


class fcfs_serve_stats_t(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_longlong), ("completed", ctypes.c_longlong),
                ("deferred", ctypes.c_longlong), ("rejected", ctypes.c_longlong), ("steps", ctypes.c_longlong),
                ("max_inflight_seen", ctypes.c_int), ("p50_ms", ctypes.c_double), ("p90_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double), ("out_pixels", ctypes.c_double),
                ("bytes_moved", ctypes.c_double), ("wall_s", ctypes.c_double), ("gpix_s", ctypes.c_double),
                ("gbytes_s", ctypes.c_double), ("canceled", ctypes.c_longlong)]


# every function include/fcfs.h declares: name -> (restype, argtypes)
_P = ctypes.c_void_p
_I = ctypes.c_int
_LL = ctypes.c_longlong
SIGNATURES = {
    "fcfs_make_weights": (_I, [_I, _I, _I, _I, _P, ctypes.POINTER(_I)]),
    "fcfs_geometry": (_I, [_I, _I, _I, _I, _LL, ctypes.POINTER(_LL), ctypes.POINTER(_LL), ctypes.POINTER(_I)]),
    "fcfs_forward": (_I, [ctypes.POINTER(fcfs_desc), _P, _P, _P]),
    "fcfs_forward_fused": (_I, [ctypes.POINTER(fcfs_desc), ctypes.POINTER(fcfs_epilogue), _P, _P, _P]),
    "fcfs_backward_workspace": (ctypes.c_size_t, [ctypes.POINTER(fcfs_desc)]),
    "fcfs_backward_fused_workspace": (ctypes.c_size_t, [ctypes.POINTER(fcfs_desc), ctypes.POINTER(fcfs_epilogue)]),
    "fcfs_backward_fused": (_I, [ctypes.POINTER(fcfs_desc), ctypes.POINTER(fcfs_epilogue), _P, _P, _P, _P, _P, _P, _P,
                                 ctypes.c_size_t, _P]),
    "fcfs_backward": (_I, [ctypes.POINTER(fcfs_desc), _P, _P, _P, _P, _P, ctypes.c_size_t, _P]),
    "fcfs_status_string": (ctypes.c_char_p, [_I]),
    "fcfs_last_error": (ctypes.c_char_p, []),
    "fcfs_tune_forward": (_I, [ctypes.POINTER(fcfs_desc), _P, _P, _P, _I, ctypes.POINTER(ctypes.c_float),
                               ctypes.POINTER(_I)]),
    "fcfs_clear_plans": (None, []),
    "fcfs_plan_count": (_I, []),
    "fcfs_device_status": (_I, [_I]),
    "fcfs_backward_noalloc": (_I, [ctypes.POINTER(fcfs_desc), _P, _P, _P, _P, _P]),
    "fcfs_serve_clock": (ctypes.c_double, []),
    "fcfs_serve_create": (_I, [ctypes.POINTER(fcfs_serve_config), _P, ctypes.POINTER(_P)]),
    "fcfs_serve_submit": (_I, [_P, ctypes.POINTER(fcfs_desc), _P, _P, ctypes.c_double,
                               ctypes.POINTER(ctypes.c_ulonglong)]),
    "fcfs_serve_submit_batch": (_I, [_P, _I, ctypes.POINTER(fcfs_desc), ctypes.POINTER(_P), ctypes.POINTER(_P),
                                     ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_ulonglong),
                                     ctypes.POINTER(_I)]),
    "fcfs_serve_poll": (_I, [_P, ctypes.POINTER(ctypes.c_ulonglong), _I, ctypes.POINTER(_I)]),
    "fcfs_serve_cancel": (_I, [_P, ctypes.c_ulonglong]),
    "fcfs_serve_result": (_I, [_P, ctypes.c_ulonglong, ctypes.POINTER(_P)]),
    "fcfs_serve_release": (_I, [_P, ctypes.c_ulonglong]),
    "fcfs_serve_drain": (_I, [_P, _I]),
    "fcfs_serve_stats": (_I, [_P, ctypes.POINTER(fcfs_serve_stats_t)]),
    "fcfs_serve_destroy": (_I, [_P]),
}
OPTIONAL = set()

_lib = None


def load():
    """Load libfcfs.so (built by paper_2203_10670_gb300.build); raises if missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libfcfs.so is not built ({LIB_PATH}); run paper_2203_10670_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        if not hasattr(lib, name):
            if name in OPTIONAL:
                continue
            raise ImportError(f"libfcfs.so does not export {name}")
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


class FCFSError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = load()
        msg = lib.fcfs_status_string(status).decode()
        detail = lib.fcfs_last_error().decode()
        super().__init__(f"{where}: {msg} ({status}){': ' + detail if detail else ''}")
        self.status = status


def check(status: int, where: str) -> None:
    if status != FCFS_OK:
        raise FCFSError(status, where)
