"""ctypes bindings to ``libdctplus.so`` (argument marshalling only).

There is no fallback: if the shared library is missing or fails to load,
every call raises. Build it with ``paper_2409_08970_gb300.build.build()``.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdctplus.so")

OK = 0
ERR_INVALID_ARG = 1
ERR_UNSUPPORTED = 2
ERR_NOT_CONVERGED = 3
ERR_CUDA = 4
ERR_TIMEOUT = 5
ERR_DEVICE_CHECK = 6
ERR_NO_DEVICE = 7
ERR_SCRATCH_LIMIT = 8

F32 = 0
F64 = 1

CAUCHY_AUTO = 0
CAUCHY_DENSE = 1
CAUCHY_HIER = 2
CAUCHY_SIMT = 3
CAUCHY_DENSE_GFT = 4
CAUCHY_NFST = 5

SEG_WORDS = 3

# every symbol include/dctplus.h declares
EXPORTS = (
    "dctplus_plan", "dctplus_destroy", "dctplus_plan_inspect", "dctplus_plan_size",
    "dctplus_plan_cauchy_mode", "dctplus_plan_far_field", "dctplus_execute", "dctplus_execute_host",
    "dctplus_execute_noalloc", "dctplus_execute_pruned", "dctplus_execute_multi", "dctplus_backward",
    "dctplus_group_create", "dctplus_group_destroy", "dctplus_execute_group",
    "dctplus_execute_group_host", "dctplus_sync_check", "dctplus_launch_count",
    "dctplus_status_string", "dctplus_trace_begin", "dctplus_trace_end", "dctplus_autotune",
    "dctplus_tune_lookup", "dctplus_tune_record",
)


class DctPlusError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        msg = _status_string(status)
        super().__init__(f"{what}: {msg} (status {status})" if what else f"{msg} (status {status})")


class Opts(ctypes.Structure):
    _fields_ = [("cauchy_mode", ctypes.c_int), ("max_secular_iter", ctypes.c_int),
                ("far_field", ctypes.c_int), ("device", ctypes.c_int),
                ("batch_hint", ctypes.c_int64), ("tune_cache", ctypes.c_char_p)]


_lib = None


def load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build the CUDA library first "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i64, c_int, c_double = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    sig = {
        "dctplus_plan": (c_int, [ctypes.POINTER(vp), c_int, vp, c_double, ctypes.POINTER(Opts)]),
        "dctplus_destroy": (None, [vp]),
        "dctplus_plan_inspect": (c_int, [vp, vp, vp, vp, vp, vp, vp]),
        "dctplus_plan_size": (c_int, [vp]),
        "dctplus_plan_cauchy_mode": (c_int, [vp]),
        "dctplus_plan_far_field": (c_int, [vp]),
        "dctplus_execute": (c_int, [vp, c_int, vp, i64, vp, i64, i64, vp]),
        "dctplus_execute_host": (c_int, [vp, c_int, vp, vp, i64, vp]),
        "dctplus_execute_noalloc": (c_int, [vp, vp, i64, vp, i64, i64, vp]),
        "dctplus_execute_pruned": (c_int, [vp, c_int, vp, i64, vp, i64, i64, c_int, c_int, vp]),
        "dctplus_execute_multi": (c_int, [vp, c_int, vp, i64, vp, i64, i64, vp]),
        "dctplus_backward": (c_int, [vp, vp, i64, vp, i64, vp, i64, vp, vp, i64, vp]),
        "dctplus_group_create": (c_int, [ctypes.POINTER(vp), c_int, vp]),
        "dctplus_group_destroy": (None, [vp]),
        "dctplus_execute_group": (c_int, [vp, vp, vp, vp, c_int, vp]),
        "dctplus_execute_group_host": (c_int, [vp, vp, vp, i64, vp, c_int, vp]),
        "dctplus_sync_check": (c_int, [vp]),
        "dctplus_launch_count": (i64, []),
        "dctplus_status_string": (ctypes.c_char_p, [c_int]),
        "dctplus_trace_begin": (c_int, [vp]),
        "dctplus_autotune": (c_int, [c_int, vp, c_double, i64, ctypes.c_char_p, vp, vp, vp, vp]),
        "dctplus_tune_lookup": (c_int, [ctypes.c_char_p, ctypes.c_char_p, c_int, i64, vp, vp]),
        "dctplus_tune_record": (c_int, [ctypes.c_char_p, ctypes.c_char_p, c_int, i64, c_int, c_int, c_double, vp]),
        "dctplus_trace_end": (c_int, [vp, vp, vp, vp, vp, c_int]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _status_string(status: int) -> str:
    try:
        return load().dctplus_status_string(int(status)).decode()
    except Exception:  # library not loadable: describe the code only
        return f"status {status}"


def check(status: int, what: str = "") -> None:
    if status != OK:
        raise DctPlusError(status, what)
