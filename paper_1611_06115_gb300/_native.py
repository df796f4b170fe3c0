"""ctypes declarations of libpm's C ABI (include/pm.h).  Marshalling only.

The library must have been built (``paper_1611_06115_gb300.build.build()``);
if it is missing this module raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpm.so")

PM_OK = 0
PM_E_ARG = -1
PM_E_SYMBOL = -2
PM_E_NOMEM = -3
PM_E_OVERFLOW = -4
PM_E_TOO_LARGE = -5
PM_E_TIMEOUT = -6
PM_E_CUDA = -7
PM_TOTAL_ERROR = (1 << 64) - 1
PM_MAX_PATTERN = 1 << 24
PM_MAX_BATCH = 1 << 16

PM_TEXT_UNKNOWN_AS_N = 1

PM_VARIANT_AUTO = 0
PM_VARIANT_PATTERN_SLICED = 1
PM_VARIANT_WINDOW_SLICED = 2
PM_VARIANT_PATTERN_SLICED_2 = 3
PM_VARIANT_ALL_CHUNKS = 4


class NativeLibraryMissing(RuntimeError):
    pass


class PmError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(message)
        self.status = status


class pm_hit(ctypes.Structure):
    _fields_ = [("location", ctypes.c_uint32), ("mismatches", ctypes.c_uint32)]


class pm_batch_options(ctypes.Structure):
    _fields_ = [("group", ctypes.c_int32), ("grid", ctypes.c_int32), ("tiles", ctypes.c_int32),
                ("ws_below", ctypes.c_int32), ("ps1_below", ctypes.c_int32),
                ("ps2_below", ctypes.c_int32)]


class pm_options(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int32), ("grid", ctypes.c_int32),
                ("events", ctypes.POINTER(ctypes.c_void_p)),
                ("batch", ctypes.POINTER(pm_batch_options))]


# Every function include/pm.h declares, with (restype, argtypes).
_vp, _u64, _u32, _i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int32
SIGNATURES = {
    "pm_encode_text": (_i32, [ctypes.c_void_p, _u64, _vp, ctypes.POINTER(_vp)]),
    "pm_text_length": (_u64, [_vp]),
    "pm_text_device_planes": (_i32, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_u64)]),
    "pm_text_free": (None, [_vp]),
    "pm_encode_text_ex": (_i32, [_vp, _u64, _u32, _vp, ctypes.POINTER(_vp)]),
    "pm_text_unknown": (_u64, [_vp]),
    "pm_text_save": (_i32, [_vp, ctypes.c_char_p]),
    "pm_text_load": (_i32, [ctypes.c_char_p, _vp, ctypes.POINTER(_vp)]),
    "pm_text_letter_counts": (_i32, [_vp, ctypes.POINTER(_u64)]),
    "pm_compile_pattern": (_i32, [ctypes.c_char_p, _u32, ctypes.POINTER(_vp)]),
    "pm_pattern_length": (_u32, [_vp]),
    "pm_pattern_unknown": (_u32, [_vp]),
    "pm_pattern_masks": (_i32, [_vp, ctypes.POINTER(_u32), _u64]),
    "pm_pattern_free": (None, [_vp]),
    "pm_search": (_i32, [_vp, ctypes.POINTER(_vp), _u32, ctypes.POINTER(_i32), _vp, _u64, _vp,
                         ctypes.POINTER(_u64), _vp]),
    "pm_search_ex": (_i32, [_vp, ctypes.POINTER(_vp), _u32, ctypes.POINTER(_i32), _vp, _u64, _vp,
                            ctypes.POINTER(_u64), ctypes.POINTER(pm_options), _vp]),
    "pm_search_noalloc": (_i32, [_vp, ctypes.POINTER(_vp), _u32, ctypes.POINTER(_i32), _vp, _u64,
                                 _vp, ctypes.POINTER(_u64), _vp]),
    "pm_set_auto_variants": (_i32, [ctypes.POINTER(_i32), _u32]),
    "pm_get_auto_variants": (_i32, [ctypes.POINTER(_i32), _u32]),
    "pm_batch_create": (_i32, [_vp, ctypes.POINTER(_vp), _u32, ctypes.POINTER(_i32), _u64,
                               ctypes.c_void_p, _vp, ctypes.POINTER(_vp)]),
    "pm_batch_run": (_i32, [_vp, _vp, _vp, _vp]),
    "pm_batch_capacity": (_u64, [_vp]),
    "pm_batch_free": (None, [_vp]),
    "pm_check_bounded_wait": (_i32, [_u64, _i32, ctypes.POINTER(_u32)]),
    "pm_measure_int_pipe": (_i32, [_i32, _u32, ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "pm_status_string": (ctypes.c_char_p, [_i32]),
    "pm_last_error": (ctypes.c_char_p, []),
}

_lock = threading.Lock()
_lib = None


def lib() -> ctypes.CDLL:
    """Load libpm.so (once).  Raises NativeLibraryMissing if it is not built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise NativeLibraryMissing(
                    f"{LIB_PATH} is not built; run paper_1611_06115_gb300.build.build() "
                    "(nvcc, sm_103a). There is no CPU fallback.")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def check(status: int, what: str) -> None:
    if status != PM_OK:
        L = lib()
        detail = L.pm_last_error().decode(errors="replace")
        name = L.pm_status_string(status).decode()
        raise PmError(status, f"{what}: {name}" + (f" ({detail})" if detail else ""))
