"""ctypes binding of libmsrc.so (the C ABI declared in include/msrc.h).

Argument marshalling only: every computation runs in the library's CUDA
kernels. Loading fails loudly when the library cannot be found or built; there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

MAX_TIERS = 4
MAX_MICS = 16

OK, ERR_INVALID_ARG, ERR_UNSUPPORTED, ERR_WORKSPACE, ERR_CUDA, ERR_TIMEOUT, ERR_STATE = range(7)
TILE_DEFAULT = -1  # MSRC_TILE_DEFAULT: the process default tile configuration
TILE_AUTO = -2     # MSRC_TILE_AUTO: chosen from the call's knot layout


class RoomDesc(ctypes.Structure):
    _fields_ = [
        ("dims", ctypes.c_double * 3),
        ("beta", ctypes.c_double * 6),
        ("c", ctypes.c_double),
        ("fs", ctypes.c_double),
        ("max_order", ctypes.c_int32),
        ("n_tiers", ctypes.c_int32),
        ("tier_max_rho", ctypes.c_int32 * 4),
        ("tier_rate_hz", ctypes.c_double * 4),
        ("taps", ctypes.c_int32),
        ("window", ctypes.c_int32),
        ("kaiser_beta", ctypes.c_double),
        ("farrow_order", ctypes.c_int32),
        ("passband", ctypes.c_double),
        ("tier_upsample", ctypes.c_int32 * 4),
        ("upsample_halfwidth", ctypes.c_int32),
        ("delay_model", ctypes.c_int32),
    ]


class TrajDesc(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32),
        ("n_ctrl", ctypes.c_int32),
        ("params", ctypes.c_double * 48),
        ("duration_s", ctypes.c_double),
    ]


class MsrcError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"msrc status {status}: {message}")
        self.status = status


_lock = threading.Lock()
_lib = None

# (name, restype, argtypes) of every entry point declared in include/msrc.h
_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64P = ctypes.POINTER(ctypes.c_int64)
_SZP = ctypes.POINTER(ctypes.c_size_t)
SIGNATURES = [
    ("msrc_create_room", _I32, [ctypes.POINTER(RoomDesc), ctypes.POINTER(_P)]),
    ("msrc_destroy_room", _I32, [_P]),
    ("msrc_set_trajectory", _I32, [_P, ctypes.POINTER(TrajDesc), ctypes.POINTER(ctypes.c_double), _I32]),
    ("msrc_set_array_trajectory", _I32, [_P, ctypes.POINTER(TrajDesc)]),
    ("msrc_trajectory_positions", _I32, [_P, ctypes.POINTER(ctypes.c_double), ctypes.c_int64,
                                         ctypes.POINTER(ctypes.c_double)]),
    ("msrc_suggest_knot_rates", _I32, [_P, ctypes.c_double, _I32, ctypes.POINTER(ctypes.c_double)]),
    ("msrc_suggest_bandlimited_rates", _I32, [_P, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]),
    ("msrc_set_reflection", _I32, [_P, ctypes.POINTER(ctypes.c_double)]),
    ("msrc_workspace_size", _I32, [ctypes.POINTER(_P), _I32, _I64P, _I64P, _SZP, _SZP]),
    ("msrc_synthesize", _I32, [ctypes.POINTER(_P), _I32, ctypes.POINTER(_P), _I64P, ctypes.POINTER(_P),
                               _I64P, _P, ctypes.c_size_t, _P]),
    ("msrc_workspace_size_cfg", _I32, [ctypes.POINTER(_P), _I32, _I64P, _I64P, _I32, _SZP, _SZP]),
    ("msrc_synthesize_cfg", _I32, [ctypes.POINTER(_P), _I32, ctypes.POINTER(_P), _I64P, ctypes.POINTER(_P),
                                   _I64P, _I32, _P, ctypes.c_size_t, _P]),
    ("msrc_synthesize_host", _I32, [ctypes.POINTER(_P), _I32, ctypes.POINTER(_P), _I64P,
                                    ctypes.POINTER(_P), _I64P, _P, ctypes.c_size_t, _P]),
    ("msrc_host_io_bytes", _I32, [ctypes.POINTER(_P), _I32, _I64P, _I64P, _SZP]),
    ("msrc_synthesize_backward", _I32, [ctypes.POINTER(_P), _I32, ctypes.POINTER(_P), _I64P,
                                        ctypes.POINTER(_P), _I64P, ctypes.POINTER(_P),
                                        ctypes.POINTER(_P), ctypes.POINTER(_P), _P, ctypes.c_size_t, _P]),
    ("msrc_synthesize_backward_ex", _I32, [ctypes.POINTER(_P), _I32, ctypes.POINTER(_P), _I64P,
                                           ctypes.POINTER(_P), _I64P, ctypes.POINTER(_P), ctypes.POINTER(_P),
                                           ctypes.POINTER(_P), ctypes.POINTER(_P), _P, ctypes.c_size_t, _P]),
    ("msrc_workspace_errors", _I32, [_P, _P, ctypes.POINTER(ctypes.c_uint32)]),
    ("msrc_test_stall_window_copies", _I32, [ctypes.c_uint32]),
    ("msrc_measure_alu_peaks", _I32, [_P, _P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    ("msrc_room_image_count", _I32, [_P, _I64P, _I64P]),
    ("msrc_room_fit_error", _I32, [_P, ctypes.POINTER(ctypes.c_double)]),
    ("msrc_room_farrow_table", _I32, [_P, _I32, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(_I32)]),
    ("msrc_set_tile_config", _I32, [_I32]),
    ("msrc_tile_configs", _I32, []),
    ("msrc_profile_enable", _I32, [_I32]),
    ("msrc_profile_read", _I32, [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32)]),
    ("msrc_synthesize_noalloc", _I32, [_P, _P, ctypes.c_int64, _P, ctypes.c_int64, _P]),
    ("msrc_noalloc_errors", _I32, [_P, ctypes.POINTER(ctypes.c_uint32)]),
    ("msrc_batch_create", _I32, [ctypes.POINTER(_P), _I32, ctypes.POINTER(_P), _I64P, ctypes.POINTER(_P),
                                 _I64P, _P, ctypes.c_size_t, _P, ctypes.POINTER(_P)]),
    ("msrc_batch_create_cfg", _I32, [ctypes.POINTER(_P), _I32, ctypes.POINTER(_P), _I64P, ctypes.POINTER(_P),
                                     _I64P, _I32, _P, ctypes.c_size_t, _P, ctypes.POINTER(_P)]),
    ("msrc_batch_run", _I32, [_P, _I32, _P]),
    ("msrc_batch_destroy", _I32, [_P]),
    ("msrc_autotune", _I32, [ctypes.POINTER(_P), _I32, ctypes.POINTER(_P), _I64P, ctypes.POINTER(_P), _I64P,
                             _P, ctypes.c_size_t, _P, _I32, ctypes.POINTER(ctypes.c_double),
                             ctypes.POINTER(_I32)]),
    ("msrc_status_string", ctypes.c_char_p, [_I32]),
    ("msrc_last_error", ctypes.c_char_p, []),
]


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Loads libmsrc.so, building it first if it is missing or stale."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if build_if_missing and not _build.up_to_date():
                path = _build.build_library()
            if not os.path.exists(path):
                raise RuntimeError(f"msrc library not found at {path}; run paper_2508_03065_gb300.build")
            lib = ctypes.CDLL(path)
            for name, res, args in SIGNATURES:
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def check(status: int) -> None:
    if status != OK:
        lib = load()
        raise MsrcError(status, lib.msrc_last_error().decode(errors="replace"))


def ptr_array(values):
    arr = (ctypes.c_void_p * len(values))()
    for i, v in enumerate(values):
        arr[i] = v
    return arr


def i64_array(values):
    arr = (ctypes.c_int64 * len(values))()
    for i, v in enumerate(values):
        arr[i] = int(v)
    return arr
