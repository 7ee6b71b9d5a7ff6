"""ctypes view of libfram's C ABI (include/fram.h).  Marshalling only: no computation here.

The library is loaded from paper_2304_08052_gb300/_build/libfram.so.  If it is missing the
import of any function fails with a RuntimeError -- there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# FRAM_LIBRARY selects another build of the same library (the bounds-checking debug build).
LIB_PATH = os.environ.get("FRAM_LIBRARY") or os.path.join(HERE, "_build", "libfram.so")

FRAM_OK = 0
FRAM_EINVAL = -1
FRAM_EWORKSPACE = -2
FRAM_ECUDA = -3
FRAM_EDEVICE = -4

FRAM_DEV_BAD_GEOMETRY = 0x1
FRAM_DEV_CAPACITY = 0x2
FRAM_DEV_NONFINITE = 0x4
FRAM_DEV_BOUNDS = 0x8          # the bounds-checking debug build only

# Every symbol include/fram.h declares (checked by tests/test_abi.py).
EXPORTED = ("fram_version", "fram_last_error", "fram_default_params", "fram_layout", "fram_workspace_size",
            "fram_sample", "fram_synthesize", "fram_synthesize_backward", "fram_status", "fram_prepare",
            "fram_synthesize_prepared", "fram_synthesize_backward_prepared", "fram_synthesize_noalloc",
            "fram_autotune", "fram_sample_backward", "fram_spatialize_workspace_size", "fram_spatialize",
            "fram_measure_alu", "fram_tuned_tile")


class FramParams(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("beta", ctypes.c_double), ("a", ctypes.c_double),
                ("b", ctypes.c_double), ("tau", ctypes.c_double), ("c0", ctypes.c_double),
                ("fs", ctypes.c_double), ("early_pre_ms", ctypes.c_double), ("early_post_ms", ctypes.c_double),
                ("half_len", ctypes.c_int32), ("tile", ctypes.c_int32), ("delay_mode", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class FramScene(ctypes.Structure):
    _fields_ = [("B", ctypes.c_int32), ("S", ctypes.c_int32), ("M", ctypes.c_int32), ("max_len", ctypes.c_int32),
                ("n_vs_total", ctypes.c_int64), ("rir_total", ctypes.c_int64), ("array_radius", ctypes.c_double),
                ("dims", ctypes.c_void_p), ("rt60", ctypes.c_void_p), ("src", ctypes.c_void_p),
                ("mic", ctypes.c_void_p), ("n_vs", ctypes.c_void_p), ("vs_off", ctypes.c_void_p),
                ("rir_len", ctypes.c_void_p), ("rir_off", ctypes.c_void_p), ("room_base", ctypes.c_int64)]


class FramSpatial(ctypes.Structure):
    _fields_ = [("n_samples", ctypes.c_int64), ("n_speech", ctypes.c_int32), ("block", ctypes.c_int32),
                ("chunk_rooms", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class FramError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libfram error {code}: {msg}")
        self.code = code


_lib = None


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libfram is not built ({LIB_PATH} missing); run python -m paper_2304_08052_gb300.build")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, f64, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_uint64
        P, S = ctypes.POINTER(FramParams), ctypes.POINTER(FramScene)
        L.fram_version.restype = ctypes.c_int
        L.fram_last_error.restype = ctypes.c_char_p
        L.fram_default_params.argtypes = [P]
        L.fram_default_params.restype = None
        L.fram_layout.argtypes = [i32, i32, i32, f64, vp, vp, vp, vp, vp]
        L.fram_workspace_size.argtypes = [S, P, ctypes.POINTER(ctypes.c_size_t)]
        L.fram_sample.argtypes = [S, P, u64, vp, vp, vp, vp, vp, vp, vp, ctypes.c_size_t, vp]
        L.fram_synthesize.argtypes = [S, P, vp, vp, vp, vp, vp, vp, vp, ctypes.c_size_t, vp]
        L.fram_synthesize_backward.argtypes = [S, P, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, ctypes.c_size_t,
                                               vp]
        L.fram_sample_backward.argtypes = [S, P, u64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, ctypes.c_size_t, vp]
        SP = ctypes.POINTER(FramSpatial)
        L.fram_spatialize_workspace_size.argtypes = [S, SP, i32, ctypes.POINTER(ctypes.c_size_t)]
        L.fram_spatialize.argtypes = [S, SP, vp, vp, vp, vp, vp, vp, vp, vp, ctypes.c_size_t, vp]
        L.fram_status.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_int32)]
        L.fram_prepare.argtypes = [S, P, vp, vp, vp, vp, ctypes.c_size_t, vp]
        L.fram_synthesize_prepared.argtypes = L.fram_synthesize.argtypes
        L.fram_synthesize_backward_prepared.argtypes = L.fram_synthesize_backward.argtypes
        L.fram_synthesize_noalloc.argtypes = [S, P, vp, vp, vp, vp, vp, vp, vp]
        L.fram_autotune.argtypes = [S, P, vp, vp, vp, vp, vp, vp, ctypes.c_size_t, vp, ctypes.POINTER(ctypes.c_int32)]
        L.fram_measure_alu.argtypes = [i32, i64, ctypes.POINTER(ctypes.c_double), vp]
        L.fram_tuned_tile.argtypes = [S, P, ctypes.POINTER(ctypes.c_int32)]
        for name in EXPORTED[3:]:
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def check(rc: int) -> None:
    if rc != FRAM_OK:
        raise FramError(rc, lib().fram_last_error().decode(errors="replace"))
