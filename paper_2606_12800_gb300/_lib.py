"""ctypes binding of libfr.so: one Python callable per C entry point, same
names as in ``include/fr.h``.  Argument marshalling only -- every step of the
computation runs in the library's CUDA kernels.

Loading fails loudly (``RuntimeError``) when the library is missing or cannot
be built; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("FR_LIB_PATH") or os.path.join(_HERE, "_build", "libfr.so")

# status codes (fr_status)
FR_OK = 0
FR_ERR_INVALID_ARG = 1
FR_ERR_CUDA = 2
FR_ERR_WORKSPACE = 3
FR_ERR_NONFINITE = 4
FR_ERR_NO_PROGRESS = 5
FR_ERR_UNSUPPORTED = 6

# flags
FR_EDGE_SINK = 0x0
FR_EDGE_ROUTE = 0x1
FR_D8_STEEPEST = 0x0
FR_D8_LOWEST = 0x2
FR_D4 = 0x8
FR_DINF = 0x10
FR_GLOBAL_WALKERS = 0x20
FR_GLOBAL_SKELETON = 0x40
FR_WEIGHTS_IN_WORKSPACE = 0x80
FR_SINK_SUMS_IN_WORKSPACE = 0x100
FR_CHECK_FINITE = 0x4
FR_SINK = 0xFF

FR_ROUTING_D8 = 0
FR_ROUTING_MFD = 1

FR_OP_RECEIVERS = 0
FR_OP_ACCUMULATE = 1
FR_OP_ADJOINT = 2
FR_OP_MASS_BALANCE = 3
FR_OP_ROUTE = 4
FR_OP_MFD = 5
FR_OP_FILL = 6

# Largest grid (cells) fr_route_d8_noalloc accepts.
FR_NOALLOC_MAX_CELLS = 1 << 20

# Every symbol include/fr.h declares (checked by the test-suite).
EXPORTS = (
    "fr_receivers_d8", "fr_receivers_mfd", "fr_accumulate", "fr_route_d8", "fr_route_mfd",
    "fr_route_adjoint", "fr_mass_balance", "fr_route_batch", "fr_batch_workspace_size",
    "fr_batch_autotune", "fr_route_d8_noalloc", "fr_accumulate_richardson", "fr_fill",
    "fr_workspace_size", "fr_get_status", "fr_status_string", "fr_version",
    "fr_receiver_index", "fr_set_wait_limit",
)


class FrError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__("%s failed: %s (status %d)" % (where, status_string(status), status))


class fr_routing(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32), ("reserved", ctypes.c_int32),
        ("nx", ctypes.c_int64), ("ny", ctypes.c_int64),
        ("dir", ctypes.c_void_p), ("mask", ctypes.c_void_p), ("dem", ctypes.c_void_p),
        ("dx", ctypes.c_double), ("p", ctypes.c_double),
        ("flags", ctypes.c_uint32), ("reserved2", ctypes.c_uint32),
    ]


class fr_tile(ctypes.Structure):
    _fields_ = [
        ("dem", ctypes.c_void_p), ("rain", ctypes.c_void_p), ("w_out", ctypes.c_void_p),
        ("w_lo_out", ctypes.c_void_p), ("area_out", ctypes.c_void_p),
        ("route_out", ctypes.c_void_p), ("nx", ctypes.c_int64), ("ny", ctypes.c_int64),
        ("dx", ctypes.c_double),
    ]


_lib = None
_lock = threading.Lock()


def load(build_if_missing: bool = True):
    """Loads libfr.so (building it in-tree with nvcc if it is missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            if not build_if_missing:
                raise RuntimeError("libfr.so not built: run python -m paper_2606_12800_gb300.build")
            from . import build as _build
            _build.build()
        L = ctypes.CDLL(LIB_PATH)
        P, I64, I32, U32, D = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32,
                               ctypes.c_double)
        S = ctypes.c_int
        sig = {
            "fr_receivers_d8": (S, [P, I64, I64, D, U32, P, P, P]),
            "fr_receivers_mfd": (S, [P, I64, I64, D, D, U32, P, P, P, P]),
            "fr_accumulate": (S, [ctypes.POINTER(fr_routing), P, P, P, P, P, ctypes.c_size_t, P]),
            "fr_fill": (S, [P, I64, I64, U32, P, I32, ctypes.POINTER(ctypes.c_int32), P,
                            ctypes.c_size_t, P]),
            "fr_accumulate_richardson": (S, [ctypes.POINTER(fr_routing), P, P, P, I32, I32,
                                             ctypes.POINTER(ctypes.c_int32), P, ctypes.c_size_t, P]),
            "fr_route_d8": (S, [P, I64, I64, D, U32, P, P, P, P, P, P, ctypes.c_size_t, P]),
            "fr_route_mfd": (S, [P, I64, I64, D, D, U32, P, P, P, P, P, ctypes.c_size_t, P]),
            "fr_route_d8_noalloc": (S, [P, I64, I64, D, U32, P, P, P, P, P, P]),
            "fr_route_adjoint": (S, [ctypes.POINTER(fr_routing), P, P, P, P, P, P, ctypes.c_size_t, P]),
            "fr_mass_balance": (S, [ctypes.POINTER(fr_routing), P, P, P, P, P, P, ctypes.c_size_t, P]),
            "fr_route_batch": (S, [ctypes.POINTER(fr_tile), P, I32, I32, D, U32, P, ctypes.c_size_t, P]),
            "fr_batch_workspace_size": (ctypes.c_size_t, [ctypes.POINTER(fr_tile), I32, I32, U32]),
            "fr_batch_autotune": (S, [ctypes.POINTER(fr_tile), P, I32, I32, D, U32, P, ctypes.c_size_t, P]),
            "fr_workspace_size": (ctypes.c_size_t, [I32, I64, I64, U32]),
            "fr_get_status": (S, [P, ctypes.c_size_t, P]),
            "fr_status_string": (ctypes.c_char_p, [S]),
            "fr_version": (I32, []),
            "fr_receiver_index": (S, [P, I64, I64, I32, P, P]),
            "fr_set_wait_limit": (ctypes.c_uint64, [ctypes.c_uint64]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
        return _lib


def status_string(status: int) -> str:
    try:
        return load().fr_status_string(status).decode()
    except Exception:  # pragma: no cover
        return "status %d" % status


def check(status: int, where: str) -> None:
    if status != FR_OK:
        raise FrError(status, where)


def __getattr__(name):  # fr_* attribute access forwards to the library
    if name.startswith("fr_"):
        return getattr(load(), name)
    raise AttributeError(name)
