"""ctypes declarations of include/projection.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libprojection.so")

PROJ_OK = 0
PROJ_EINVAL = -1
PROJ_ENOMEM = -2
PROJ_ECAPACITY = -3
PROJ_ECUDA = -4
PROJ_ETIMEOUT = -5
PROJ_EBADCHAR = -6
PROJ_ENOTSUP = -7
PROJ_EM_FP32 = 0
PROJ_EM_BF16_SPLIT = 1

STATUS_NAMES = {0: "PROJ_OK", -1: "PROJ_EINVAL", -2: "PROJ_ENOMEM", -3: "PROJ_ECAPACITY",
                -4: "PROJ_ECUDA", -5: "PROJ_ETIMEOUT", -6: "PROJ_EBADCHAR", -7: "PROJ_ENOTSUP"}

# every function declared in include/projection.h, with its ctypes signature
P = ctypes.c_void_p
i32, i64, u64, f32 = ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_float


class ProjectionResult(ctypes.Structure):
    _fields_ = [("status", i32), ("t", i32), ("l", i32), ("k", i32), ("s", i32), ("m", i32),
                ("n_candidates", i64), ("n_members", i64), ("win_index", i64),
                ("win_trial", i32), ("win_key", ctypes.c_uint32), ("loglik", ctypes.c_double),
                ("score", i32), ("pwm", ctypes.POINTER(ctypes.c_float)),
                ("consensus", ctypes.c_char_p), ("sites", ctypes.POINTER(ctypes.c_int32)),
                ("n_refined", i64)]


SIGNATURES = {
    "projection_last_error": ([], ctypes.c_char_p),
    "projection_packed_words": ([i64], i64),
    "projection_default_params": ([i32, P, i32, i32, P, P, P], i32),
    "projection_pack": ([P, i64, P, P, P], i32),
    "projection_background": ([P, i64, P, P], i32),
    "projection_positions": ([u64, i64, i64, i32, i32, P, P], i32),
    "trial_hash": ([P, P, i32, i32, i32, i32, u64, i64, i64, P, P, P, i64, i64, P, P, P, P, P,
                    P, P], i32),
    "trial_hash_noalloc": ([P, P, i32, i32, i32, i32, u64, i64, i64, P, P, P, i64, i64, P, P, P,
                            P, P, P, P], i32),
    "trial_hash_top": ([P, P, i32, i32, i32, i32, u64, i64, i64, i64, P, P, P, P, P, P, P, P],
                       i32),
    "theta0_build": ([P, P, i32, i32, P, P, i64, f32, P, P], i32),
    "em_refine": ([P, P, i32, i32, P, P, i64, i32, f32, i32, P, P, P, P], i32),
    "em_refine_zoops": ([P, P, i32, i32, P, P, i64, i32, f32, i32, ctypes.c_double, P, P, P,
                         P], i32),
    "projection_find_packed_zoops": ([P, P, i32, i32, i32, i32, i32, i32, u64, i32, f32, i32,
                                      ctypes.c_double, i64, ctypes.POINTER(ProjectionResult), P],
                                     i32),
    "projection_ex2_peak": ([P, P], i32),
    "projection_find_protein": ([P, P, i32, i32, i32, i32, i32, u64, i32, f32,
                                 ctypes.POINTER(ProjectionResult), P], i32),
    "projection_finalize": ([P, P, i32, i32, P, P, P, i64, P, P, P, P, P], i32),
    "projection_find": ([P, P, i32, i32, i32, i32, i32, i32, u64, i32, f32, i32,
                         ctypes.POINTER(ProjectionResult), P], i32),
    "projection_find_packed": ([P, P, i32, i32, i32, i32, i32, i32, u64, i32, f32, i32,
                                ctypes.POINTER(ProjectionResult), P], i32),
    "projection_find_top": ([P, P, i32, i32, i32, i32, i32, i32, u64, i32, f32, i32, i64,
                             ctypes.POINTER(ProjectionResult), P], i32),
    "projection_find_packed_top": ([P, P, i32, i32, i32, i32, i32, i32, u64, i32, f32, i32, i64,
                                    ctypes.POINTER(ProjectionResult), P], i32),
    "projection_find_batch": ([P, P, P, i32, P, P, P, P, P, P, i32, f32, i32,
                               ctypes.POINTER(ProjectionResult), P], i32),
    "projection_result_free": ([ctypes.POINTER(ProjectionResult)], None),
    "projection_selftest_wait": ([i64, P], i32),
    "projection_hist_peak": ([i32, P, P], i32),
    "trial_hash_allpairs": ([P, P, i32, i32, i32, i32, u64, i64, i64, i64, i64, P, P, P, P, P, P,
                             P], i32),
    "projection_params_batch": ([i32, P, P, P, P, P, P, P, P, ctypes.c_double, P], i32),
    "projection_trace_enable": ([i32], i32),
    "projection_trace_read": ([ctypes.c_char_p, P, P], i32),
}

_lock = threading.Lock()
_lib = None


class ProjectionError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def lib():
    """The loaded CUDA library.  Raises if it has not been built: there is no
    other implementation to fall back to."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"{LIB_PATH} is missing: build it with "
                    "`python -c 'import __graft_entry__ as g; g.build()'` (needs nvcc)")
            L = ctypes.CDLL(LIB_PATH)
            for name, (args, res) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = res
            _lib = L
    return _lib


def check(status: int) -> None:
    if status != PROJ_OK:
        msg = lib().projection_last_error()
        raise ProjectionError(status, msg.decode() if msg else "")
