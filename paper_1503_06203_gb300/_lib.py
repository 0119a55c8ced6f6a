"""ctypes view of the C ABI in include/xengine.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_libxengine.so")

CORR_OK = 0
CORR_EINVAL = -1
CORR_ENOMEM = -2
CORR_ECUDA = -3
CORR_EOVERFLOW = -4
CORR_ETIMEOUT = -5
CORR_EBUSY = -6
CORR_MAX_N = 16384
CORR_OPT_PRODUCT = 1
CORR_OPT_SPLIT = 2
CORR_OPT_MMA_STEPS = 3
CORR_MAX_SAMPLES = 16777215
CORR_BATCH_ALONE_WAVES = 4

# (name, restype, argtypes) for every symbol include/xengine.h declares
_vp, _i32, _i64, _int = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_int
SIGNATURES = [
    ("corr_create", _vp, [_i32, _i32, _i32]),
    ("corr_create_ex", _vp, [_i32, _i32, _i32, _vp]),
    ("corr_create_bands", _vp, [_i32, _i32, _i32, _i32, _i32]),
    ("corr_bands", _int, [_vp, _vp, _vp, _vp]),
    ("corr_accumulate", _int, [_vp, _vp, _vp]),
    ("corr_accumulate_host", _int, [_vp, _vp, _vp]),
    ("corr_readout", _int, [_vp, _vp, _int, _vp]),
    ("corr_readout_host", _int, [_vp, _vp, _int, _vp]),
    ("corr_readout_async", _int, [_vp, _vp, _vp]),
    ("corr_readout_host_async", _int, [_vp, _vp, _vp]),
    ("corr_reset", _int, [_vp, _vp]),
    ("corr_accumulate_batch", _int, [_vp, _vp, _int, _vp]),
    ("corr_accumulate_batch_ex", _int, [_vp, _vp, _vp, _int, _vp]),
    ("corr_accumulate_gated", _int, [_vp, _int, _vp, _i32, _i32, _i32, _vp]),
    ("corr_shift_lags", _int, [_vp, _vp, _i32, _i32, _i32, _vp, _vp]),
    ("corr_set_option", _int, [_vp, _int, _i64]),
    ("corr_get_option", _i64, [_vp, _int]),
    ("corr_synchronize", _int, [_vp, _i64]),
    ("corr_status", _int, [_vp]),
    ("corr_samples", _i64, [_vp]),
    ("corr_kernel_launches", _i64, [_vp]),
    ("corr_dims", _int, [_vp, _vp, _vp, _vp]),
    ("corr_last_error", ctypes.c_char_p, []),
    ("corr_destroy", None, [_vp]),
    ("corr_plan_tiles", _i64, [_i32, _i32, _vp, _vp, _i64]),
    ("corr_plan_schedule", _i64, [_i32, _i32, _i32, _i32, _vp, _i64, _vp]),
    ("corr_effective_ops", ctypes.c_double, [_i32, _i32, _i32]),
    ("corr_correlate_noalloc", _int, [_vp, _i32, _i32, _i32, _vp, _vp, _vp]),
    ("corr_selftest_wait_timeout", _int, [_i32, _vp]),
    # microbenchmarks (include/xengine_peaks.h)
    ("xe_peak_imma_s8", ctypes.c_double, [_int, _vp]),
    ("xe_peak_dp4a", ctypes.c_double, [_int, _vp]),
    ("xe_peak_imma_dp4a", ctypes.c_double, [_int, _int, _vp, _vp, _vp]),
]

_lib = None


class XEngineError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


def lib():
    """Load the in-tree CUDA library; fail loudly if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"the CUDA library {LIB_PATH} is not built; run `python -m paper_1503_06203_gb300.builder` "
                "(there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def last_error() -> str:
    return (lib().corr_last_error() or b"").decode()


def check(rc: int) -> int:
    if rc != CORR_OK:
        raise XEngineError(rc, last_error())
    return rc
