"""ctypes binding of libgb300fft.so: argument marshalling only.

Every function here forwards to the C ABI declared in include/gb300fft.h with
the same name.  There is no fallback: if the library is missing this module
raises, and the Python API refuses tensors that are not on a CUDA device.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libgb300fft.so")

FFT_FORWARD = -1
FFT_INVERSE = 1
FFT_PREC_FP32 = 0
FFT_PREC_SPLIT_FP16_TC = 1
FFT_OK = 0
FFT_ERR_INVALID_SIZE = -1
FFT_ERR_INVALID_ARG = -2
FFT_ERR_ALLOC = -3
FFT_ERR_CUDA = -4
FFT_ERR_UNSUPPORTED = -5
FFT_ERR_TIMEOUT = -6

# (name, restype, argtypes) for every symbol the header declares
_P = ctypes.c_void_p
_I = ctypes.c_int
_F = ctypes.c_float
_LL = ctypes.c_longlong
SIGNATURES = [
    ("fft_plan_create", _P, [_I, _I, _I, _I, _I]),
    ("fft_plan_create_columns", _P, [_I, _I, _I, _I, _I]),
    ("fft_slab_pack", _I, [_P, _P, _I, _I, _I, _I, _P]),
    ("fft_slab_unpack", _I, [_P, _P, _I, _I, _I, _I, _P]),
    ("fft_execute", _I, [_P, _P, _P, _P]),
    ("fft_execute_host", _I, [_P, _P, _P, _P]),
    ("fft_backward", _I, [_P, _P, _P, _P]),
    ("fft_backward_weighted", _I, [_P, _P, _P, _F, _P, _P]),
    ("fft_backward_weighted_dev", _I, [_P, _P, _P, _P, _F, _P, _P]),
    ("fft_weighted_power", _I, [_P, _P, _P, _P, _P]),
    ("fft_weighted_power_parts", _I, [_P]),
    ("fft_weighted_power_adjoint", _I, [_P, _P, _P, _P, _P, _P]),
    ("fft_weighted_power_adjoint_parts", _I, [_P]),
    ("fft_backward_rows_scaled", _I, [_P, _P, _P, _F, _P, _P]),
    ("fft_plan_destroy", _I, [_P]),
    ("fft_last_error", _I, []),
    ("fft_error_string", ctypes.c_char_p, [_I]),
    ("fft_plan_create_ragged", _P, [_I, ctypes.POINTER(_I), ctypes.POINTER(_I), _I, _I]),
    ("fft_ragged_offset", _I, [_P, _I, ctypes.POINTER(_LL)]),
    ("fft_execute_ragged", _I, [_P, _P, _P, _P]),
    ("fft_execute_ragged_loop", _I, [_P, _P, _P, _P]),
    ("fft_execute_ragged_noalloc", _I, [_I, ctypes.POINTER(_I), ctypes.POINTER(_I), _I, _P, _P, _P, _P]),
    ("fft_plan_status", _I, [_P, _P]),
    ("fft_plan_set_pass_events", _I, [_P, _P, _P, _P]),
    ("fft_plan_describe", _I, [_P, ctypes.c_char_p, _I]),
    ("fft_plan_autotune", _I, [_P, _P]),
    ("fft_debug_reorder_map", _I, [_I, _I, _P, _P]),
    ("fft_debug_radices", _I, [_I, _I, ctypes.POINTER(_I)]),
    ("fft_debug_row_variant", _I, [_I, _I, _I, ctypes.POINTER(_I)]),
    ("fft_debug_tc_layout", _I, [_I, _I, ctypes.POINTER(ctypes.c_longlong)]),
    ("fft_debug_mixed_plan", _I, [_I, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    ("fft_debug_root", _I, [_I, _I, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)]),
    ("fft_debug_last_cuda_error", ctypes.c_char_p, []),
    ("fft_version", ctypes.c_char_p, []),
]

_lib = None


class FFTError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = int(code)
        msg = error_string(code) if _lib is not None else f"error {code}"
        super().__init__(f"{what}: {msg} (code {code})" if what else f"{msg} (code {code})")


def load(path: str = LIB_PATH):
    """Load libgb300fft.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            f"{path} is missing: build it with __graft_entry__.build() or "
            "`python -m paper_2506_15437_gb300.build` (needs nvcc)")
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def error_string(code: int) -> str:
    return load().fft_error_string(int(code)).decode()


def check(rc: int, what: str = ""):
    if rc != FFT_OK:
        raise FFTError(rc, what)
    return rc
