"""ctypes binding of libsfft (include/sfft.h): argument marshalling only.

Every step of the sparse FFT runs in the library's CUDA kernels; this module turns torch
tensors (device memory, streams) and numpy arrays (host memory) into the C ABI's plain
pointers and back.  There is no CPU fallback: if the library cannot be loaded, every call
raises."""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

SFFT_OK = 0
SFFT_PENDING = 1
SFFT_INCOMPLETE = 2
SFFT_EINVAL = -1
SFFT_ENOMEM = -2
SFFT_ECUDA = -3
SFFT_ETIMEDOUT = -4
SFFT_EADMIT = -5
SFFT_ENOTFOUND = -6
SFFT_EBUSY = -7
SFFT_ETOOBIG = -8

C64, C128 = 0, 1
PREC_FP64, PREC_FP32 = 0, 1
LOCATE_ARG, LOCATE_ML, LOCATE_KAY = 0, 1, 2
DECODER_PEEL, DECODER_ONESHOT, DECODER_DSFFT = 0, 1, 2


class SfftError(RuntimeError):
    def __init__(self, code: int, what: str):
        lib = load()
        msg = lib.sfft_error_string(code).decode()
        if code == SFFT_ECUDA:
            msg += f" ({lib.sfft_last_cuda_error().decode()})"
        super().__init__(f"{what}: {msg} [{code}]")
        self.code = code


class Opts(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("locate", ctypes.c_int32), ("max_rounds", ctypes.c_int32),
                ("max_batch", ctypes.c_int32), ("max_tile", ctypes.c_int32),
                ("noise_var", ctypes.c_double), ("a_min", ctypes.c_double),
                ("eta", ctypes.c_double), ("c0", ctypes.c_double), ("c1", ctypes.c_double),
                ("wait_limit_log2", ctypes.c_int32), ("fault_inject", ctypes.c_int32),
                ("decode_ctas", ctypes.c_int32), ("decoder", ctypes.c_int32),
                ("oneshot_am", ctypes.c_int32), ("kay_m", ctypes.c_int32),
                ("noise_auto", ctypes.c_int32), ("host_gather", ctypes.c_int32),
                ("oneshot_method", ctypes.c_int32), ("dft_fma_only", ctypes.c_int32),
                ("peel_atomic", ctypes.c_int32), ("overlap_gather", ctypes.c_int32),
                ("classify_lanes", ctypes.c_int32), ("arg_mode", ctypes.c_int32),
                ("ml_tc_tf32", ctypes.c_int32)]


_lock = threading.Lock()
_lib = None

EXPORTS = {
    # name: (restype, argtypes)
    "sfft_opts_default": (None, [ctypes.POINTER(Opts)]),
    "sfft_plan_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int64,
                                        ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                        ctypes.c_int32, ctypes.c_void_p, ctypes.POINTER(Opts)]),
    "sfft_plan_destroy": (None, [ctypes.c_void_p]),
    "sfft_plan_num_bins": (ctypes.c_int64, [ctypes.c_void_p]),
    "sfft_plan_noise_var": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]),
    "sfft_execute": (ctypes.c_int, [ctypes.c_void_p] * 6),
    "sfft_execute_batch": (ctypes.c_int, [ctypes.c_int32] + [ctypes.c_void_p] * 6),
    "sfft_bucketize": (ctypes.c_int, [ctypes.c_void_p] * 4),
    "sfft_decode_bins": (ctypes.c_int, [ctypes.c_void_p] * 6),
    "sfft_plan_set_profiling": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "sfft_plan_profile": (ctypes.c_int, [ctypes.c_void_p] * 4 + [ctypes.c_int]),
    "sfft_server_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_size_t,
                                          ctypes.c_int32]),
    "sfft_server_reserve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32]),
    "sfft_submit": (ctypes.c_int, [ctypes.c_void_p] * 6 + [ctypes.POINTER(ctypes.c_uint64)]),
    "sfft_poll": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64,
                                 ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double)]),
    "sfft_server_drain": (ctypes.c_int, [ctypes.c_void_p]),
    "sfft_server_destroy": (None, [ctypes.c_void_p]),
    "sfft_bucketize_static": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p,
                                             ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32,
                                             ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_void_p]),
    "sfft_autotune": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                     ctypes.c_int32, ctypes.c_void_p, ctypes.POINTER(Opts),
                                     ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.POINTER(Opts), ctypes.POINTER(ctypes.c_double)]),
    "sfft_autotune_cache": (ctypes.c_int, [ctypes.c_char_p]),
    "sfft_error_string": (ctypes.c_char_p, [ctypes.c_int]),
    "sfft_last_cuda_error": (ctypes.c_char_p, []),
}


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libsfft.so (building it with nvcc first when it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if build_if_missing and not _build.up_to_date():
                path = _build.build()
            if not os.path.exists(path):
                raise RuntimeError(f"libsfft not built: {path} missing")
            lib = ctypes.CDLL(path)
            for name, (res, args) in EXPORTS.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def check(code: int, what: str) -> int:
    if code < 0:
        raise SfftError(code, what)
    return code


def ptr_of(obj) -> int:
    """Raw address of a torch tensor (device or host) or a numpy array (host)."""
    if obj is None:
        return 0
    if isinstance(obj, np.ndarray):
        if not obj.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be contiguous")
        return obj.ctypes.data
    if hasattr(obj, "data_ptr"):
        if not obj.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return obj.data_ptr()
    if isinstance(obj, int):
        return obj
    raise TypeError(f"cannot take the address of {type(obj)}")


def stream_handle(stream) -> int:
    if stream is None:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
        return 0
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream
