"""ctypes binding of libflash.so (include/flash.h).  Argument marshalling only:
every step of the method runs in the CUDA library; there is no CPU fallback.
A missing library or a machine without CUDA raises immediately."""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

_LOCK = threading.Lock()
_LIB = None

FLASH_OK, FLASH_EINVAL, FLASH_ENOMEM, FLASH_ECUDA, FLASH_ETIMEOUT, FLASH_EDATA = range(6)
DEVERR_COL_RANGE, DEVERR_ROW_PTR, DEVERR_TIMEOUT = 1, 2, 4


class FlashError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} (status {code})")


class Params(ctypes.Structure):
    _fields_ = [("K", ctypes.c_uint32), ("L", ctypes.c_uint32), ("R", ctypes.c_uint32),
                ("range_bits", ctypes.c_uint32), ("seed", ctypes.c_uint64), ("densify", ctypes.c_uint32),
                ("share_pool", ctypes.c_uint32)]


class Csr(ctypes.Structure):
    _fields_ = [("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p), ("val", ctypes.c_void_p),
                ("n_rows", ctypes.c_int64), ("nnz", ctypes.c_int64), ("dim", ctypes.c_int64)]


class IndexInfo(ctypes.Structure):
    _fields_ = [("params", Params), ("n_rows", ctypes.c_int64), ("bytes", ctypes.c_int64)]


def lib():
    """The loaded library.  Raises if it is not built (call paper_1709_01190_gb300.build())."""
    global _LIB
    if _LIB is not None:
        return _LIB
    with _LOCK:
        if _LIB is not None:
            return _LIB
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"CUDA library not built ({_build.LIB}); run paper_1709_01190_gb300.build()")
        L = ctypes.CDLL(_build.LIB)
        P, I64, I32, U32, VP = ctypes.POINTER(Params), ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32, ctypes.c_void_p
        C = ctypes.POINTER(Csr)
        sig = {
            "flash_hash": ([P, C, VP, VP], ctypes.c_int),
            "flash_keys": ([P, C, VP, VP], ctypes.c_int),
            "flash_build": ([P, C, ctypes.POINTER(VP), VP], ctypes.c_int),
            "flash_query": ([VP, C, I32, VP, VP, VP, VP], ctypes.c_int),
            "flash_add": ([VP, C, VP], ctypes.c_int),
            "flash_knn_graph": ([P, C, I32, VP, VP, VP], ctypes.c_int),
            "flash_query_noalloc": ([VP, C, I32, VP, VP, VP, VP], ctypes.c_int),
            "flash_knn_graph_plain": ([P, C, I32, VP, VP, VP], ctypes.c_int),
            "flash_eval_quality": ([C, VP, I64, VP, I32, VP, VP, VP, VP], ctypes.c_int),
            "flash_knn_graph_host": ([P, VP, VP, I64, I64, I32, VP, VP, VP], ctypes.c_int),
            "flash_index_free": ([VP], None),
            "flash_index_get_info": ([VP, ctypes.POINTER(IndexInfo)], ctypes.c_int),
            "flash_index_export": ([VP, VP, VP, VP], ctypes.c_int),
            "flash_device_error": ([VP], U32),
            "flash_set_scratch_budget": ([ctypes.c_size_t], ctypes.c_size_t),
            "flash_knn_graph_scratch_bytes": ([P, I64], ctypes.c_size_t),
            "flash_query_scratch_bytes": ([P, I64], ctypes.c_size_t),
            "flash_enable_phase_timing": ([ctypes.c_int], ctypes.c_int),
            "flash_phase_times": ([ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_char_p), ctypes.c_int],
                                  ctypes.c_int),
            "flash_last_launch_count": ([], ctypes.c_int),
            "flash_strerror": ([ctypes.c_int], ctypes.c_char_p),
            "flash_version": ([], ctypes.c_char_p),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _LIB = L
        return L


def strerror(code: int) -> str:
    try:
        return lib().flash_strerror(code).decode()
    except RuntimeError:
        return {0: "ok", 1: "invalid argument", 2: "out of memory", 3: "CUDA error", 4: "timeout",
                5: "invalid data"}.get(code, "unknown")


def check(code: int, what: str) -> None:
    if code != 0:
        raise FlashError(code, what)
