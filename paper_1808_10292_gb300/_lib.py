"""ctypes binding of libisort.so: argument marshalling only.

Every step of a sort runs in the library's CUDA kernels. There is no CPU
fallback: if the library is missing or cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import re

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libisort.so")
HEADER = os.path.join(os.path.dirname(PKG), "include", "isort.h")

STATUS = {0: "ISORT_OK", 1: "ISORT_EINVAL", 2: "ISORT_ENOMEM", 3: "ISORT_ECUDA",
          4: "ISORT_ETIMEOUT", 5: "ISORT_EUNSUPPORTED"}
OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EUNSUPPORTED = range(6)
DEBUG_SPIN_LIMIT, DEBUG_STALL_TILE, DEBUG_KERNEL_TIMING = 1, 2, 3
DEBUG_PREFETCH_TILES = 6
DEBUG_CHECK_MODE = 7
DEBUG_HOST_COPY = 8
NOALLOC_MAX_KEYS = 1 << 20
NET_BTN, NET_OET = 0, 1

_lib = None


class IsortError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what} failed: {STATUS.get(status, status)}")


def _sig(lib):
    vp, i64, i32, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_size_t
    sigs = {
        "isort_keys": [vp, i64, i32, i32, vp],
        "isort_pairs": [vp, vp, i64, i32, i32, i32, vp],
        "isort_keys_host": [vp, vp, i64, i32, i32, vp],
        "isort_pairs_host": [vp, vp, vp, vp, i64, i32, i32, i32, vp],
        "isort_segmented": [vp, vp, vp, i64, i64, i32, i32, i32, vp],
        "isort_workspace_size": [i64, i32, i32, i32, ctypes.POINTER(sz)],
        "isort_set_workspace": [vp, sz, vp],
        "isort_stream_status": [vp],
        "isort_release_workspaces": [],
        "isort_tune_set": [i32, i32, i32, i32],
        "isort_tune_num_variants": [i32, i32, i32],
        "isort_tune_describe": [i32, i32, i32, i32, ctypes.POINTER(i32), ctypes.POINTER(i32)],
        "isort_debug_set": [i32, i64],
        "isort_keys_noalloc": [vp, i64, vp, vp],
        "isort_tune_segmented": [i32, i32, i64],
        "isort_tune_segmented_network": [i32, i32, i32],
        "isort_segmented_workspace_size": [i64, i64, i32, i32, ctypes.POINTER(sz)],
        "isort_sample_sort": [vp, vp, i64, i32, i32, i32, i32, ctypes.c_uint64, vp, vp],
        "isort_sample_sort_workspace_size": [i64, i32, i32, i32, i32, ctypes.POINTER(sz)],
        "isort_gsd_sort": [vp, vp, i64, i32, i32, i32, i32, vp, vp],
        "isort_gsd_sort_workspace_size": [i64, i32, i32, i32, i32, ctypes.POINTER(sz)],
        "isort_tune_auto": [i32, i32, i32, i32, i32],
        "isort_tune_resolve": [i64, i32, i32, i32, ctypes.POINTER(i32), ctypes.POINTER(i32)],
    }
    for name, args in sigs.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.isort_debug_kernel_times.argtypes = [ctypes.POINTER(ctypes.c_char_p),
                                             ctypes.POINTER(ctypes.c_float), i32]
    lib.isort_debug_kernel_times.restype = i32
    lib.isort_debug_launch_count.argtypes = []
    lib.isort_debug_launch_count.restype = ctypes.c_int64
    lib.isort_debug_workspace_bytes.argtypes = []
    lib.isort_debug_workspace_bytes.restype = ctypes.c_int64
    lib.isort_strerror.argtypes = [ctypes.c_int]
    lib.isort_strerror.restype = ctypes.c_char_p
    return lib


def load():
    """The loaded library; raises if libisort.so has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it with "
                "`python -m paper_1808_10292_gb300.build` (needs nvcc); there is no CPU fallback")
        _lib = _sig(ctypes.CDLL(LIB_PATH))
    return _lib


def declared_symbols() -> list[str]:
    """Function names declared in include/isort.h."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(isort_[a-z0-9_]+)\s*\(", text)))


def check(status: int, what: str):
    if status != OK:
        raise IsortError(status, what)
