"""Python face of the serial C oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers. The GPU library never
imports this package and shares no code with it.

Every function copies its inputs and returns new numpy arrays; nothing here
touches a GPU.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (plain gcc, host only)."""
    if force or not os.path.exists(LIB_PATH) or os.path.getmtime(LIB_PATH) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        tmp = LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-Wall", "-Werror",
                               _SRC, "-o", tmp])
        os.replace(tmp, LIB_PATH)
    return LIB_PATH


def load_library(path: str):
    """Bind a compiled oracle library at `path` (the default one is LIB_PATH)."""
    lib = ctypes.CDLL(path)
    i64, i32, vp = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
    lib.oracle_count_sort_round.argtypes = [vp, vp, vp, vp, i64, i32, i32, i32, i32]
    lib.oracle_radix_sort.argtypes = [vp, vp, i64, i32, i32, i32]
    lib.oracle_segmented_sort.argtypes = [vp, vp, vp, i64, i32, i32, i32]
    lib.oracle_num_passes.argtypes = [i32, i32]
    lib.oracle_gvr_sort.argtypes = [vp, vp, i64, i32, i32, i32, i32, ctypes.c_uint64, vp, vp]
    lib.oracle_gsd_sort.argtypes = [vp, vp, i64, i32, i32, i32, i32, vp, vp]
    for f in (lib.oracle_count_sort_round, lib.oracle_radix_sort, lib.oracle_segmented_sort,
              lib.oracle_num_passes, lib.oracle_gvr_sort, lib.oracle_gsd_sort):
        f.restype = i32
    return lib


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = load_library(LIB_PATH)
    return _lib


def _bits(a: np.ndarray | None) -> int:
    if a is None:
        return 0
    if a.dtype == np.uint32:
        return 32
    if a.dtype == np.uint64:
        return 64
    raise TypeError(f"unsupported dtype {a.dtype}; use uint32 or uint64")


def _ptr(a: np.ndarray | None):
    return None if a is None or a.size == 0 else a.ctypes.data


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def num_passes(key_bits: int, radix_bits: int) -> int:
    return _load().oracle_num_passes(key_bits, radix_bits)


def count_sort_round(keys: np.ndarray, shift: int, digit_bits: int, vals: np.ndarray | None = None,
                     lib=None):
    """One stable count-sort round on digit (k >> shift) & (2^digit_bits - 1)."""
    k_in = np.ascontiguousarray(keys)
    k_out = np.empty_like(k_in)
    v_in = None if vals is None else np.ascontiguousarray(vals)
    v_out = None if v_in is None else np.empty_like(v_in)
    _check((lib or _load()).oracle_count_sort_round(_ptr(k_in), _ptr(k_out), _ptr(v_in), _ptr(v_out),
                                                    k_in.size, _bits(k_in), _bits(v_in), shift,
                                                    digit_bits),
           "count_sort_round")
    return k_out if vals is None else (k_out, v_out)


def radix_sort(keys: np.ndarray, vals: np.ndarray | None = None, radix_bits: int = 8, lib=None):
    """Stable ascending LSD radix sort (SR4 structure). Returns sorted copies."""
    k = np.array(keys, copy=True, order="C")
    v = None if vals is None else np.array(vals, copy=True, order="C")
    if v is not None and v.size != k.size:
        raise ValueError("keys and vals differ in length")
    _check((lib or _load()).oracle_radix_sort(_ptr(k), _ptr(v), k.size, _bits(k), _bits(v),
                                              radix_bits), "radix_sort")
    return k if vals is None else (k, v)


def segmented_sort(keys: np.ndarray, offsets: np.ndarray, vals: np.ndarray | None = None,
                   radix_bits: int = 8, lib=None):
    """Each [offsets[s], offsets[s+1]) sorted independently. Returns sorted copies."""
    k = np.array(keys, copy=True, order="C")
    v = None if vals is None else np.array(vals, copy=True, order="C")
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    nseg = max(0, off.size - 1)
    _check((lib or _load()).oracle_segmented_sort(_ptr(k), _ptr(v), _ptr(off) if nseg else None,
                                                  nseg, _bits(k), _bits(v), radix_bits),
           "segmented_sort")
    return k if vals is None else (k, v)


def gvr_sort(keys: np.ndarray, vals: np.ndarray | None = None, buckets: int = 256,
             oversample: int = 16, seed: int = 1, lib=None):
    """GVR sample sort (Algorithm 3). Returns (sorted keys[, vals], bucket counts,
    splitters) as copies."""
    k = np.array(keys, copy=True, order="C")
    v = None if vals is None else np.array(vals, copy=True, order="C")
    counts = np.zeros(buckets, dtype=np.uint32)
    split = np.zeros(max(buckets - 1, 1), dtype=np.uint64)
    _check((lib or _load()).oracle_gvr_sort(_ptr(k), _ptr(v), k.size, _bits(k), _bits(v), buckets,
                                            oversample, seed, _ptr(counts), _ptr(split)),
           "gvr_sort")
    out = (k,) if v is None else (k, v)
    return out + (counts, split[:buckets - 1])


def gsd_sort(keys: np.ndarray, vals: np.ndarray | None = None, buckets: int = 16,
             oversample: int = 4, lib=None):
    """GSD (Algorithm 1). Returns (sorted keys[, vals], bucket sizes, splitters) as copies."""
    k = np.array(keys, copy=True, order="C")
    v = None if vals is None else np.array(vals, copy=True, order="C")
    counts = np.zeros(buckets, dtype=np.uint32)
    split = np.zeros(max(buckets - 1, 1), dtype=np.uint64)
    _check((lib or _load()).oracle_gsd_sort(_ptr(k), _ptr(v), k.size, _bits(k), _bits(v), buckets,
                                            oversample, _ptr(counts), _ptr(split)), "gsd_sort")
    out = (k,) if v is None else (k, v)
    return out + (counts, split[:buckets - 1])
