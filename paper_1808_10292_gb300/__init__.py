"""isort: LSD radix sort of unsigned integer keys on one GB300 GPU.

Thin Python face of the C-ABI library (include/isort.h). Tensors are used only
for memory and streams: each call passes ``data_ptr()`` and the current CUDA
stream to the library, whose kernels do all the work. Sorting is in place on
CUDA tensors; sort_keys_host / sort_pairs_host take CPU tensors (host memory),
which the library copies to the device and back around the same sort.
"""
from __future__ import annotations

import ctypes

from . import _lib
from ._lib import IsortError, check, load

__all__ = ["sort_keys", "sort_pairs", "sort_keys_host", "sort_pairs_host", "sort_segmented",
           "workspace_size", "set_workspace", "stream_status", "release_workspaces", "IsortError",
           "load"]


def _torch():
    import torch
    return torch


def _bits(t) -> int:
    torch = _torch()
    if t.dtype in (torch.uint32, torch.int32):
        return 32
    if t.dtype in (torch.uint64, torch.int64):
        return 64
    raise TypeError(f"unsupported dtype {t.dtype}: keys and payloads are 32- or 64-bit words")


def _stream(stream) -> int:
    torch = _torch()
    s = torch.cuda.current_stream() if stream is None else stream
    return int(s.cuda_stream) if hasattr(s, "cuda_stream") else int(s)


_tuned_devices = set()


def _tuned():
    """Load the autotuner's cache for the current GPU into the library, once per
    device (a no-op without a GPU or a cache entry for it)."""
    torch = _torch()
    if not torch.cuda.is_available():
        return
    dev = torch.cuda.current_device()
    if dev in _tuned_devices:
        return
    _tuned_devices.add(dev)
    from . import tune
    tune.apply_all(torch.cuda.get_device_name(dev))


def _dev(t, name):
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def sort_keys(keys, radix_bits: int = 0, stream=None):
    """Sort a CUDA uint32/uint64 tensor ascending in place; returns it.

    radix_bits 0 lets the library choose the radix width and kernel variant
    (the autotuner's cache for this GPU is loaded into it on first use)."""
    _dev(keys, "keys")
    _tuned()
    check(load().isort_keys(keys.data_ptr(), keys.numel(), _bits(keys), radix_bits,
                            _stream(stream)), "isort_keys")
    return keys


def sort_keys_noalloc(keys, err_word, stream=None):
    """Sort a CUDA uint32 tensor in place with the library's fixed scratch array
    (isort_keys_noalloc): no device memory is allocated. At most
    NOALLOC_MAX_KEYS keys; calls must not overlap on the GPU.

    err_word: a CUDA 32-bit tensor (at least one element) on the keys' device,
    zeroed by the caller; device errors are OR-ed into its first element.
    The keys must be on the current CUDA device."""
    torch = _torch()
    _dev(keys, "keys")
    if _bits(keys) != 32:
        raise TypeError("isort_keys_noalloc sorts 32-bit keys")
    if err_word is None:
        raise ValueError("err_word is required: the device error bits are reported there")
    _dev(err_word, "err_word")
    if err_word.dtype not in (torch.int32, torch.uint32) or err_word.numel() < 1:
        raise ValueError("err_word must be a 32-bit tensor with at least one element")
    if err_word.device != keys.device:
        raise ValueError("err_word must be on the keys' device")
    if keys.device.index != torch.cuda.current_device():
        raise ValueError("keys must be on the current CUDA device (the fixed scratch array is "
                         "looked up per device)")
    check(load().isort_keys_noalloc(keys.data_ptr(), keys.numel(), err_word.data_ptr(),
                                    _stream(stream)), "isort_keys_noalloc")
    return keys


def _host(t, name):
    if t.is_cuda:
        raise ValueError(f"{name} must be a CPU tensor (host memory)")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def sort_keys_host(keys_in, keys_out=None, radix_bits: int = 0, stream=None):
    """Sort a CPU (host-memory) uint32/uint64 tensor through isort_keys_host:
    keys_out (default: keys_in, in place) receives the keys in ascending order.
    The copies in and out and the sort are enqueued on the CUDA stream; the
    result is there once the stream has reached that point (synchronize it).
    With pinned (page-locked) tensors the call returns at once; with pageable
    ones the copies complete before it returns."""
    keys_out = keys_in if keys_out is None else keys_out
    _host(keys_in, "keys_in")
    _host(keys_out, "keys_out")
    if keys_out.dtype != keys_in.dtype or keys_out.numel() != keys_in.numel():
        raise ValueError("keys_out must match keys_in in dtype and size")
    _tuned()
    check(load().isort_keys_host(keys_in.data_ptr(), keys_out.data_ptr(), keys_in.numel(),
                                 _bits(keys_in), radix_bits, _stream(stream)), "isort_keys_host")
    return keys_out


def sort_pairs_host(keys_in, vals_in, keys_out=None, vals_out=None, radix_bits: int = 0,
                    stream=None):
    """Stable key-value sort of CPU tensors through isort_pairs_host (outputs
    default to the inputs, in place); stream semantics as sort_keys_host."""
    keys_out = keys_in if keys_out is None else keys_out
    vals_out = vals_in if vals_out is None else vals_out
    for t, name in ((keys_in, "keys_in"), (vals_in, "vals_in"), (keys_out, "keys_out"),
                    (vals_out, "vals_out")):
        _host(t, name)
    n = keys_in.numel()
    if vals_in.numel() != n or keys_out.numel() != n or vals_out.numel() != n:
        raise ValueError("keys and payloads must have the same number of elements")
    if keys_out.dtype != keys_in.dtype or vals_out.dtype != vals_in.dtype:
        raise ValueError("outputs must match the inputs' dtypes")
    _tuned()
    check(load().isort_pairs_host(keys_in.data_ptr(), vals_in.data_ptr(), keys_out.data_ptr(),
                                  vals_out.data_ptr(), n, _bits(keys_in), _bits(vals_in),
                                  radix_bits, _stream(stream)), "isort_pairs_host")
    return keys_out, vals_out


def sort_pairs(keys, vals, radix_bits: int = 0, stream=None):
    """Stable key-value sort in place (vals follow their keys); returns (keys, vals)."""
    _dev(keys, "keys")
    _dev(vals, "vals")
    if keys.numel() != vals.numel():
        raise ValueError("keys and vals differ in length")
    _tuned()
    check(load().isort_pairs(keys.data_ptr(), vals.data_ptr(), keys.numel(), _bits(keys),
                             _bits(vals), radix_bits, _stream(stream)), "isort_pairs")
    return keys, vals


def sort_segmented(keys, offsets, vals=None, radix_bits: int = 0, stream=None):
    """Sort each [offsets[s], offsets[s+1]) independently, in place.

    offsets: CUDA int64 tensor of num_segments + 1 entries, offsets[0] = 0,
    non-decreasing, offsets[-1] == keys.numel().
    """
    torch = _torch()
    _dev(keys, "keys")
    _dev(offsets, "offsets")
    if offsets.dtype != torch.int64:
        raise TypeError("offsets must be int64")
    vb = 0
    vptr = None
    if vals is not None:
        _dev(vals, "vals")
        if vals.numel() != keys.numel():
            raise ValueError("keys and vals differ in length")
        vb, vptr = _bits(vals), vals.data_ptr()
    nseg = max(0, offsets.numel() - 1)
    check(load().isort_segmented(keys.data_ptr(), vptr, offsets.data_ptr(), nseg, keys.numel(),
                                 _bits(keys), vb, radix_bits, _stream(stream)), "isort_segmented")
    return keys if vals is None else (keys, vals)


def sample_sort(keys, vals=None, buckets: int = 256, oversample: int = 16, seed: int = 1,
                bucket_counts=None, stream=None):
    """The paper's GVR sample sort (Algorithm 3), in place: s*p - 1 sampled keys
    sorted, p - 1 splitters, one stable count-sort round by bucket, then the
    buckets sorted independently. bucket_counts: optional CUDA uint32 tensor of
    at least `buckets` entries that receives the bucket sizes."""
    _dev(keys, "keys")
    vb, vptr = 0, None
    if vals is not None:
        _dev(vals, "vals")
        if vals.numel() != keys.numel():
            raise ValueError("keys and vals differ in length")
        vb, vptr = _bits(vals), vals.data_ptr()
    cptr = None
    if bucket_counts is not None:
        _dev(bucket_counts, "bucket_counts")
        if _bits(bucket_counts) != 32 or bucket_counts.numel() < buckets:
            raise ValueError("bucket_counts must be uint32 with at least `buckets` entries")
        cptr = bucket_counts.data_ptr()
    check(load().isort_sample_sort(keys.data_ptr(), vptr, keys.numel(), _bits(keys), vb, buckets,
                                   oversample, seed, cptr, _stream(stream)), "isort_sample_sort")
    return keys if vals is None else (keys, vals)


def gsd_sort(keys, vals=None, buckets: int = 16, oversample: int = 4, bucket_counts=None,
             stream=None):
    """The paper's GSD (Algorithm 1), in place: p sequences sorted locally,
    r*p regular samples from each, p - 1 splitters, each sequence split by
    binary search and every bucket's parts merged. buckets: a power of two
    up to 64; oversample * buckets^2 <= 4096. bucket_counts: optional CUDA
    uint32 tensor of at least `buckets` entries for the bucket sizes."""
    _dev(keys, "keys")
    vb, vptr = 0, None
    if vals is not None:
        _dev(vals, "vals")
        if vals.numel() != keys.numel():
            raise ValueError("keys and vals differ in length")
        vb, vptr = _bits(vals), vals.data_ptr()
    cptr = None
    if bucket_counts is not None:
        _dev(bucket_counts, "bucket_counts")
        if _bits(bucket_counts) != 32 or bucket_counts.numel() < buckets:
            raise ValueError("bucket_counts must be uint32 with at least `buckets` entries")
        cptr = bucket_counts.data_ptr()
    check(load().isort_gsd_sort(keys.data_ptr(), vptr, keys.numel(), _bits(keys), vb, buckets,
                                oversample, cptr, _stream(stream)), "isort_gsd_sort")
    return keys if vals is None else (keys, vals)


def gsd_sort_workspace_size(n: int, key_bits: int = 32, val_bits: int = 0, buckets: int = 16,
                            oversample: int = 4) -> int:
    out = ctypes.c_size_t(0)
    check(load().isort_gsd_sort_workspace_size(n, key_bits, val_bits, buckets, oversample,
                                               ctypes.byref(out)),
          "isort_gsd_sort_workspace_size")
    return out.value


def sample_sort_workspace_size(n: int, key_bits: int = 32, val_bits: int = 0, buckets: int = 256,
                               oversample: int = 16) -> int:
    out = ctypes.c_size_t(0)
    check(load().isort_sample_sort_workspace_size(n, key_bits, val_bits, buckets, oversample,
                                                  ctypes.byref(out)),
          "isort_sample_sort_workspace_size")
    return out.value


def workspace_size(n: int, key_bits: int = 32, val_bits: int = 0, radix_bits: int = 0) -> int:
    _tuned()
    out = ctypes.c_size_t(0)
    check(load().isort_workspace_size(n, key_bits, val_bits, radix_bits, ctypes.byref(out)),
          "isort_workspace_size")
    return out.value


def set_workspace(buffer=None, stream=None):
    """Bind a CUDA uint8 tensor as the stream's workspace (None unbinds)."""
    if buffer is None:
        check(load().isort_set_workspace(None, 0, _stream(stream)), "isort_set_workspace")
        return
    _dev(buffer, "workspace")
    check(load().isort_set_workspace(buffer.data_ptr(), buffer.numel() * buffer.element_size(),
                                     _stream(stream)), "isort_set_workspace")


def stream_status(stream=None) -> int:
    """Synchronise the stream and return (and clear) its latched status code."""
    return load().isort_stream_status(_stream(stream))


def release_workspaces():
    check(load().isort_release_workspaces(), "isort_release_workspaces")


def tune_variants(key_bits: int = 32, val_bits: int = 0, radix_bits: int = 8):
    """[(threads, keys_per_thread)] of the compiled variants of one kernel family."""
    L = load()
    out = []
    for v in range(L.isort_tune_num_variants(key_bits, val_bits, radix_bits)):
        t, k = ctypes.c_int(0), ctypes.c_int(0)
        check(L.isort_tune_describe(key_bits, val_bits, radix_bits, v, ctypes.byref(t),
                                    ctypes.byref(k)), "isort_tune_describe")
        out.append((t.value, k.value))
    return out


def tune_segmented(key_bits: int = 32, val_bits: int = 0, btn_max_keys: int = -1):
    """Ranges of at most btn_max_keys keys take the BTN network (-1: default)."""
    check(load().isort_tune_segmented(key_bits, val_bits, btn_max_keys), "isort_tune_segmented")


def resolve(n: int, key_bits: int = 32, val_bits: int = 0, radix_bits: int = 0):
    """(radix_bits, variant) that a sort of n keys with these arguments uses."""
    _tuned()
    rb, v = ctypes.c_int(0), ctypes.c_int(0)
    check(load().isort_tune_resolve(n, key_bits, val_bits, radix_bits, ctypes.byref(rb),
                                    ctypes.byref(v)), "isort_tune_resolve")
    return rb.value, v.value


def tune_auto(key_bits: int, val_bits: int, size_log2: int, radix_bits: int, variant: int = 0):
    """Record the automatic choice (radix width, variant) for a size bucket;
    radix_bits < 0 clears (every bucket of the widths when size_log2 < 0)."""
    check(load().isort_tune_auto(key_bits, val_bits, size_log2, radix_bits, variant),
          "isort_tune_auto")


def workspace_bytes() -> int:
    """Device bytes the library holds in workspaces it allocated itself."""
    return int(load().isort_debug_workspace_bytes())


def launch_count() -> int:
    """Kernels the library has enqueued since it was loaded (a measurement hook)."""
    return int(load().isort_debug_launch_count())


def tune_segmented_network(key_bits: int = 32, val_bits: int = 0, network: str = "btn"):
    """Network of the short ranges of a segmented sort: "btn" (default) or "oet"."""
    net = {"btn": _lib.NET_BTN, "oet": _lib.NET_OET}[network]
    check(load().isort_tune_segmented_network(key_bits, val_bits, net),
          "isort_tune_segmented_network")


def segmented_workspace_size(num_segments: int, total_keys: int, key_bits: int = 32,
                             val_bits: int = 0) -> int:
    out = ctypes.c_size_t(0)
    check(load().isort_segmented_workspace_size(num_segments, total_keys, key_bits, val_bits,
                                                ctypes.byref(out)),
          "isort_segmented_workspace_size")
    return out.value


def tune_set(key_bits: int, val_bits: int, radix_bits: int, variant: int):
    check(load().isort_tune_set(key_bits, val_bits, radix_bits, variant), "isort_tune_set")


def debug_set(what: int, value: int):
    check(load().isort_debug_set(what, value), "isort_debug_set")


def kernel_times(max_kernels: int = 64):
    """[(kernel name, ms)] of the most recent sort (needs DEBUG_KERNEL_TIMING on)."""
    names = (ctypes.c_char_p * max_kernels)()
    ms = (ctypes.c_float * max_kernels)()
    n = load().isort_debug_kernel_times(names, ms, max_kernels)
    return [(names[i].decode(), float(ms[i])) for i in range(n)]
