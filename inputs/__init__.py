"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This module holds no sorting arithmetic. It defines one counter-based random
generator and the recipes that turn its draws into keys, payloads, segment
layouts and request streams. The same generator is implemented for the GPU in
``inputs/synth.cu`` (bit-identical; a test checks that), so full-size inputs can
be made on the device without a host round trip.

Generator (counter-based SplitMix64; Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014). All arithmetic is mod 2^64::

    mix64(z)  = z ^= z >> 30; z *= 0xBF58476D1CE4E5B9;
                z ^= z >> 27; z *= 0x94D049BB133111EB; z ^ (z >> 31)
    S(seed, stream) = mix64(seed * GAMMA  ^  stream * 0xD1B54A32D192ED03)
    draw(seed, stream, i) = mix64(S + (i + 1) * GAMMA),   GAMMA = 0x9E3779B97F4A7C15

A 32-bit draw is the high half of the 64-bit draw.

Key distributions (the paper never states its inputs, so these six stand in for
its 8M/32M/128M runs; ``stream`` defaults to the distribution id):

    0 uniform   : draw (u64) / hi32(draw) (u32), uniform over the key range
    1 u16       : low 16 bits of the uniform draw, i.e. uniform in [0, 2^16)
    2 equal     : every key = draw(seed, stream, 0)
    3 sorted    : u32: floor((i * 2^32 + hi32(draw_i)) / n)  -- a stratified uniform
                  sample, non-decreasing by construction, every digit non-trivial;
                  u64: (i << (64 - L)) | (draw_i >> L), L = bit length of n - 1
    4 reverse   : the ``sorted`` formula taken at index n - 1 - i (non-increasing)
    5 and4      : AND of the draws at 4i, 4i+1, 4i+2, 4i+3 (each bit set w.p. 1/16)

Payloads are the original index (stability is then checkable).
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
STREAM_MUL = 0xD1B54A32D192ED03
M1 = 0xBF58476D1CE4E5B9
M2 = 0x94D049BB133111EB
MASK64 = (1 << 64) - 1

DISTS = ("uniform", "u16", "equal", "sorted", "reverse", "and4")
DIST_ID = {name: i for i, name in enumerate(DISTS)}

# Stream ids for the non-key draws (distinct from the six key streams).
STREAM_SEGMENTS = 10
STREAM_SERVE = 20
STREAM_REQUEST_BASE = 1000  # request r draws its keys from stream 1000 + r


def mix64_int(z: int) -> int:
    """SplitMix64 finaliser on a Python int (mod 2^64)."""
    z &= MASK64
    z = ((z ^ (z >> 30)) * M1) & MASK64
    z = ((z ^ (z >> 27)) * M2) & MASK64
    return z ^ (z >> 31)


def stream_key(seed: int, stream: int) -> int:
    return mix64_int(((seed * GAMMA) & MASK64) ^ ((stream * STREAM_MUL) & MASK64))


def _mix64_np(z: np.ndarray) -> np.ndarray:
    z = z ^ (z >> np.uint64(30))
    z = z * np.uint64(M1)
    z = z ^ (z >> np.uint64(27))
    z = z * np.uint64(M2)
    return z ^ (z >> np.uint64(31))


def draws_u64(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """draw(seed, stream, i) for i in [start, start + count), as uint64."""
    if count <= 0:
        return np.zeros(0, dtype=np.uint64)
    s = np.uint64(stream_key(seed, stream))
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + 1 + count, dtype=np.uint64)
        z = s + i * np.uint64(GAMMA)
        return _mix64_np(z)


def _hi32(x: np.ndarray) -> np.ndarray:
    return (x >> np.uint64(32)).astype(np.uint32)


def _sorted_u32(n: int, seed: int, stream: int, idx: np.ndarray) -> np.ndarray:
    r = _hi32(draws_u64(seed, stream, 0, n))[idx].astype(np.uint64)
    num = (idx.astype(np.uint64) << np.uint64(32)) + r
    return (num // np.uint64(n)).astype(np.uint32)


def _sorted_u64(n: int, seed: int, stream: int, idx: np.ndarray) -> np.ndarray:
    d = draws_u64(seed, stream, 0, n)[idx]
    L = (n - 1).bit_length()
    if L == 0:
        return d
    return (idx.astype(np.uint64) << np.uint64(64 - L)) | (d >> np.uint64(L))


def keys(n: int, key_bits: int = 32, dist: str | int = "uniform", seed: int = 1,
         stream: int | None = None) -> np.ndarray:
    """Seeded keys of one of the six distributions (see module docstring)."""
    if key_bits not in (32, 64):
        raise ValueError("key_bits must be 32 or 64")
    dist_id = DIST_ID[dist] if isinstance(dist, str) else int(dist)
    if not 0 <= dist_id < len(DISTS):
        raise ValueError(f"unknown distribution {dist!r}")
    st = dist_id if stream is None else int(stream)
    dt = np.uint32 if key_bits == 32 else np.uint64
    if n == 0:
        return np.zeros(0, dtype=dt)
    if dist_id == 0:
        d = draws_u64(seed, st, 0, n)
        return _hi32(d) if key_bits == 32 else d
    if dist_id == 1:
        d = draws_u64(seed, st, 0, n)
        k = _hi32(d) if key_bits == 32 else d
        return (k & dt(0xFFFF)).astype(dt)
    if dist_id == 2:
        d = draws_u64(seed, st, 0, 1)
        k = _hi32(d) if key_bits == 32 else d
        return np.full(n, k[0], dtype=dt)
    if dist_id in (3, 4):
        idx = np.arange(n, dtype=np.int64)
        if dist_id == 4:
            idx = idx[::-1].copy()
        return _sorted_u32(n, seed, st, idx) if key_bits == 32 else _sorted_u64(n, seed, st, idx)
    # and4
    d = draws_u64(seed, st, 0, 4 * n).reshape(n, 4)
    if key_bits == 32:
        d = _hi32(d)
    return (d[:, 0] & d[:, 1] & d[:, 2] & d[:, 3]).astype(dt)


def iota(n: int, val_bits: int = 32) -> np.ndarray:
    """Payload = original index."""
    return np.arange(n, dtype=np.uint32 if val_bits == 32 else np.uint64)


def unit_doubles(seed: int, stream: int, count: int) -> np.ndarray:
    """u_i = (draw >> 11) * 2^-53, uniform in [0, 1)."""
    d = draws_u64(seed, stream, 0, count)
    return (d >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def segment_lengths(num_segments: int, seed: int = 1, max_log2: int = 20) -> np.ndarray:
    """L_i = max(1, floor(2^(max_log2 * u_i))): log-uniform lengths in [1, 2^max_log2]."""
    u = unit_doubles(seed, STREAM_SEGMENTS, num_segments)
    return np.maximum(1, np.floor(np.exp2(max_log2 * u))).astype(np.int64)


def segment_offsets(lengths: np.ndarray) -> np.ndarray:
    """int64 exclusive prefix sums, num_segments + 1 entries, offsets[0] = 0."""
    off = np.zeros(len(lengths) + 1, dtype=np.int64)
    np.cumsum(lengths, out=off[1:])
    return off


def requests(num: int, seed: int = 1, rate: float = 2000.0, min_log2: int = 10,
             max_log2: int = 24, payload_prob: float = 0.5):
    """Poisson request stream: (arrival_s, n_keys, has_payload) per request.

    Inter-arrival -ln(1 - u)/rate; size floor(2^(min_log2 + (max_log2 - min_log2) u'));
    payload when u'' < payload_prob. Request r's keys are uniform u32 from stream
    STREAM_REQUEST_BASE + r.
    """
    u = unit_doubles(seed, STREAM_SERVE, 3 * num).reshape(num, 3) if num else np.zeros((0, 3))
    gaps = -np.log1p(-u[:, 0]) / rate
    arrivals = np.cumsum(gaps)
    sizes = np.floor(np.exp2(min_log2 + (max_log2 - min_log2) * u[:, 1])).astype(np.int64)
    sizes = np.minimum(sizes, 1 << max_log2)
    payload = u[:, 2] < payload_prob
    return arrivals, sizes, payload


def expected_and4_bit_density() -> float:
    """Probability that one bit of an AND-of-4 key is set."""
    return 1.0 / 16.0


def lengths_mean(max_log2: int = 20) -> float:
    """E[L] for L = floor(2^(m u)), u ~ U[0,1), approximated by the continuous mean (2^m - 1)/(m ln 2)."""
    return (2.0 ** max_log2 - 1.0) / (max_log2 * math.log(2.0))


# ---- device-side generation (same recipes, inputs/synth.cu) -----------------
_synth = None
SYNTH_LIB = __file__.rsplit("/", 1)[0] + "/libsynth.so"


def _synth_lib():
    global _synth
    if _synth is None:
        import ctypes
        import os
        if not os.path.exists(SYNTH_LIB):
            raise RuntimeError(f"{SYNTH_LIB} is missing; build it with "
                               "`python -m paper_1808_10292_gb300.build`")
        lib = ctypes.CDLL(SYNTH_LIB)
        vp, i64, i32, u64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_uint64
        lib.synth_keys.argtypes = [vp, i64, i32, i32, u64, u64, vp]
        lib.synth_keys.restype = i32
        lib.synth_iota.argtypes = [vp, i64, i32, vp]
        lib.synth_iota.restype = i32
        _synth = lib
    return _synth


def device_keys(n: int, key_bits: int = 32, dist: str | int = "uniform", seed: int = 1,
                stream: int | None = None, out=None, cuda_stream=None):
    """Same keys as keys(...), generated in device memory (a torch CUDA tensor)."""
    import torch
    dist_id = DIST_ID[dist] if isinstance(dist, str) else int(dist)
    st = dist_id if stream is None else int(stream)
    if out is None:
        out = torch.empty(n, dtype=torch.uint32 if key_bits == 32 else torch.uint64, device="cuda")
    cs = torch.cuda.current_stream() if cuda_stream is None else cuda_stream
    rc = _synth_lib().synth_keys(out.data_ptr() if n else None, n, key_bits, dist_id,
                                 seed & MASK64, st & MASK64, cs.cuda_stream)
    if rc:
        raise RuntimeError(f"synth_keys failed ({rc})")
    return out


def device_iota(n: int, val_bits: int = 32, out=None, cuda_stream=None):
    import torch
    if out is None:
        out = torch.empty(n, dtype=torch.uint32 if val_bits == 32 else torch.uint64, device="cuda")
    cs = torch.cuda.current_stream() if cuda_stream is None else cuda_stream
    rc = _synth_lib().synth_iota(out.data_ptr() if n else None, n, val_bits, cs.cuda_stream)
    if rc:
        raise RuntimeError(f"synth_iota failed ({rc})")
    return out
