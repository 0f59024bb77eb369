"""Autotuner: measures the library's kernel variants on this GPU and picks the
fastest, with a JSON cache keyed by GPU name, key/payload widths and size bucket.

What it tunes:
  * plain sorts: the radix-256 pass variant (threads x keys per thread, i.e.
    tile size and keys per thread) and the radix width (8, 11 or 16 bits) for
    (key_bits, val_bits, n-bucket); apply_all loads the winners into the
    library, where radix_bits = 0 resolves through them (isort_tune_auto);
  * segmented sorts: the longest range that still takes the BTN network
    (btn_max) for (key_bits, val_bits).
Measurement: CUDA events on the current stream around the library call, inputs
restored before each timed call, median of a few repetitions. Inputs are the
seeded uniform keys of the inputs module.
"""
from __future__ import annotations

import json
import os
import statistics

from . import _lib
from . import (load, resolve, sort_keys, sort_pairs, sort_segmented, stream_status,
               tune_auto, tune_segmented, tune_set, tune_variants)

CACHE = os.environ.get("ISORT_TUNE_CACHE",
                       os.path.join(os.path.dirname(os.path.abspath(__file__)), "tune_cache.json"))


def _gpu_name() -> str:
    import torch
    return torch.cuda.get_device_name()


def _bucket(n: int) -> int:
    """Size bucket: floor(log2 n)."""
    return max(0, int(n).bit_length() - 1)


def _time(fn, restore, reps: int = 5) -> float:
    import torch
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms = []
    for _ in range(reps + 1):
        restore()
        s.record()
        fn()
        e.record()
        e.synchronize()
        ms.append(s.elapsed_time(e))
    if stream_status() != _lib.OK:
        raise RuntimeError("device error while tuning")
    return statistics.median(ms[1:])


def load_cache(path: str = CACHE) -> dict:
    try:
        return json.load(open(path))
    except (OSError, ValueError):
        return {}


def save_cache(cache: dict, path: str = CACHE):
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune_plain(n: int, key_bits: int = 32, val_bits: int = 0, reps: int = 5) -> dict:
    """Time every radix-256 variant and the radix-65536 path on n seeded keys."""
    import torch
    import inputs
    pristine = inputs.device_keys(n, key_bits, "uniform", seed=1)
    keys = torch.empty_like(pristine)
    pv = inputs.device_iota(n, val_bits) if val_bits else None
    vals = torch.empty_like(pv) if val_bits else None

    def restore():
        keys.copy_(pristine)
        if val_bits:
            vals.copy_(pv)

    def run(rb):
        return (lambda: sort_pairs(keys, vals, rb)) if val_bits else (lambda: sort_keys(keys, rb))

    results = []
    for vi, (threads, kpt) in enumerate(tune_variants(key_bits, val_bits, 8)):
        tune_set(key_bits, val_bits, 8, vi)
        results.append({"radix_bits": 8, "variant": vi, "threads": threads, "kpt": kpt,
                        "ms": _time(run(8), restore, reps)})
    tune_set(key_bits, val_bits, 8, -1)
    for rb in (11, 16):
        results.append({"radix_bits": rb, "variant": 0, "ms": _time(run(rb), restore, reps)})
    best = min(results, key=lambda r: r["ms"])
    return {"best": best, "all": results, "n": n}


def tune_seg(num_segments: int, max_log2: int, key_bits: int = 32, val_bits: int = 0,
             reps: int = 3) -> dict:
    """Time the segmented sort for several BTN/radix thresholds."""
    import torch
    import inputs
    L = inputs.segment_lengths(num_segments, seed=1, max_log2=max_log2)
    off = torch.from_numpy(inputs.segment_offsets(L)).cuda()
    n = int(L.sum())
    pristine = inputs.device_keys(n, key_bits, "uniform", seed=1)
    keys = torch.empty_like(pristine)
    pv = inputs.device_iota(n, val_bits) if val_bits else None
    vals = torch.empty_like(pv) if val_bits else None

    def restore():
        keys.copy_(pristine)
        if val_bits:
            vals.copy_(pv)

    cap = 4096 if key_bits == 32 else 2048
    results = []
    for btn_max in sorted({512, 1024, 2048, cap}):
        if btn_max > cap:
            continue
        tune_segmented(key_bits, val_bits, btn_max)
        ms = _time(lambda: sort_segmented(keys, off, vals), restore, reps)
        results.append({"btn_max": btn_max, "ms": ms})
    tune_segmented(key_bits, val_bits, -1)
    best = min(results, key=lambda r: r["ms"])
    return {"best": best, "all": results, "num_segments": num_segments, "max_log2": max_log2,
            "keys": n}


def plain_key(key_bits, val_bits, n):
    return f"plain/k{key_bits}/v{val_bits}/b{_bucket(n)}"


def seg_key(key_bits, val_bits):
    return f"segmented/k{key_bits}/v{val_bits}"


def autotune(plain_sizes=((1 << 24, 32, 0),), segmented=((4000, 20, 32, 0),),
             path: str = CACHE) -> dict:
    """Run the sweeps and store the winners under this GPU's name."""
    load()
    cache = load_cache(path)
    gpu = cache.setdefault(_gpu_name(), {})
    for n, kb, vb in plain_sizes:
        gpu[plain_key(kb, vb, n)] = tune_plain(n, kb, vb)
    for nseg, ml, kb, vb in segmented:
        gpu[seg_key(kb, vb)] = tune_seg(nseg, ml, kb, vb)
    save_cache(cache, path)
    return cache


def parse_plain_key(key: str):
    """(key_bits, val_bits, size bucket) of a cache key "plain/k32/v0/b24", or None."""
    parts = key.split("/")
    if len(parts) != 4 or parts[0] != "plain":
        return None
    try:
        kb, vb, b = int(parts[1][1:]), int(parts[2][1:]), int(parts[3][1:])
    except ValueError:
        return None
    if parts[1][0] != "k" or parts[2][0] != "v" or parts[3][0] != "b":
        return None
    return kb, vb, b


def apply_all(gpu_name: str | None = None, path: str = CACHE) -> dict:
    """Load every choice the cache holds for this GPU into the library: per
    (key_bits, val_bits, size bucket) the fastest radix width and variant (what
    radix_bits = 0 then uses), and per widths the segmented BTN threshold.
    Returns {cache key: choice applied}; {} when the cache has nothing for it."""
    load()
    gpu = load_cache(path).get(gpu_name or _gpu_name(), {})
    applied = {}
    for key, entry in sorted(gpu.items()):
        parsed = parse_plain_key(key)
        if parsed:
            kb, vb, b = parsed
            best = entry["best"]
            tune_auto(kb, vb, b, best["radix_bits"], best.get("variant", 0))
            applied[key] = {"radix_bits": best["radix_bits"], "variant": best.get("variant", 0)}
        elif key.startswith("segmented/"):
            kb, vb = (int(x[1:]) for x in key.split("/")[1:3])
            tune_segmented(kb, vb, entry["best"]["btn_max"])
            applied[key] = {"btn_max": entry["best"]["btn_max"]}
    return applied


def apply(key_bits: int, val_bits: int, n: int | None = None, path: str = CACHE) -> dict:
    """Load the cache for this GPU into the library (apply_all) and report what
    a sort of (key_bits, val_bits, n) keys now resolves to."""
    applied = apply_all(path=path)
    out = {}
    if n is not None:
        rb, v = resolve(n, key_bits, val_bits, 0)
        out["plain"] = {"radix_bits": rb, "variant": v}
    seg = applied.get(seg_key(key_bits, val_bits))
    if seg:
        out["segmented"] = seg
    return out


def best_radix(key_bits: int, val_bits: int, n: int) -> int:
    """Radix width the library uses for radix_bits = 0 at n keys."""
    return resolve(n, key_bits, val_bits, 0)[0]


if __name__ == "__main__":
    import sys
    import torch
    torch.cuda.init()
    quick = "--quick" in sys.argv
    plain = ((1 << 24, 32, 0), (1 << 28, 32, 0), (1 << 26, 32, 32), (1 << 25, 64, 0)) if not quick \
        else ((1 << 24, 32, 0),)
    seg = ((20000, 20, 32, 0),) if not quick else ((2000, 16, 32, 0),)
    print(json.dumps(autotune(plain, seg), indent=1))
