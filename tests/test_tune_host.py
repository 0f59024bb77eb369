"""The autotuner's choices reach the library: radix_bits = 0 resolves through
the per-size-bucket table (isort_tune_auto), with the built-in defaults when
nothing was tuned, and the Python tuner loads its JSON cache into that table.
Host-side only: isort_tune_auto / isort_tune_resolve do no device work."""
import json

import pytest

import paper_1808_10292_gb300 as isort
from paper_1808_10292_gb300 import _lib, tune
from paper_1808_10292_gb300.build import build


@pytest.fixture(autouse=True)
def clean_tables():
    build()
    _lib.load()
    for kb in (32, 64):
        for vb in (0, 32, 64):
            isort.tune_auto(kb, vb, -1, -1)
            for rb in (8, 11, 16):
                isort.tune_set(kb, vb, rb, -1)
    yield
    for kb in (32, 64):
        for vb in (0, 32, 64):
            isort.tune_auto(kb, vb, -1, -1)
            for rb in (8, 11, 16):
                isort.tune_set(kb, vb, rb, -1)


# The built-in choices (the tuner's picks on a GB300, compiled into the
# library): 32-bit keys alone at 2^24 and 2^28 -> radix 256 variant 0; other
# widths tuned at one size -> variant 0.
BUILTIN_K32 = {24: (8, 0), 28: (8, 0)}


def test_defaults_without_tuning():
    # nearest built-in bucket (the lower one on a tie)
    for n, b in ((2, 24), (1000, 24), (1 << 20, 24), (1 << 26, 24), (1 << 27, 28),
                 (1 << 28, 28), (1 << 30, 28)):
        assert isort.resolve(n, 32, 0, 0) == BUILTIN_K32[b], n
    for n in (2, 1 << 20, 1 << 30):
        assert isort.resolve(n, 64, 32, 0) == (8, 0)   # no built-in entry
        assert isort.resolve(n, 32, 32, 0) == (8, 0)
        assert isort.resolve(n, 64, 0, 0) == (8, 0)
    assert isort.resolve(1 << 20, 32, 0, 16) == (16, 0)
    assert isort.resolve(1 << 20, 32, 0, 11) == (11, 0)


def test_nearest_bucket_and_ties():
    isort.tune_auto(32, 0, 20, 11, 0)
    assert isort.resolve(1 << 20, 32, 0, 0) == (11, 0)
    assert isort.resolve((1 << 21) - 1, 32, 0, 0) == (11, 0)   # floor(log2) = 20
    assert isort.resolve(5, 32, 0, 0) == (11, 0)               # the only entry
    isort.tune_auto(32, 0, 26, 8, 3)
    assert isort.resolve(1 << 23, 32, 0, 0) == (11, 0)         # 3 from both: the lower bucket
    assert isort.resolve(1 << 24, 32, 0, 0) == (8, 3)
    assert isort.resolve(1 << 30, 32, 0, 0) == (8, 3)
    # other widths are not affected
    assert isort.resolve(1 << 20, 32, 32, 0) == (8, 0)
    assert isort.resolve(1 << 20, 64, 0, 0) == (8, 0)


def test_explicit_width_takes_the_nearest_entry_of_that_width():
    isort.tune_auto(32, 0, 20, 11, 0)
    isort.tune_auto(32, 0, 26, 8, 3)
    assert isort.resolve(1 << 20, 32, 0, 8) == (8, 3)     # nearest radix-256 entry
    assert isort.resolve(1 << 26, 32, 0, 16) == (16, 0)   # no radix-65536 entry
    isort.tune_set(32, 0, 8, 2)                           # a fixed variant wins
    assert isort.resolve(1 << 20, 32, 0, 8) == (8, 2)
    assert isort.resolve(1 << 26, 32, 0, 0) == (8, 2)


def test_clearing_and_bad_arguments():
    isort.tune_auto(32, 0, 20, 11, 0)
    isort.tune_auto(32, 0, 26, 16, 0)
    isort.tune_auto(32, 0, 20, -1)                        # clear one bucket
    assert isort.resolve(1 << 20, 32, 0, 0) == (16, 0)
    isort.tune_auto(32, 0, -1, -1)                        # clear every bucket
    assert isort.resolve(1 << 20, 32, 0, 0) == BUILTIN_K32[24]   # back to the built-in
    lib = _lib.load()
    nv = len(isort.tune_variants(32, 0, 8))
    assert lib.isort_tune_auto(32, 0, 20, 8, nv) == _lib.EINVAL      # no such variant
    assert lib.isort_tune_auto(32, 0, 20, 16, 1) == _lib.EINVAL      # radix 65536 has one
    assert lib.isort_tune_auto(32, 0, 20, 12, 0) == _lib.EINVAL      # no such width
    assert lib.isort_tune_auto(32, 0, 31, 8, 0) == _lib.EINVAL       # bucket beyond 2^30
    assert lib.isort_tune_auto(16, 0, 20, 8, 0) == _lib.EINVAL       # key width
    assert lib.isort_tune_auto(32, 8, 20, 8, 0) == _lib.EINVAL       # payload width
    with pytest.raises(isort.IsortError):
        isort.resolve(1 << 20, 32, 0, 7)


def test_workspace_size_follows_the_resolved_width():
    n = 1 << 20
    base = isort.workspace_size(n, 32, 0, 0)
    assert base == isort.workspace_size(n, 32, 0, 8)
    isort.tune_auto(32, 0, 20, 16, 0)
    assert isort.workspace_size(n, 32, 0, 0) == isort.workspace_size(n, 32, 0, 16) != base


def test_cache_keys_and_loading(tmp_path):
    assert tune.parse_plain_key("plain/k32/v0/b24") == (32, 0, 24)
    assert tune.parse_plain_key("plain/k64/v32/b26") == (64, 32, 26)
    assert tune.parse_plain_key("segmented/k32/v0") is None
    assert tune.parse_plain_key("plain/x32/v0/b24") is None
    assert tune.plain_key(32, 0, (1 << 24) + 5) == "plain/k32/v0/b24"
    assert tune._bucket(1) == 0 and tune._bucket(1 << 20) == 20 and tune._bucket((1 << 20) - 1) == 19
    cache = {
        "GPU A": {
            "plain/k32/v0/b20": {"best": {"radix_bits": 11, "variant": 0, "ms": 1.0}},
            "plain/k32/v0/b28": {"best": {"radix_bits": 8, "variant": 1, "ms": 3.0}},
            "plain/k64/v0/b25": {"best": {"radix_bits": 8, "variant": 2, "ms": 2.0}},
        },
        "GPU B": {"plain/k32/v0/b20": {"best": {"radix_bits": 16, "variant": 0, "ms": 9.0}}},
    }
    path = tmp_path / "cache.json"
    path.write_text(json.dumps(cache))
    assert tune.apply_all("GPU C", path=str(path)) == {}     # nothing for this GPU: defaults stay
    assert isort.resolve(1 << 20, 32, 0, 0) == BUILTIN_K32[24]
    applied = tune.apply_all("GPU A", path=str(path))
    assert applied["plain/k32/v0/b20"] == {"radix_bits": 11, "variant": 0}
    assert isort.resolve(1 << 20, 32, 0, 0) == (11, 0)
    assert isort.resolve(1 << 28, 32, 0, 0) == (8, 1)
    assert isort.resolve(1 << 25, 64, 0, 0) == (8, 2)
    assert isort.resolve(1 << 25, 64, 32, 0) == (8, 0)       # not in the cache
    assert tune.load_cache(str(tmp_path / "missing.json")) == {}


def test_shipped_cache_is_well_formed():
    cache = tune.load_cache()
    assert cache, "the repository ships the tuner's cache measured on a GB300"
    for gpu, entries in cache.items():
        for key, entry in entries.items():
            if key.startswith("plain/"):
                kb, vb, b = tune.parse_plain_key(key)
                best = entry["best"]
                assert best["radix_bits"] in (8, 11, 16)
                nv = len(isort.tune_variants(kb, vb, best["radix_bits"]))
                assert 0 <= best.get("variant", 0) < nv, (gpu, key)


def test_builtin_table_is_the_shipped_cache():
    """The compiled-in choices are the shipped cache's GB300 winners."""
    gpu = tune.load_cache().get("NVIDIA GB300", {})
    plain = {tune.parse_plain_key(k): v["best"] for k, v in gpu.items() if k.startswith("plain/")}
    assert plain
    for (kb, vb, b), best in plain.items():
        assert isort.resolve(1 << b, kb, vb, 0) == (best["radix_bits"], best.get("variant", 0))
