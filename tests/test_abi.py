"""The C-ABI library loads and exports what include/isort.h declares; host-side
argument checks answer without touching a GPU (no compute calls here)."""
import ctypes
import os
import subprocess

import pytest

import paper_1808_10292_gb300 as isort
from paper_1808_10292_gb300 import _lib
from paper_1808_10292_gb300.build import build, LIB, SYNTH_LIB

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build()
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    names = _lib.declared_symbols()
    assert "isort_keys" in names and "isort_segmented" in names and "isort_pairs" in names
    out = subprocess.run(["nm", "-D", "--defined-only", LIB], capture_output=True, text=True,
                         check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = [n for n in names if n not in exported]
    assert not missing, f"declared but not exported: {missing}"
    for n in names:
        getattr(lib, n)  # resolvable through ctypes too


def test_synth_library_exports(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", SYNTH_LIB], capture_output=True,
                         text=True, check=True).stdout
    assert "synth_keys" in out and "synth_iota" in out


def test_argument_errors_need_no_gpu(lib):
    dummy = ctypes.c_void_p(256)
    assert lib.isort_keys(dummy, 10, 16, 8, None) == _lib.EINVAL        # bad key width
    assert lib.isort_keys(dummy, 10, 32, 7, None) == _lib.EUNSUPPORTED  # radix 2^7
    assert lib.isort_keys(dummy, 10, 32, 12, None) == _lib.EUNSUPPORTED  # radix 2^12
    assert lib.isort_keys(dummy, 10, 32, 40, None) == _lib.EINVAL       # nonsense radix
    assert lib.isort_keys(dummy, -1, 32, 8, None) == _lib.EINVAL
    assert lib.isort_keys(dummy, (1 << 30) + 1, 32, 8, None) == _lib.EUNSUPPORTED
    assert lib.isort_keys(None, 10, 32, 8, None) == _lib.EINVAL
    assert lib.isort_keys(ctypes.c_void_p(258), 10, 32, 8, None) == _lib.EINVAL  # misaligned
    assert lib.isort_keys(None, 0, 32, 8, None) == _lib.OK   # empty: no-op
    assert lib.isort_keys(None, 1, 64, 8, None) == _lib.OK   # one key: no-op
    assert lib.isort_pairs(dummy, None, 10, 32, 32, 8, None) == _lib.EINVAL
    assert lib.isort_pairs(dummy, dummy, 10, 32, 16, 8, None) == _lib.EINVAL
    # host-buffer entry points: the same checks, no device work for n <= 1 in place
    assert lib.isort_keys_host(dummy, dummy, 10, 16, 8, None) == _lib.EINVAL
    assert lib.isort_keys_host(None, dummy, 10, 32, 8, None) == _lib.EINVAL
    assert lib.isort_keys_host(dummy, None, 10, 32, 8, None) == _lib.EINVAL
    assert lib.isort_keys_host(ctypes.c_void_p(258), dummy, 10, 32, 8, None) == _lib.EINVAL
    assert lib.isort_keys_host(dummy, dummy, -1, 32, 8, None) == _lib.EINVAL
    assert lib.isort_keys_host(dummy, dummy, (1 << 30) + 1, 32, 8, None) == _lib.EUNSUPPORTED
    assert lib.isort_keys_host(dummy, dummy, 10, 32, 12, None) == _lib.EUNSUPPORTED
    assert lib.isort_keys_host(None, None, 0, 32, 8, None) == _lib.OK
    assert lib.isort_keys_host(dummy, dummy, 1, 32, 8, None) == _lib.OK   # in place: nothing
    assert lib.isort_pairs_host(dummy, None, dummy, dummy, 10, 32, 32, 8, None) == _lib.EINVAL
    assert lib.isort_pairs_host(dummy, dummy, dummy, None, 10, 32, 32, 8, None) == _lib.EINVAL
    assert lib.isort_pairs_host(dummy, dummy, dummy, dummy, 10, 32, 16, 8, None) == _lib.EINVAL
    assert lib.isort_pairs_host(dummy, ctypes.c_void_p(260), dummy, dummy, 10, 32, 64, 8,
                                None) == _lib.EINVAL                      # misaligned payloads
    assert lib.isort_pairs_host(dummy, dummy, dummy, dummy, 1, 32, 32, 8, None) == _lib.OK
    assert lib.isort_debug_set(_lib.DEBUG_HOST_COPY, 3) == _lib.EINVAL
    assert lib.isort_debug_set(4, 0) == _lib.EINVAL                       # no such hook
    assert lib.isort_debug_set(99, 0) == _lib.EINVAL
    assert lib.isort_tune_segmented_network(32, 0, 2) == _lib.EINVAL    # no such network
    assert lib.isort_tune_segmented_network(16, 0, _lib.NET_OET) == _lib.EINVAL
    assert lib.isort_tune_segmented_network(32, 0, _lib.NET_BTN) == _lib.OK
    assert lib.isort_strerror(_lib.ETIMEOUT) == b"bounded device wait gave up"
    # segmented batches: each radix tile records its first key in 40 bits
    assert lib.isort_segmented(dummy, None, dummy, 1, 1 << 40, 32, 0, 8, None) == _lib.EINVAL
    assert lib.isort_segmented(dummy, None, dummy, 1, -1, 32, 0, 8, None) == _lib.EINVAL
    size = ctypes.c_size_t(0)
    assert lib.isort_segmented_workspace_size(1, 1 << 40, 32, 0, ctypes.byref(size)) == _lib.EINVAL


def test_workspace_size_and_tuning_tables(lib):
    n = 1 << 20
    size = isort.workspace_size(n, 32, 0, 8)
    assert size >= n * 4  # at least the alternate key buffer
    assert isort.workspace_size(n, 32, 32, 8) >= size + n * 4
    assert isort.workspace_size(n, 64, 0, 8) >= n * 8
    assert isort.workspace_size(n, 32, 0, 16) >= n * 4 + 2 * 65536 * 4  # radix 65536: matrix
    assert len(isort.tune_variants(32, 0, 16)) == 1
    # radix 2048: three passes (11, 11, 10 bits), a count matrix of 2^16-key rows
    assert isort.workspace_size(n, 32, 0, 11) >= n * 4 + 2048 * 4 * (n >> 16)
    assert len(isort.tune_variants(32, 0, 11)) == 1 and len(isort.tune_variants(64, 64, 11)) == 1
    v = isort.tune_variants(32, 0, 8)
    assert len(v) >= 2 and all(t % 32 == 0 and k > 0 for t, k in v)
    with pytest.raises(isort.IsortError):
        isort.tune_set(32, 0, 8, len(v))
    isort.tune_set(32, 0, 8, 1)
    isort.tune_set(32, 0, 8, -1)


def test_no_cpu_fallback_when_library_missing(tmp_path, monkeypatch):
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "libisort.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        _lib.load()
