"""The ordered keys-only rounds: ranks from the order in which shared atomics
serve the lanes of a warp, checked per tile, with a stable re-rank for tiles
that fail the check. These tests drive the check and the fallback through the
library's test hook (ISORT_DEBUG_CHECK_MODE): mode 1 sends every tile through
the fallback, mode 2 makes the fast ranks deliberately unstable (odd lanes
first), which the check must catch. Either way the result must equal the
oracle's, bit for bit."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import inputs
import oracle
import paper_1808_10292_gb300 as isort
from paper_1808_10292_gb300 import _lib

pytestmark = pytest.mark.gpu

MODES = [0, 1, 2]


@pytest.fixture
def check_mode():
    def set_mode(m):
        isort.debug_set(_lib.DEBUG_CHECK_MODE, m)
    yield set_mode
    isort.debug_set(_lib.DEBUG_CHECK_MODE, 0)


def _oracle(k):
    return oracle.radix_sort(k, radix_bits=8)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("key_bits", [32, 64])
@pytest.mark.parametrize("dist", inputs.DISTS)
def test_plain_sort_every_check_mode(check_mode, mode, key_bits, dist):
    n = 3 * 8192 + 4099  # several tiles and a ragged one
    k = inputs.keys(n, key_bits, dist, seed=11)
    expect = _oracle(k)
    check_mode(mode)
    for variant in range(len(isort.tune_variants(key_bits, 0, 8))):
        isort.tune_set(key_bits, 0, 8, variant)
        d = torch.from_numpy(k).cuda()
        isort.sort_keys(d, 8)
        assert isort.stream_status() == _lib.OK
        assert np.array_equal(d.cpu().numpy(), expect), (mode, variant)
    isort.tune_set(key_bits, 0, 8, -1)


@pytest.mark.parametrize("mode", MODES)
def test_segmented_every_check_mode(check_mode, mode):
    L = inputs.segment_lengths(300, seed=12, max_log2=15)
    off = inputs.segment_offsets(L)
    k = inputs.keys(int(off[-1]), 32, "and4", seed=13)
    check_mode(mode)
    d = torch.from_numpy(k).cuda()
    isort.sort_segmented(d, torch.from_numpy(off).cuda())
    assert isort.stream_status() == _lib.OK
    assert np.array_equal(d.cpu().numpy(), oracle.segmented_sort(k, off))


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("radix_bits", [16, 11])
@pytest.mark.parametrize("key_bits,val_bits", [(32, 0), (32, 32), (64, 0)])
@pytest.mark.parametrize("dist", ["uniform", "and4", "u16", "sorted"])
def test_wide_radix_every_check_mode(check_mode, mode, radix_bits, key_bits, val_bits, dist):
    """Radix 65536 and 2048 route each round in two ordered steps (the high
    part of the digit over all keys, checked against the bits below the whole
    digit; the low byte inside every bucket); both steps must survive a forced
    fallback and perturbed ranks."""
    n = 400_003
    k = inputs.keys(n, key_bits, dist, seed=15)
    check_mode(mode)
    d = torch.from_numpy(k).cuda()
    if val_bits:
        v = inputs.iota(n, val_bits)
        dv = torch.from_numpy(v).cuda()
        isort.sort_pairs(d, dv, radix_bits)
        ok, ov = oracle.radix_sort(k, v, radix_bits=radix_bits)
        assert isort.stream_status() == _lib.OK
        assert np.array_equal(dv.cpu().numpy(), ov)
    else:
        isort.sort_keys(d, radix_bits)
        ok = oracle.radix_sort(k, radix_bits=radix_bits)
        assert isort.stream_status() == _lib.OK
    assert np.array_equal(d.cpu().numpy(), ok)


def test_perturbed_ranks_fail_the_check_and_are_repaired(check_mode):
    """With odd lanes first, a round whose rows hold equal digits with different
    low bits is unstable; the result is still exact, so the check caught every
    such tile (a 2^20-key uniform sort has many)."""
    k = inputs.keys(1 << 20, 32, "uniform", seed=14)
    check_mode(2)
    d = torch.from_numpy(k).cuda()
    isort.sort_keys(d, 8)
    assert isort.stream_status() == _lib.OK
    assert np.array_equal(d.cpu().numpy(), np.sort(k))


def test_check_mode_argument():
    lib = _lib.load()
    assert lib.isort_debug_set(_lib.DEBUG_CHECK_MODE, 3) == _lib.EINVAL
    assert lib.isort_debug_set(_lib.DEBUG_CHECK_MODE, -1) == _lib.EINVAL
    assert lib.isort_debug_set(_lib.DEBUG_CHECK_MODE, 0) == _lib.OK


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("key_bits,val_bits", [(32, 0), (32, 32), (64, 0)])
@pytest.mark.parametrize("dist", ["uniform", "and4", "sorted"])
def test_sample_sort_buckets_every_check_mode(check_mode, mode, key_bits, val_bits, dist):
    """With 256 buckets the top digit takes one or two values inside a bucket,
    and the buckets' top pass ranks such tiles by one ballot per digit value
    instead of slot adds; those ranks, the forced fallback after them and the
    perturbed ranks must all give the oracle's result."""
    n = 3_000_017  # buckets of about 1.4 tiles: whole and ragged tiles
    k = inputs.keys(n, key_bits, dist, seed=16)
    v = inputs.iota(n, val_bits) if val_bits else None
    check_mode(mode)
    dk = torch.from_numpy(k).cuda()
    dv = None if v is None else torch.from_numpy(v).cuda()
    isort.sample_sort(dk, dv, buckets=256, oversample=16, seed=5)
    assert isort.stream_status() == _lib.OK
    if val_bits:
        ok, ov, _, _ = oracle.gvr_sort(k, v, buckets=256, oversample=16, seed=5)
        assert np.array_equal(dv.cpu().numpy(), ov)
    else:
        ok, _, _ = oracle.gvr_sort(k, buckets=256, oversample=16, seed=5)
    assert np.array_equal(dk.cpu().numpy(), ok)
