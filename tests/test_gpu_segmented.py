"""GPU parity of the segmented sort (BTN for short ranges, radix passes for long
ones) against the serial oracle's per-range sort, element by element."""
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

# lengths around every class edge: warp BTN (<= 128), 64-thread BTN (<= 512),
# 256-thread BTN (<= 4096 for 32-bit keys, 2048 for 64-bit), radix tiles (8192 keys for
# 32-bit keys alone, 5120 with 32-bit payloads or for 64-bit keys, 4096 / 3072 for the rest)
EDGE_LENGTHS = [0, 1, 2, 3, 31, 32, 33, 127, 128, 129, 511, 512, 513, 2047, 2048, 2049, 3071, 5119,
                5120, 5121, 8192, 10241, 12287, 12288, 12289, 16385, 24577,
                3072, 3073, 4095, 4096, 4097, 8191, 8193, 12289, 100_000, 0, 1, 5]


def run_segmented(keys, offsets, vals=None, radix_bits=0):
    k = torch.from_numpy(keys).cuda()
    off = torch.from_numpy(offsets).cuda()
    v = None if vals is None else torch.from_numpy(vals).cuda()
    isort.sort_segmented(k, off, v, radix_bits)
    status = isort.stream_status()
    return status, k.cpu().numpy(), (None if v is None else v.cpu().numpy())


@pytest.mark.parametrize("key_bits,val_bits", [(32, 0), (32, 32), (32, 64), (64, 0), (64, 32),
                                               (64, 64)])
@pytest.mark.parametrize("dist", ["uniform", "and4", "equal", "reverse"])
def test_class_edges(key_bits, val_bits, dist):
    L = np.array(EDGE_LENGTHS, dtype=np.int64)
    off = inputs.segment_offsets(L)
    n = int(off[-1])
    k = inputs.keys(n, key_bits, dist, seed=41)
    v = inputs.iota(n, val_bits) if val_bits else None
    st, gk, gv = run_segmented(k, off, v)
    assert st == _lib.OK
    if v is None:
        assert np.array_equal(gk, oracle.segmented_sort(k, off))
    else:
        ok, ov = oracle.segmented_sort(k, off, v)
        assert np.array_equal(gk, ok)
        assert np.array_equal(gv, ov)


@pytest.mark.parametrize("key_bits,val_bits", [(32, 0), (32, 32), (64, 0), (64, 64)])
@pytest.mark.parametrize("dist", ["uniform", "and4", "equal", "reverse"])
def test_oet_network_class_edges(key_bits, val_bits, dist):
    """The odd-even transposition network (Algorithm OET) on the short-range
    classes gives the same stable result as BTN and the oracle."""
    L = np.array(EDGE_LENGTHS, dtype=np.int64)
    off = inputs.segment_offsets(L)
    n = int(off[-1])
    k = inputs.keys(n, key_bits, dist, seed=43)
    v = inputs.iota(n, val_bits) if val_bits else None
    try:
        isort.tune_segmented_network(key_bits, val_bits, "oet")
        st, gk, gv = run_segmented(k, off, v)
    finally:
        isort.tune_segmented_network(key_bits, val_bits, "btn")
    assert st == _lib.OK
    if v is None:
        assert np.array_equal(gk, oracle.segmented_sort(k, off))
    else:
        ok, ov = oracle.segmented_sort(k, off, v)
        assert np.array_equal(gk, ok)
        assert np.array_equal(gv, ov)


@pytest.mark.parametrize("key_bits", [32, 64])
def test_log_uniform_lengths(key_bits):
    """The batched workload's recipe at reduced scale: 3000 ranges, lengths
    log-uniform in [1, 2^16]."""
    L = inputs.segment_lengths(3000, seed=5, max_log2=16)
    off = inputs.segment_offsets(L)
    n = int(off[-1])
    k = inputs.keys(n, key_bits, "uniform", seed=6)
    v = inputs.iota(n, 32)
    st, gk, gv = run_segmented(k, off, v)
    assert st == _lib.OK
    ok, ov = oracle.segmented_sort(k, off, v)
    assert np.array_equal(gk, ok)
    assert np.array_equal(gv, ov)


@pytest.mark.parametrize("key_bits,val_bits", [(32, 0), (32, 32), (64, 0), (64, 64)])
def test_per_range_pass_skip(key_bits, val_bits):
    """Ranges whose digit is constant in some passes skip those passes for
    themselves only, so ranges end after odd and even numbers of executed
    passes (the odd ones are copied home): low-entropy ranges (keys below
    2^16, or a constant middle byte), all-equal ranges, a range constant in
    every pass but one, uniform ranges, side by side in one batch."""
    rng_len = [20000, 9000, 30000, 12000, 50000, 8193, 17000, 40000]
    off = np.concatenate([[0], np.cumsum(rng_len)]).astype(np.int64)
    n = int(off[-1])
    k = inputs.keys(n, key_bits, "uniform", seed=21)
    one = np.array(1, dtype=k.dtype)
    seg = [k[off[i]:off[i + 1]] for i in range(len(rng_len))]
    seg[0] &= np.array(0xFFFF, dtype=k.dtype)              # upper digits constant (zero)
    seg[1][:] = seg[1][0]                                   # every pass trivial
    seg[2] = (seg[2] & ~np.array(0xFF00, dtype=k.dtype)) | np.array(0x3400, dtype=k.dtype)
    seg[3] = (seg[3] & np.array(0xFF, dtype=k.dtype)) | np.array(0x5A00, dtype=k.dtype)
    seg[5] = (seg[5] >> np.array(8, dtype=k.dtype)) << np.array(8, dtype=k.dtype)  # digit 0 = 0
    seg[6] = seg[6] & (one << np.array(8 * (key_bits // 8 - 1), dtype=k.dtype)) | \
        np.array(7, dtype=k.dtype)                          # one varying bit, in the top digit
    k = np.concatenate(seg)
    v = inputs.iota(n, val_bits) if val_bits else None
    status, gk, gv = run_segmented(k, off, v)
    assert status == _lib.OK
    want = oracle.segmented_sort(k, off, v)
    if val_bits:
        assert np.array_equal(gk, want[0]) and np.array_equal(gv, want[1])
    else:
        assert np.array_equal(gk, want)


def test_btn_threshold_tuning_keeps_results():
    L = inputs.segment_lengths(800, seed=7, max_log2=13)
    off = inputs.segment_offsets(L)
    k = inputs.keys(int(off[-1]), 32, "and4", seed=8)
    want = oracle.segmented_sort(k, off)
    try:
        for btn_max in (512, 1024, 4096):
            isort.tune_segmented(32, 0, btn_max)
            st, gk, _ = run_segmented(k, off)
            assert st == _lib.OK
            assert np.array_equal(gk, want), btn_max
    finally:
        isort.tune_segmented(32, 0, -1)


def test_single_range_equals_plain_sort():
    n = 300_001
    k = inputs.keys(n, 32, "uniform", seed=9)
    st, gk, _ = run_segmented(k, np.array([0, n], dtype=np.int64))
    assert st == _lib.OK
    assert np.array_equal(gk, oracle.radix_sort(k))


def test_bad_offsets_are_flagged_not_faulted():
    n = 10_000
    k = inputs.keys(n, 32, "uniform", seed=10)
    bad = np.array([0, 5000, 4000, n], dtype=np.int64)  # a decreasing pair
    st, _, _ = run_segmented(k, bad)
    assert st == _lib.EINVAL
    bad_end = np.array([0, 5000, n - 7], dtype=np.int64)  # does not end at total
    st, gk, _ = run_segmented(k, bad_end)
    assert st == _lib.EINVAL
    # valid offsets afterwards: the context is fine and the result exact
    off = np.array([0, 5000, n], dtype=np.int64)
    st, gk, _ = run_segmented(k, off)
    assert st == _lib.OK
    assert np.array_equal(gk, oracle.segmented_sort(k, off))


def test_empty_and_degenerate():
    st, gk, _ = run_segmented(np.zeros(0, np.uint32), np.array([0], dtype=np.int64))
    assert st == _lib.OK and gk.size == 0
    k = inputs.keys(64, 32, "uniform", seed=11)
    off = np.arange(0, 65, dtype=np.int64)  # 64 ranges of one key: identity
    st, gk, _ = run_segmented(k, off)
    assert st == _lib.OK and np.array_equal(gk, k)


@pytest.mark.slow
def test_full_size_20000_ranges():
    """The batched workload itself: 20,000 ranges, lengths log-uniform in [1, 2^20]
    (about 1.5e9 uniform u32 keys), launched as the benchmark launches it, and
    compared with the oracle's per-range sort of the whole batch, element by
    element."""
    L = inputs.segment_lengths(20_000, seed=1)
    off = inputs.segment_offsets(L)
    n = int(off[-1])
    t = inputs.device_keys(n, 32, "uniform", seed=1)
    before = t.cpu().numpy()
    d_off = torch.from_numpy(off).cuda()
    isort.sort_segmented(t, d_off)
    assert isort.stream_status() == _lib.OK
    after = t.cpu().numpy()
    del t
    torch.cuda.empty_cache()
    want = oracle.segmented_sort(before, off)
    del before
    assert np.array_equal(after, want)
