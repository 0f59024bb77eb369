"""Pins for the seeded input generator (host side)."""
import numpy as np
import pytest

import inputs


def test_splitmix64_published_vector():
    # SplitMix64 started from state 0 yields e220a8397b1dcdaf, 6e789e6aa1b965f4,
    # 06c45d188009454f (the reference sequence of Steele, Lea & Flood's generator,
    # as shipped with xoshiro's seeding code). S(0, 0) = mix64(0) = 0, so our
    # draws for seed 0, stream 0 must be exactly that sequence.
    d = inputs.draws_u64(0, 0, 0, 3)
    assert [int(x) for x in d] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_numpy_matches_integer_formula():
    for seed, stream in [(1, 0), (1, 5), (12345, 1000), (2**63 + 7, 20)]:
        s = inputs.stream_key(seed, stream)
        want = [inputs.mix64_int(s + (i + 1) * inputs.GAMMA) for i in range(50)]
        got = inputs.draws_u64(seed, stream, 0, 50)
        assert [int(x) for x in got] == want
        # offset windows agree with the full sequence
        assert [int(x) for x in inputs.draws_u64(seed, stream, 17, 5)] == want[17:22]


@pytest.mark.parametrize("bits", [32, 64])
def test_distribution_shapes(bits):
    n = 1 << 14
    u = inputs.keys(n, bits, "uniform", 1)
    assert u.dtype == (np.uint32 if bits == 32 else np.uint64)
    assert len(np.unique(u)) > n - 10
    s16 = inputs.keys(n, bits, "u16", 1)
    assert int(s16.max()) < 1 << 16 and len(np.unique(s16)) > 1000
    eq = inputs.keys(n, bits, "equal", 1)
    assert (eq == eq[0]).all()
    srt = inputs.keys(n, bits, "sorted", 1)
    assert (np.diff(srt.astype(np.float64)) >= 0).all()
    rev = inputs.keys(n, bits, "reverse", 1)
    assert (np.diff(rev.astype(np.float64)) <= 0).all()
    a4 = inputs.keys(n, bits, "and4", 1)
    # each bit of an AND of four independent uniform words is set w.p. 1/16
    density = np.unpackbits(a4.view(np.uint8)).mean()
    assert abs(density - 1 / 16) < 0.005


def test_sorted_spans_every_digit():
    k = inputs.keys(1 << 16, 32, "sorted", 1)
    for p in range(4):
        assert len(np.unique((k >> np.uint32(8 * p)) & np.uint32(255))) == 256


def test_segments_and_requests():
    L = inputs.segment_lengths(20000, 1)
    assert L.min() >= 1 and L.max() <= 1 << 20
    off = inputs.segment_offsets(L)
    assert off[0] == 0 and off[-1] == L.sum() and (np.diff(off) == L).all()
    # log-uniform lengths: mean close to (2^20 - 1) / (20 ln 2) ~ 75,639
    assert abs(L.mean() / inputs.lengths_mean() - 1) < 0.08
    arr, sizes, pay = inputs.requests(5000, 1)
    assert (np.diff(arr) >= 0).all()
    assert abs(5000 / arr[-1] / 2000 - 1) < 0.06
    assert sizes.min() >= 1 << 10 and sizes.max() <= 1 << 24
    assert abs(pay.mean() - 0.5) < 0.03
