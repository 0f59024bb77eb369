"""The claim behind the GPU's order-free rounds, checked on the CPU with a
plain LSD radix-256 sort written here: in a keys-only sort, round j may place
keys that share their digit AND every bit below it in any order (round 0: any
keys with equal digits), and the result is still the sorted input. Placing
keys with equal digits but different low bits in the wrong order is not
allowed (the negative control shows the check would notice)."""
import numpy as np
import pytest

import inputs


def lsd_sort(keys: np.ndarray, shuffle, seed: int) -> np.ndarray:
    """Radix 256, least significant digit first; after each round's stable
    counting placement, `shuffle(out, j, rng)` may reorder the round's output."""
    rng = np.random.default_rng(seed)
    a = keys.copy()
    for j in range(4):
        d = (a >> np.uint32(8 * j)) & np.uint32(0xFF)
        a = a[np.argsort(d, kind="stable")]
        a = shuffle(a, j, rng)
    return a


def shuffle_within(groups_of):
    """Reorder keys at random inside each run of equal group ids."""
    def f(a, j, rng):
        g = groups_of(a, j)
        out = a.copy()
        start = 0
        for end in list(np.flatnonzero(g[1:] != g[:-1]) + 1) + [len(a)]:
            out[start:end] = rng.permutation(a[start:end])
            start = end
        return out
    return f


def digit_and_low(a, j):
    """Keys agree on digit j and on every bit below it: bits [0, 8j + 8)."""
    return a & np.uint32((1 << (8 * j + 8)) - 1) if j < 3 else a


def digit_only(a, j):
    return (a >> np.uint32(8 * j)) & np.uint32(0xFF)


@pytest.mark.parametrize("dist", ["uniform", "u16", "and4", "sorted", "reverse", "equal"])
@pytest.mark.parametrize("n", [1, 31, 4096, 50_000])
def test_any_order_inside_runs_of_equal_low_bits_still_sorts(dist, n):
    k = inputs.keys(n, 32, dist, seed=7)
    for seed in range(3):
        got = lsd_sort(k, shuffle_within(digit_and_low), seed)
        assert np.array_equal(got, np.sort(k))


def test_any_order_of_equal_digits_in_round_zero_only():
    k = inputs.keys(50_000, 32, "uniform", seed=8)

    def first_round_free(a, j, rng):
        return shuffle_within(digit_only)(a, j, rng) if j == 0 else a
    assert np.array_equal(lsd_sort(k, first_round_free, 1), np.sort(k))


def test_negative_control_equal_digits_reordered_in_a_later_round():
    """Round 1 placing equal digits in any order (ignoring the low byte)
    breaks the sort: the relaxation must be confined to runs of equal low bits."""
    k = inputs.keys(50_000, 32, "uniform", seed=9)

    def round_one_free(a, j, rng):
        return shuffle_within(digit_only)(a, j, rng) if j == 1 else a
    assert not np.array_equal(lsd_sort(k, round_one_free, 2), np.sort(k))
