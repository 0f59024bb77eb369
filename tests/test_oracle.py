"""Pins for the serial C oracle against things other than itself.

* brute force: Python's comparison sort on (key, index) for tiny inputs;
* a library routine: numpy's stable argsort for medium inputs;
* hand-worked count-sort rounds (tests/golden/count_sort_rounds.txt);
* special cases with closed forms (all-equal, sorted, reversed distinct keys);
* invariants (non-decreasing, same multiset via per-digit histograms, stability);
* planted mistakes: mutated copies of oracle.c must fail at least one pin.
"""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import inputs
import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden", "count_sort_rounds.txt")
SIZES_TINY = [0, 1, 2, 3, 7, 31, 32, 33, 100, 255, 256, 257, 1000]


def brute_force_stable(keys, vals):
    """Comparison sort on (key, input index): the plain stable order."""
    order = sorted(range(len(keys)), key=lambda i: (int(keys[i]), i))
    return keys[order], vals[order]


def load_golden():
    cases, cur = [], None
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        tok = line.split()
        if tok[0] == "case":
            cur = {"name": tok[1]}
            cases.append(cur)
        elif tok[0] == "shift":
            cur["shift"], cur["bits"] = int(tok[1]), int(tok[3])
        elif tok[0] == "key_bits":
            cur["key_bits"] = int(tok[1])
        elif tok[0] in ("keys_in", "keys_out"):
            cur[tok[0]] = [int(t, 16) for t in tok[1:]]
        else:
            cur[tok[0]] = [int(t) for t in tok[1:]]
    return cases


@pytest.mark.parametrize("case", load_golden(), ids=lambda c: c["name"])
def test_golden_rounds(case):
    dt = np.uint32 if case["key_bits"] == 32 else np.uint64
    k = np.array(case["keys_in"], dtype=dt)
    v = np.array(case["vals_in"], dtype=np.uint32)
    ko, vo = oracle.count_sort_round(k, case["shift"], case["bits"], v)
    assert ko.tolist() == case["keys_out"]
    assert vo.tolist() == case["vals_out"]


def test_golden_two_rounds_make_a_sort():
    cases = {c["name"]: c for c in load_golden()}
    c0 = cases["two_rounds_round0"]
    k = np.array(c0["keys_in"], dtype=np.uint32)
    v = np.array(c0["vals_in"], dtype=np.uint32)
    # an 8-bit key sorted with two hex rounds == the whole-sort result; the upper
    # 24 bits are zero, so the remaining rounds of a radix-16 sort are identity
    ks, vs = oracle.radix_sort(k, v, radix_bits=4)
    assert ks.tolist() == cases["two_rounds_round1"]["keys_out"]
    assert vs.tolist() == cases["two_rounds_round1"]["vals_out"]


@pytest.mark.parametrize("key_bits", [32, 64])
@pytest.mark.parametrize("dist", inputs.DISTS)
@pytest.mark.parametrize("radix_bits", [1, 4, 8, 11, 16])
def test_brute_force_tiny(key_bits, dist, radix_bits):
    for n in SIZES_TINY:
        k = inputs.keys(n, key_bits, dist, seed=3)
        v = inputs.iota(n)
        ks, vs = oracle.radix_sort(k, v, radix_bits=radix_bits)
        bk, bv = brute_force_stable(k, v)
        assert np.array_equal(ks, bk), (n, dist)
        assert np.array_equal(vs, bv), (n, dist)
        assert np.array_equal(oracle.radix_sort(k, radix_bits=radix_bits), bk)


@pytest.mark.parametrize("key_bits", [32, 64])
@pytest.mark.parametrize("dist", inputs.DISTS)
def test_numpy_stable_argsort_medium(key_bits, dist):
    n = 200_003
    k = inputs.keys(n, key_bits, dist, seed=7)
    v = inputs.iota(n, 64)
    ref = np.argsort(k, kind="stable")
    for rb in (8, 11, 16):
        ks, vs = oracle.radix_sort(k, v, radix_bits=rb)
        assert np.array_equal(ks, k[ref])
        assert np.array_equal(vs, ref.astype(np.uint64))


def test_special_cases():
    n = 5000
    v = inputs.iota(n)
    eq = inputs.keys(n, 32, "equal", 1)
    ks, vs = oracle.radix_sort(eq, v)
    assert np.array_equal(vs, v) and np.array_equal(ks, eq)  # identity
    srt = inputs.keys(n, 32, "sorted", 1)
    ks, vs = oracle.radix_sort(srt, v)
    assert np.array_equal(vs, v) and np.array_equal(ks, srt)  # already sorted: identity
    distinct = np.arange(n, dtype=np.uint32)[::-1] * np.uint32(977) + np.uint32(5)
    ks, vs = oracle.radix_sort(distinct, v)
    assert np.array_equal(vs, v[::-1])  # reversed distinct keys: reversal


def digit_histograms(k, key_bits, radix_bits):
    out = []
    for p in range(-(-key_bits // radix_bits)):
        d = (k >> k.dtype.type(p * radix_bits)) & k.dtype.type((1 << radix_bits) - 1)
        out.append(np.bincount(d.astype(np.int64), minlength=1 << radix_bits))
    return out


@pytest.mark.parametrize("dist", inputs.DISTS)
def test_invariants(dist):
    n = 1 << 18
    k = inputs.keys(n, 32, dist, seed=11)
    v = inputs.iota(n)
    ks, vs = oracle.radix_sort(k, v, radix_bits=8)
    assert (ks[1:] >= ks[:-1]).all()
    for a, b in zip(digit_histograms(k, 32, 8), digit_histograms(ks, 32, 8)):
        assert np.array_equal(a, b)
    assert np.array_equal(k[vs], ks)  # payload = index: out_key[i] == in_key[out_val[i]]
    assert np.array_equal(np.sort(vs), v)  # payloads are a permutation
    same = ks[1:] == ks[:-1]
    assert (vs[1:][same] > vs[:-1][same]).all()  # stability


def test_segmented_matches_per_segment_numpy():
    L = inputs.segment_lengths(300, seed=2, max_log2=12)
    L[5] = 0  # empty segments are allowed
    L[6] = 0
    off = inputs.segment_offsets(L)
    k = inputs.keys(int(off[-1]), 32, "and4", seed=2)
    v = inputs.iota(int(off[-1]))
    ks, vs = oracle.segmented_sort(k, off, v, radix_bits=8)
    for s in range(len(L)):
        a, b = off[s], off[s + 1]
        o = np.argsort(k[a:b], kind="stable")
        assert np.array_equal(ks[a:b], k[a:b][o])
        assert np.array_equal(vs[a:b], v[a:b][o])


def test_bad_arguments_rejected():
    with pytest.raises(RuntimeError):
        oracle.radix_sort(np.zeros(4, np.uint32), radix_bits=0)
    with pytest.raises(RuntimeError):
        oracle.segmented_sort(np.zeros(4, np.uint32), np.array([0, 3, 2, 4]))
    with pytest.raises(RuntimeError):
        oracle.count_sort_round(np.zeros(4, np.uint32), 30, 4)  # digit past the key width
    assert oracle.num_passes(32, 8) == 4 and oracle.num_passes(32, 11) == 3
    assert oracle.num_passes(32, 16) == 2 and oracle.num_passes(64, 8) == 8


# ---- GVR sample sort (Algorithm 3) ------------------------------------------
def gvr_definition(k, p, s, seed):
    """Splitters and bucket sizes recomputed with numpy from the algorithm's
    definitions: sample positions from the inputs module's SplitMix64 (stream
    30), splitters = the (i*s)-th smallest sampled keys, bucket j = the keys
    above splitter j-1 and at most splitter j."""
    n = k.size
    if n == 0:
        return np.zeros(max(p - 1, 0), np.uint64), np.zeros(p, np.int64)
    d = inputs.draws_u64(seed, 30, 0, s * p - 1)
    pos = ((d >> np.uint64(32)) * np.uint64(n)) >> np.uint64(32)
    sample = np.sort(k[pos.astype(np.int64)].astype(np.uint64))
    split = sample[np.arange(1, p) * s - 1]
    srt = np.sort(k).astype(np.uint64)
    edges = np.concatenate([[0], np.searchsorted(srt, split, side="right"), [n]])
    return split, np.diff(edges)


@pytest.mark.parametrize("key_bits", [32, 64])
@pytest.mark.parametrize("dist", inputs.DISTS)
@pytest.mark.parametrize("p,s", [(1, 1), (2, 3), (16, 8), (256, 16)])
def test_gvr_sorts_stably_and_its_intermediates_follow_the_definition(key_bits, dist, p, s):
    for n in (0, 1, 5, 1000, 20_011):
        k = inputs.keys(n, key_bits, dist, seed=n + 7)
        v = inputs.iota(n)
        ks, vs, counts, split = oracle.gvr_sort(k, v, buckets=p, oversample=s, seed=9)
        order = np.argsort(k, kind="stable")  # a library routine: the stable order
        assert np.array_equal(ks, k[order]) and np.array_equal(vs, v[order]), n
        want_split, want_counts = gvr_definition(k, p, s, 9)
        assert np.array_equal(counts.astype(np.int64), want_counts), n
        if n:
            assert np.array_equal(split, want_split), n


# ---- GSD (Algorithm 1) ------------------------------------------------------
def gsd_definition(k, p, r):
    """Splitters and bucket sizes recomputed with numpy from the algorithm's
    definitions: sequences [n*j/p, n*(j+1)/p) sorted, the keys ending their
    r*p evenly sized segments sampled, splitters = the (i*r*p)-th smallest
    samples, bucket j = the keys above splitter j-1 and at most splitter j."""
    n = k.size
    rp = r * p
    maxkey = np.iinfo(k.dtype).max
    samples = []
    for j in range(p):
        seq = np.sort(k[n * j // p:n * (j + 1) // p]).astype(np.uint64)
        for i in range(1, rp + 1):
            pos = max(i * seq.size // rp - 1, 0)
            samples.append(seq[pos] if seq.size else np.uint64(maxkey))
    samples = np.sort(np.array(samples, dtype=np.uint64))
    split = samples[np.arange(1, p) * rp - 1]
    srt = np.sort(k).astype(np.uint64)
    edges = np.concatenate([[0], np.searchsorted(srt, split, side="right"), [n]])
    return split, np.diff(edges)


@pytest.mark.parametrize("key_bits", [32, 64])
@pytest.mark.parametrize("dist", inputs.DISTS)
@pytest.mark.parametrize("p,r", [(1, 1), (2, 3), (8, 4), (16, 16), (64, 1)])
def test_gsd_sorts_stably_and_its_intermediates_follow_the_definition(key_bits, dist, p, r):
    for n in (0, 1, 5, 63, 1000, 20_011):
        k = inputs.keys(n, key_bits, dist, seed=n + 13)
        v = inputs.iota(n)
        ks, vs, counts, split = oracle.gsd_sort(k, v, buckets=p, oversample=r)
        order = np.argsort(k, kind="stable")
        assert np.array_equal(ks, k[order]) and np.array_equal(vs, v[order]), n
        want_split, want_counts = gsd_definition(k, p, r)
        assert np.array_equal(counts.astype(np.int64), want_counts), n
        assert np.array_equal(split, want_split), n


# ---- planted mistakes -------------------------------------------------------
# Each mutant is a textual edit of oracle.c that a plausible bug would make. None
# writes out of bounds (every output slot stays in [0, n)), so running it is safe.
MUTANTS = {
    "unstable_output_loop": (
        "for (int64_t i = 0; i < n; ++i) {\n    uint64_t k = get_key(keys_in, i, kb);",
        "for (int64_t i = n - 1; i >= 0; --i) {\n    uint64_t k = get_key(keys_in, i, kb);"),
    "digit_off_by_one_bit": ("const uint64_t mask = (uint64_t)r - 1;",
                             "const uint64_t mask = (uint64_t)r - 1;\n  if (shift > 0) shift -= 1;"),
    "msd_first": ("int shift = p * radix_bits;",
                  "int shift = (passes - 1 - p) * radix_bits;"),
    "no_copy_back": ("if (rc == 0 && kin != keys) {", "if (0) {"),
    "payload_not_moved": ("if (vb) copy_val(vals_out, pos, vals_in, i, vb);",
                          "if (vb) copy_val(vals_out, i, vals_in, i, vb);"),
    "narrow_mask": ("const uint64_t mask = (uint64_t)r - 1;",
                    "const uint64_t mask = ((uint64_t)r - 1) >> 1;"),
    "gvr_bucket_takes_equal_keys_up": ("split[j] < k) ++j;", "split[j] <= k) ++j;"),
    "gvr_splitter_rank_off_by_one": ("sample[(int64_t)i * s - 1]", "sample[(int64_t)i * s]"),
    "gsd_sample_position_off_by_one": ("int64_t pos = (int64_t)i * len / rp - 1;",
                                       "int64_t pos = (int64_t)i * len / rp - 2;"),
    "gsd_merge_prefers_later_sequence": ("if (best < 0 || x < bk) {", "if (best < 0 || x <= bk) {"),
    "gsd_split_takes_equal_keys_up": ("if (get_key(keys, mid, kb) <= s)",
                                      "if (get_key(keys, mid, kb) < s)"),
    "gvr_split_round_backwards": (
        "for (int64_t i = 0; i < n; ++i) {\n      const int64_t o = next[dest[i]]++;",
        "for (int64_t i = n - 1; i >= 0; --i) {\n      const int64_t o = next[dest[i]]++;"),
}


def _pins_pass(lib):
    """The pins above, compressed; returns False as soon as one fails."""
    for dist in inputs.DISTS:
        for n in (33, 257, 1000):
            for rb in (8, 11):
                k = inputs.keys(n, 32, dist, seed=3)
                v = inputs.iota(n)
                try:
                    ks, vs = oracle.radix_sort(k, v, radix_bits=rb, lib=lib)
                except RuntimeError:
                    return False
                bk, bv = brute_force_stable(k, v)
                if not (np.array_equal(ks, bk) and np.array_equal(vs, bv)):
                    return False
    for dist in ("uniform", "u16", "and4", "equal"):
        k = inputs.keys(3000, 32, dist, seed=4)
        v = inputs.iota(3000)
        try:
            ks, vs, counts, split = oracle.gvr_sort(k, v, buckets=16, oversample=4, seed=7,
                                                    lib=lib)
        except RuntimeError:
            return False
        order = np.argsort(k, kind="stable")
        want_split, want_counts = gvr_definition(k, 16, 4, 7)
        if not (np.array_equal(ks, k[order]) and np.array_equal(vs, v[order]) and
                np.array_equal(counts.astype(np.int64), want_counts) and
                np.array_equal(split, want_split)):
            return False
    for dist in ("uniform", "u16", "and4", "equal"):
        k = inputs.keys(3000, 32, dist, seed=5)
        v = inputs.iota(3000)
        try:
            ks, vs, counts, split = oracle.gsd_sort(k, v, buckets=8, oversample=4, lib=lib)
        except (RuntimeError, IndexError):
            return False
        order = np.argsort(k, kind="stable")
        want_split, want_counts = gsd_definition(k, 8, 4)
        if not (np.array_equal(ks, k[order]) and np.array_equal(vs, v[order]) and
                np.array_equal(counts.astype(np.int64), want_counts) and
                np.array_equal(split, want_split)):
            return False
    for c in load_golden():
        dt = np.uint32 if c["key_bits"] == 32 else np.uint64
        ko, vo = oracle.count_sort_round(np.array(c["keys_in"], dt), c["shift"], c["bits"],
                                         np.array(c["vals_in"], np.uint32), lib=lib)
        if ko.tolist() != c["keys_out"] or vo.tolist() != c["vals_out"]:
            return False
    return True


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_planted_mistakes_are_caught():
    src = open(os.path.join(os.path.dirname(oracle.__file__), "oracle.c")).read()
    assert _pins_pass(oracle.load_library(oracle.build()))
    with tempfile.TemporaryDirectory() as tmp:
        shutil.copy(os.path.join(os.path.dirname(oracle.__file__), "oracle.h"), tmp)
        for name, (old, new) in MUTANTS.items():
            assert src.count(old) == 1, f"mutant {name} no longer applies to oracle.c"
            path = os.path.join(tmp, f"{name}.c")
            open(path, "w").write(src.replace(old, new))
            so = os.path.join(tmp, f"lib{name}.so")
            subprocess.check_call(["gcc", "-O1", "-std=c99", "-fPIC", "-shared", path, "-o", so])
            assert not _pins_pass(oracle.load_library(so)), f"mutant {name} survived the pins"
