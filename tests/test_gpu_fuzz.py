"""Seeded random cross-check of every sort entry point: random sizes (1 key to
a few million, so tile counts, ragged tails and single partial tiles all
occur), the six key distributions, every radix width, the radix-256 kernel
variants, payload widths, host buffers and segmented batches. Every result is
compared element by element with the oracle on the same input; a failure
prints the case's parameters, which reproduce it."""
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

KINDS = ("keys", "pairs", "host_keys", "host_pairs", "segmented")


def _case(i):
    rng = np.random.default_rng(1000 + i)
    kind = KINDS[i % len(KINDS)]
    key_bits = int(rng.choice([32, 64]))
    val_bits = int(rng.choice([32, 64]))
    radix = int(rng.choice([0, 8, 8, 11, 16]))
    n = int(np.exp(rng.uniform(0.0, np.log(3_000_000))))
    dist = str(rng.choice(inputs.DISTS))
    nvar = len(isort.tune_variants(key_bits, val_bits if "pairs" in kind else 0, 8))
    variant = int(rng.integers(-1, nvar)) if radix in (0, 8) else -1
    seed = int(rng.integers(1, 1 << 30))
    return kind, key_bits, val_bits, radix, n, dist, variant, seed


@pytest.mark.parametrize("i", range(240))
def test_random_case(i):
    kind, key_bits, val_bits, radix, n, dist, variant, seed = _case(i)
    what = f"case {i}: {kind} k{key_bits} v{val_bits} radix {radix} n {n} {dist} variant {variant}"
    k = inputs.keys(n, key_bits, dist, seed=seed)
    pairs = "pairs" in kind
    vb = val_bits if pairs else 0
    v = inputs.iota(n, val_bits) if pairs else None
    isort.tune_set(key_bits, vb, 8, variant)
    try:
        if kind == "segmented":
            lens = inputs.segment_lengths(max(1, n // 5000), seed=seed, max_log2=16)
            off = inputs.segment_offsets(lens)
            m = int(off[-1])
            kk = inputs.keys(m, key_bits, dist, seed=seed)
            d = torch.from_numpy(kk).cuda()
            isort.sort_segmented(d, torch.from_numpy(off).cuda())
            assert isort.stream_status() == _lib.OK, what
            assert np.array_equal(d.cpu().numpy(), oracle.segmented_sort(kk, off)), what
            return
        if pairs:
            ok, ov = oracle.radix_sort(k, v, radix_bits=8)
        else:
            ok = oracle.radix_sort(k, radix_bits=8)
        if kind.startswith("host"):
            hk = torch.from_numpy(k.copy()).pin_memory()
            hout = torch.empty_like(hk).pin_memory()
            if pairs:
                hv = torch.from_numpy(v.copy()).pin_memory()
                hvo = torch.empty_like(hv).pin_memory()
                isort.sort_pairs_host(hk, hv, hout, hvo, radix)
            else:
                isort.sort_keys_host(hk, hout, radix)
            torch.cuda.synchronize()
            assert isort.stream_status() == _lib.OK, what
            assert np.array_equal(hout.numpy(), ok), what
            if pairs:
                assert np.array_equal(hvo.numpy(), ov), what
            return
        dk = torch.from_numpy(k).cuda()
        if pairs:
            dv = torch.from_numpy(v).cuda()
            isort.sort_pairs(dk, dv, radix)
        else:
            isort.sort_keys(dk, radix)
        assert isort.stream_status() == _lib.OK, what
        assert np.array_equal(dk.cpu().numpy(), ok), what
        if pairs:
            assert np.array_equal(dv.cpu().numpy(), ov), what
    finally:
        isort.tune_set(key_bits, vb, 8, -1)
