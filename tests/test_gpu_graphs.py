"""CUDA-graph capture of the library calls: with a workspace bound to the
capturing stream, isort_keys / isort_pairs / isort_segmented enqueue only
kernels and stream-ordered memsets, so a captured call replays on new inputs
written into the same buffers. Every replay is compared with the oracle."""
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


def _capture(stream, fn):
    with torch.cuda.stream(stream):  # first call outside the capture: kernel attributes set
        fn()
    stream.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        fn()
    return g


def test_segmented_sort_in_a_graph_replays_exactly():
    L = inputs.segment_lengths(600, seed=21, max_log2=15)  # every class, radix ranges too
    off = inputs.segment_offsets(L)
    n = int(off[-1])
    s = torch.cuda.Stream()
    ws = torch.empty(isort.segmented_workspace_size(len(L), n, 32, 32), dtype=torch.uint8,
                     device="cuda")
    isort.set_workspace(ws, stream=s)
    try:
        keys = torch.from_numpy(inputs.keys(n, 32, "uniform", seed=20)).cuda()
        vals = torch.from_numpy(inputs.iota(n, 32)).cuda()
        d_off = torch.from_numpy(off).cuda()
        g = _capture(s, lambda: isort.sort_segmented(keys, d_off, vals))
        for seed, dist in ((22, "and4"), (23, "uniform")):
            k = inputs.keys(n, 32, dist, seed=seed)
            v = inputs.iota(n, 32)
            keys.copy_(torch.from_numpy(k))
            vals.copy_(torch.from_numpy(v))
            torch.cuda.synchronize()
            g.replay()
            torch.cuda.synchronize()
            assert isort.stream_status(s) == _lib.OK
            ok, ov = oracle.segmented_sort(k, off, v)
            assert np.array_equal(keys.cpu().numpy(), ok)
            assert np.array_equal(vals.cpu().numpy(), ov)
    finally:
        isort.set_workspace(None, stream=s)


@pytest.mark.parametrize("key_bits,val_bits,radix_bits", [(32, 0, 8), (64, 32, 8), (32, 0, 11)])
def test_plain_sort_in_a_graph_replays_exactly(key_bits, val_bits, radix_bits):
    n = 1_000_003
    s = torch.cuda.Stream()
    ws = torch.empty(isort.workspace_size(n, key_bits, val_bits, radix_bits), dtype=torch.uint8,
                     device="cuda")
    isort.set_workspace(ws, stream=s)
    try:
        keys = torch.from_numpy(inputs.keys(n, key_bits, "uniform", seed=30)).cuda()
        vals = torch.from_numpy(inputs.iota(n, val_bits)).cuda() if val_bits else None
        if val_bits:
            fn = lambda: isort.sort_pairs(keys, vals, radix_bits)  # noqa: E731
        else:
            fn = lambda: isort.sort_keys(keys, radix_bits)  # noqa: E731
        g = _capture(s, fn)
        for seed in (31, 32):
            k = inputs.keys(n, key_bits, "u16" if seed == 31 else "reverse", seed=seed)
            keys.copy_(torch.from_numpy(k))
            if val_bits:
                vals.copy_(torch.from_numpy(inputs.iota(n, val_bits)))
            torch.cuda.synchronize()
            g.replay()
            torch.cuda.synchronize()
            assert isort.stream_status(s) == _lib.OK
            if val_bits:
                ok, ov = oracle.radix_sort(k, inputs.iota(n, val_bits), radix_bits=radix_bits)
                assert np.array_equal(vals.cpu().numpy(), ov)
            else:
                ok = oracle.radix_sort(k, radix_bits=radix_bits)
            assert np.array_equal(keys.cpu().numpy(), ok)
    finally:
        isort.set_workspace(None, stream=s)
