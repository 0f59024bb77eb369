"""Canary words around a caller-bound workspace: every entry point (radix 256,
2048 and 65536 sorts, pairs, the segmented sort, GVR and GSD) writes only
inside the bytes it was given, and each result matches the oracle."""
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

CANARY = 1 << 20  # bytes of seeded pattern on each side of the workspace


def test_workspace_canaries_survive_every_entry_point():
    n = 300_001
    L = inputs.segment_lengths(200, seed=71, max_log2=13)
    off = inputs.segment_offsets(L)
    need = max(isort.workspace_size(n, 32, 32, 8), isort.workspace_size(n, 64, 64, 8),
               isort.workspace_size(n, 32, 0, 11), isort.workspace_size(n, 32, 0, 16),
               isort.segmented_workspace_size(len(L), int(off[-1]), 32, 32),
               isort.sample_sort_workspace_size(n, 32, 32, 256, 16),
               isort.gsd_sort_workspace_size(n, 32, 32, 16, 4))
    need = (need + 255) // 256 * 256
    buf = torch.empty(need + 2 * CANARY, dtype=torch.uint8, device="cuda")
    g = torch.Generator(device="cpu").manual_seed(7)
    pattern = torch.randint(0, 256, (CANARY,), dtype=torch.uint8, generator=g).cuda()
    buf[:CANARY] = pattern
    buf[-CANARY:] = pattern
    s = torch.cuda.Stream()
    isort.set_workspace(buf[CANARY:CANARY + need], stream=s)

    def intact():
        torch.cuda.synchronize()
        return bool(torch.equal(buf[:CANARY], pattern) and torch.equal(buf[-CANARY:], pattern))

    def run(fn):
        with torch.cuda.stream(s):
            fn()
        assert isort.stream_status(s) == _lib.OK
        assert intact()

    try:
        k32 = inputs.keys(n, 32, "and4", seed=72)
        v32 = inputs.iota(n, 32)
        k64 = inputs.keys(n, 64, "uniform", seed=73)
        v64 = inputs.iota(n, 64)
        for rb in (8, 11, 16):
            t = torch.from_numpy(k32).cuda()
            run(lambda: isort.sort_keys(t, rb))
            assert np.array_equal(t.cpu().numpy(), oracle.radix_sort(k32, radix_bits=rb))
        tk, tv = torch.from_numpy(k64).cuda(), torch.from_numpy(v64).cuda()
        run(lambda: isort.sort_pairs(tk, tv, 8))
        ok, ov = oracle.radix_sort(k64, v64)
        assert np.array_equal(tk.cpu().numpy(), ok) and np.array_equal(tv.cpu().numpy(), ov)
        m = int(off[-1])
        sk = torch.from_numpy(k32[:m].copy()).cuda()
        sv = torch.from_numpy(v32[:m].copy()).cuda()
        d_off = torch.from_numpy(off).cuda()
        run(lambda: isort.sort_segmented(sk, d_off, sv))
        ok, ov = oracle.segmented_sort(k32[:m], off, v32[:m])
        assert np.array_equal(sk.cpu().numpy(), ok) and np.array_equal(sv.cpu().numpy(), ov)
        for name in ("gvr", "gsd"):
            tk, tv = torch.from_numpy(k32).cuda(), torch.from_numpy(v32).cuda()
            if name == "gvr":
                run(lambda: isort.sample_sort(tk, tv, buckets=256, oversample=16, seed=5))
            else:
                run(lambda: isort.gsd_sort(tk, tv, buckets=16, oversample=4))
            order = np.argsort(k32, kind="stable")
            assert np.array_equal(tk.cpu().numpy(), k32[order]), name
            assert np.array_equal(tv.cpu().numpy(), v32[order]), name
    finally:
        isort.set_workspace(None, stream=s)
