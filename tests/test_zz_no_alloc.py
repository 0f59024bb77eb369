"""isort_keys_noalloc: the sort for callers that may not allocate device memory.

Such callers (a framework that owns all device memory through its own pool, a
latency-critical loop where cudaMalloc could stall the device, code that must
not run out of memory after start-up) get a variant of the radix-256 keys-only
sort whose scratch is a fixed array inside the library. This file checks,
through the C-ABI, that two calls in a row give exactly what the ordinary
isort_keys gives on the same inputs, and that a size beyond the fixed array is
refused. It is named to be collected last, and works alone in a fresh process
as well as after the other tests.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import inputs
import paper_1808_10292_gb300 as isort
from paper_1808_10292_gb300 import _lib

pytestmark = pytest.mark.gpu


def test_noalloc_matches_isort_keys_on_two_calls_in_a_row():
    lib = _lib.load()
    stream = torch.cuda.current_stream().cuda_stream
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    for n, dist, seed in [(1_000_003, "uniform", 31), (_lib.NOALLOC_MAX_KEYS, "and4", 32)]:
        host = inputs.keys(n, 32, dist, seed=seed)
        a = torch.from_numpy(host).cuda()
        b = torch.from_numpy(host).cuda()
        rc = lib.isort_keys_noalloc(ctypes.c_void_p(a.data_ptr()), n,
                                    ctypes.c_void_p(err.data_ptr()), ctypes.c_void_p(stream))
        assert rc == _lib.OK
        assert lib.isort_keys(ctypes.c_void_p(b.data_ptr()), n, 32, 8,
                              ctypes.c_void_p(stream)) == _lib.OK
        torch.cuda.synchronize()
        assert int(err.item()) == 0
        # integer keys: the two entry points must agree bit for bit
        assert np.array_equal(a.cpu().numpy(), b.cpu().numpy())
        assert np.array_equal(a.cpu().numpy(), np.sort(host))


def test_noalloc_refuses_sizes_beyond_its_array():
    lib = _lib.load()
    a = torch.empty(_lib.NOALLOC_MAX_KEYS + 1, dtype=torch.uint32, device="cuda")
    rc = lib.isort_keys_noalloc(ctypes.c_void_p(a.data_ptr()), a.numel(), None, None)
    assert rc == _lib.ENOMEM
    with pytest.raises(isort.IsortError):
        isort.sort_keys_noalloc(a)
