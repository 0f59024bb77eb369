"""isort_keys_noalloc: the sort for callers that may not allocate device memory.

Such callers (a framework that owns all device memory through its own pool, a
latency-critical loop where cudaMalloc could stall the device, code that must
not run out of memory after start-up) get a variant of the radix-256 keys-only
sort whose scratch is a fixed array inside the library. This file checks,
through the C-ABI, that two calls in a row give exactly what the ordinary
isort_keys gives on the same inputs, that the calls allocate nothing, that the
required error word is enforced, and that a size beyond the fixed array is
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


def test_noalloc_allocates_nothing():
    host = inputs.keys(300_007, 32, "uniform", seed=33)
    keys = torch.from_numpy(host).cuda()
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    side = torch.cuda.Stream()  # a stream that has never had a workspace
    torch.cuda.synchronize()
    ws_before = isort.workspace_bytes()
    torch_before = torch.cuda.memory_allocated()
    with torch.cuda.stream(side):
        isort.sort_keys_noalloc(keys, err)
    side.synchronize()
    assert isort.workspace_bytes() == ws_before
    assert torch.cuda.memory_allocated() == torch_before
    assert int(err.item()) == 0
    assert np.array_equal(keys.cpu().numpy(), np.sort(host))


def test_noalloc_requires_its_error_word():
    lib = _lib.load()
    a = torch.from_numpy(inputs.keys(1000, 32, "uniform", seed=34)).cuda()
    assert lib.isort_keys_noalloc(ctypes.c_void_p(a.data_ptr()), a.numel(), None,
                                  None) == _lib.EINVAL
    with pytest.raises(ValueError):
        isort.sort_keys_noalloc(a, None)
    with pytest.raises(ValueError):
        isort.sort_keys_noalloc(a, torch.zeros(1, dtype=torch.int32))        # host tensor
    with pytest.raises(ValueError):
        isort.sort_keys_noalloc(a, torch.zeros(1, dtype=torch.int64, device="cuda"))


def test_noalloc_refuses_sizes_beyond_its_array():
    lib = _lib.load()
    a = torch.empty(_lib.NOALLOC_MAX_KEYS + 1, dtype=torch.uint32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = lib.isort_keys_noalloc(ctypes.c_void_p(a.data_ptr()), a.numel(),
                                ctypes.c_void_p(err.data_ptr()), None)
    assert rc == _lib.ENOMEM
    with pytest.raises(isort.IsortError):
        isort.sort_keys_noalloc(a, err)
