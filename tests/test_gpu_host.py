"""Host-buffer sorts (isort_keys_host / isort_pairs_host): keys and payloads in
host memory, copied in, sorted and copied out on one stream. Buffers move by
the copy engines; ISORT_DEBUG_HOST_COPY 2 moves pinned, aligned ones by copy
kernels over the host link instead. Every result must equal the
oracle's, bit for bit, and the inputs must be left as they were (out of
place) or sorted (in place)."""
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

SIZES = [2, 5, 3 * 8192 + 4099, (1 << 20) + 3]


@pytest.fixture
def copy_mode():
    def set_mode(m):
        isort.debug_set(_lib.DEBUG_HOST_COPY, m)
    yield set_mode
    isort.debug_set(_lib.DEBUG_HOST_COPY, 0)


def _host_tensor(a, pinned):
    t = torch.from_numpy(a.copy())
    return t.pin_memory() if pinned else t


def _copy_kernels_ran():
    return any(name in ("k_copy_h2d", "k_copy_d2h") for name, _ in isort.kernel_times())


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("in_place", [True, False])
@pytest.mark.parametrize("key_bits", [32, 64])
@pytest.mark.parametrize("n", SIZES)
def test_keys_host(copy_mode, mode, pinned, in_place, key_bits, n):
    k = inputs.keys(n, key_bits, "uniform", seed=21)
    expect = oracle.radix_sort(k, radix_bits=8)
    copy_mode(mode)
    src = _host_tensor(k, pinned)
    out = src if in_place else _host_tensor(np.zeros_like(k), pinned)
    isort.debug_set(_lib.DEBUG_KERNEL_TIMING, 1)
    try:
        isort.sort_keys_host(src, out, 8)
        torch.cuda.synchronize()
        kernels = _copy_kernels_ran()
    finally:
        isort.debug_set(_lib.DEBUG_KERNEL_TIMING, 0)
    assert isort.stream_status() == _lib.OK
    assert np.array_equal(out.numpy(), expect)
    if not in_place:
        assert np.array_equal(src.numpy(), k)  # the input is left as it was
    # only mode 2 takes the copy kernels, and only for pinned, aligned buffers
    assert kernels == (pinned and mode == 2)


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("key_bits,val_bits", [(32, 32), (32, 64), (64, 32), (64, 64)])
@pytest.mark.parametrize("dist", ["uniform", "and4"])
def test_pairs_host(pinned, key_bits, val_bits, dist):
    n = 3 * 8192 + 4099
    k = inputs.keys(n, key_bits, dist, seed=22)
    v = inputs.iota(n, val_bits)
    ok, ov = oracle.radix_sort(k, v, radix_bits=8)
    ks, vs = _host_tensor(k, pinned), _host_tensor(v, pinned)
    ko, vo = _host_tensor(np.zeros_like(k), pinned), _host_tensor(np.zeros_like(v), pinned)
    isort.sort_pairs_host(ks, vs, ko, vo, 8)
    torch.cuda.synchronize()
    assert isort.stream_status() == _lib.OK
    assert np.array_equal(ko.numpy(), ok) and np.array_equal(vo.numpy(), ov)
    assert np.array_equal(ks.numpy(), k) and np.array_equal(vs.numpy(), v)


@pytest.mark.parametrize("radix_bits", [0, 11, 16])
def test_keys_host_every_radix(radix_bits):
    n = 400_003
    k = inputs.keys(n, 32, "uniform", seed=23)
    t = _host_tensor(k, True)
    isort.sort_keys_host(t, radix_bits=radix_bits)
    torch.cuda.synchronize()
    assert isort.stream_status() == _lib.OK
    assert np.array_equal(t.numpy(), np.sort(k))


def test_unaligned_pinned_buffers_take_the_copy_engines(copy_mode):
    """A pinned buffer that does not start on 16 bytes (a slice one key in)
    cannot take the copy kernels even when they are asked for; the copy
    engines move it, and the ragged element count round-trips exactly."""
    n = 100_001
    k = inputs.keys(n + 1, 32, "uniform", seed=24)
    base = _host_tensor(k, True)
    src = base[1:]
    out = torch.zeros(n + 1, dtype=base.dtype).pin_memory()[1:]
    copy_mode(2)
    isort.debug_set(_lib.DEBUG_KERNEL_TIMING, 1)
    try:
        isort.sort_keys_host(src, out, 8)
        torch.cuda.synchronize()
        assert not _copy_kernels_ran()
    finally:
        isort.debug_set(_lib.DEBUG_KERNEL_TIMING, 0)
    assert np.array_equal(out.numpy(), np.sort(k[1:]))


def test_tail_words_by_the_copy_kernel(copy_mode):
    """Copy kernels, pinned, aligned, and a byte count that is not a multiple of
    16: the last 4-byte words go through the tail kernel."""
    copy_mode(2)
    for n in (4 * 1000 + 1, 4 * 1000 + 2, 4 * 1000 + 3):
        k = inputs.keys(n, 32, "uniform", seed=n)
        t = _host_tensor(k, True)
        isort.sort_keys_host(t)
        torch.cuda.synchronize()
        assert np.array_equal(t.numpy(), np.sort(k)), n


def test_one_and_zero_keys():
    k = np.array([7], dtype=np.uint32)
    src, out = _host_tensor(k, True), torch.zeros(1, dtype=torch.uint32).pin_memory()
    isort.sort_keys_host(src, out)
    torch.cuda.synchronize()
    assert out.item() == 7
    empty = torch.empty(0, dtype=torch.uint32)
    isort.sort_keys_host(empty)


def test_binding_rejects_device_tensors():
    d = torch.zeros(8, dtype=torch.uint32, device="cuda")
    with pytest.raises(ValueError):
        isort.sort_keys_host(d)
    with pytest.raises(ValueError):
        isort.sort_keys_host(torch.zeros(8, dtype=torch.uint32), torch.zeros(9, dtype=torch.uint32))


def _round256(x):
    return (x + 255) // 256 * 256


@pytest.mark.parametrize("val_bits", [0, 32])
def test_bound_workspace_size_for_host_sorts(val_bits):
    """The header's size: isort_workspace_size plus the device copies rounded
    up to 256 bytes. A bound workspace of exactly that size sorts; one that
    holds only isort_keys' needs returns ENOMEM and enqueues nothing."""
    n = (1 << 16) + 3
    s = torch.cuda.Stream()
    base = isort.workspace_size(n, 32, val_bits, 8)
    exact = base + _round256(n * 4) + (_round256(n * val_bits // 8) if val_bits else 0)
    k = inputs.keys(n, 32, "uniform", seed=25)
    v = inputs.iota(n, 32)
    try:
        ws = torch.empty(base, dtype=torch.uint8, device="cuda")
        isort.set_workspace(ws, stream=s)
        hk = _host_tensor(k, True)
        with pytest.raises(isort.IsortError):
            if val_bits:
                isort.sort_pairs_host(hk, _host_tensor(v, True), radix_bits=8, stream=s)
            else:
                isort.sort_keys_host(hk, radix_bits=8, stream=s)
        assert np.array_equal(hk.numpy(), k)  # nothing was enqueued
        ws = torch.empty(exact, dtype=torch.uint8, device="cuda")
        isort.set_workspace(ws, stream=s)
        hv = _host_tensor(v, True)
        if val_bits:
            isort.sort_pairs_host(hk, hv, radix_bits=8, stream=s)
        else:
            isort.sort_keys_host(hk, radix_bits=8, stream=s)
        s.synchronize()
        assert isort.stream_status(s) == _lib.OK
        ok, ov = oracle.radix_sort(k, v, radix_bits=8)
        assert np.array_equal(hk.numpy(), ok)
        if val_bits:
            assert np.array_equal(hv.numpy(), ov)
    finally:
        isort.set_workspace(None, stream=s)
