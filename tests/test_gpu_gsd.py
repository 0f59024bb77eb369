"""GPU parity of GSD (Algorithm 1) with the oracle's GSD: the sorted keys and
payloads element by element, and the bucket sizes (deterministic: they depend
on the input only)."""
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


def gpu_gsd(k, v=None, p=16, r=4):
    dk = torch.from_numpy(k).cuda()
    dv = None if v is None else torch.from_numpy(v).cuda()
    counts = torch.zeros(p, dtype=torch.int32, device="cuda")
    isort.gsd_sort(dk, dv, buckets=p, oversample=r, bucket_counts=counts)
    st = isort.stream_status()
    return (st, dk.cpu().numpy(), None if dv is None else dv.cpu().numpy(),
            counts.cpu().numpy().astype(np.uint32))


@pytest.mark.parametrize("key_bits,val_bits", [(32, 0), (32, 32), (32, 64), (64, 0), (64, 32),
                                               (64, 64)])
@pytest.mark.parametrize("dist", inputs.DISTS)
def test_gsd_matches_oracle(key_bits, val_bits, dist):
    n = 555_557  # 16 sequences of ~34,722 keys; merge tiles with ragged ends
    k = inputs.keys(n, key_bits, dist, seed=61)
    v = inputs.iota(n, val_bits) if val_bits else None
    st, gk, gv, gc = gpu_gsd(k, v, p=16, r=4)
    assert st == _lib.OK
    if v is None:
        ok, oc, _ = oracle.gsd_sort(k, buckets=16, oversample=4)
    else:
        ok, ov, oc, _ = oracle.gsd_sort(k, v, buckets=16, oversample=4)
        assert np.array_equal(gv, ov)
    assert np.array_equal(gk, ok)
    assert np.array_equal(gc, oc)


@pytest.mark.parametrize("p,r", [(1, 1), (2, 1), (2, 5), (4, 16), (8, 64), (32, 2), (64, 1)])
def test_gsd_bucket_and_oversampling_edges(p, r):
    for n in (0, 1, 2, 3, 63, 64, 65, 2047, 2048, 2049, 2303, 2304, 2305, 3839, 3840, 3841, 4609, 7681, 100_003):
        k = inputs.keys(n, 32, "and4", seed=n + 17)
        v = inputs.iota(n)
        st, gk, gv, gc = gpu_gsd(k, v, p=p, r=r)
        assert st == _lib.OK
        if n == 0:
            continue
        ok, ov, oc, _ = oracle.gsd_sort(k, v, buckets=p, oversample=r)
        assert np.array_equal(gk, ok), (p, r, n)
        assert np.array_equal(gv, ov), (p, r, n)
        assert np.array_equal(gc, oc), (p, r, n)


def test_gsd_argument_errors():
    k = torch.zeros(10, dtype=torch.int32, device="cuda")
    L = _lib.load()
    assert L.isort_gsd_sort(k.data_ptr(), None, 10, 32, 0, 3, 1, None, None) == _lib.EINVAL
    assert L.isort_gsd_sort(k.data_ptr(), None, 10, 32, 0, 128, 1, None, None) == _lib.EINVAL
    assert L.isort_gsd_sort(k.data_ptr(), None, 10, 32, 0, 16, 17, None, None) == _lib.EINVAL
    assert L.isort_gsd_sort(k.data_ptr(), None, 10, 32, 0, 16, 0, None, None) == _lib.EINVAL


@pytest.mark.slow
@pytest.mark.parametrize("dist", ["uniform", "and4"])
def test_full_size_2p28_gsd(dist):
    """2^28 uint32 keys, p = 16, r = 4, as the benchmark runs it; element by
    element against the oracle's GSD (keys and bucket sizes)."""
    n = 1 << 28
    t = inputs.device_keys(n, 32, dist, seed=1)
    host_in = t.cpu().numpy()
    counts = torch.zeros(16, dtype=torch.int32, device="cuda")
    isort.gsd_sort(t, buckets=16, oversample=4, bucket_counts=counts)
    assert isort.stream_status() == _lib.OK
    got = t.cpu().numpy()
    del t
    torch.cuda.empty_cache()
    ok, oc, _ = oracle.gsd_sort(host_in, buckets=16, oversample=4)
    assert np.array_equal(got, ok)
    assert np.array_equal(counts.cpu().numpy().astype(np.uint32), oc)
