"""GPU parity of the GVR sample sort (Algorithm 3) with the oracle's GVR: the
sorted keys and payloads element by element, and the bucket sizes (which depend
on the sample: both sides draw it from the same counter-based generator)."""
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


def gpu_sample_sort(k, v=None, p=256, s=16, seed=1):
    dk = torch.from_numpy(k).cuda()
    dv = None if v is None else torch.from_numpy(v).cuda()
    counts = torch.zeros(p, dtype=torch.int32, device="cuda")
    isort.sample_sort(dk, dv, buckets=p, oversample=s, seed=seed, bucket_counts=counts)
    st = isort.stream_status()
    return (st, dk.cpu().numpy(), None if dv is None else dv.cpu().numpy(),
            counts.cpu().numpy().astype(np.uint32))


@pytest.mark.parametrize("key_bits,val_bits", [(32, 0), (32, 32), (32, 64), (64, 0), (64, 32),
                                               (64, 64)])
@pytest.mark.parametrize("dist", inputs.DISTS)
def test_sample_sort_matches_oracle(key_bits, val_bits, dist):
    n = 777_777  # many split tiles, a ragged tail; buckets of ~3000 keys (BTN and radix ranges)
    k = inputs.keys(n, key_bits, dist, seed=51)
    v = inputs.iota(n, val_bits) if val_bits else None
    st, gk, gv, gc = gpu_sample_sort(k, v, p=256, s=16, seed=3)
    assert st == _lib.OK
    if v is None:
        ok, oc, _ = oracle.gvr_sort(k, buckets=256, oversample=16, seed=3)
    else:
        ok, ov, oc, _ = oracle.gvr_sort(k, v, buckets=256, oversample=16, seed=3)
        assert np.array_equal(gv, ov)
    assert np.array_equal(gk, ok)
    assert np.array_equal(gc, oc)


@pytest.mark.parametrize("p,s", [(1, 1), (2, 1), (3, 7), (64, 64), (256, 1), (256, 16), (128, 32)])
def test_sample_sort_bucket_and_oversampling_edges(p, s):
    for n in (0, 1, 2, 3, 255, 256, 8191, 8192, 8193, 100_003):
        k = inputs.keys(n, 32, "and4", seed=n + 11)
        v = inputs.iota(n)
        st, gk, gv, gc = gpu_sample_sort(k, v, p=p, s=s, seed=n + 1)
        assert st == _lib.OK
        if n == 0:
            continue
        ok, ov, oc, _ = oracle.gvr_sort(k, v, buckets=p, oversample=s, seed=n + 1)
        assert np.array_equal(gk, ok), (p, s, n)
        assert np.array_equal(gv, ov), (p, s, n)
        assert np.array_equal(gc, oc), (p, s, n)


def test_sample_sort_argument_errors():
    k = torch.zeros(10, dtype=torch.int32, device="cuda")
    L = _lib.load()
    assert L.isort_sample_sort(k.data_ptr(), None, 10, 32, 0, 0, 4, 1, None, None) == _lib.EINVAL
    assert L.isort_sample_sort(k.data_ptr(), None, 10, 32, 0, 257, 4, 1, None, None) == _lib.EINVAL
    assert L.isort_sample_sort(k.data_ptr(), None, 10, 32, 0, 256, 17, 1, None, None) == _lib.EINVAL
    assert L.isort_sample_sort(k.data_ptr(), None, 10, 32, 0, 16, 0, 1, None, None) == _lib.EINVAL


@pytest.mark.slow
@pytest.mark.parametrize("dist", ["uniform", "and4"])
def test_full_size_2p28_sample_sort(dist):
    """2^28 uint32 keys, 256 buckets, oversampling 16, as the benchmark runs it;
    element by element against the oracle's GVR (keys and bucket sizes)."""
    n = 1 << 28
    t = inputs.device_keys(n, 32, dist, seed=1)
    host_in = t.cpu().numpy()
    counts = torch.zeros(256, dtype=torch.int32, device="cuda")
    isort.sample_sort(t, buckets=256, oversample=16, seed=1, bucket_counts=counts)
    assert isort.stream_status() == _lib.OK
    got = t.cpu().numpy()
    del t
    torch.cuda.empty_cache()
    ok, oc, _ = oracle.gvr_sort(host_in, buckets=256, oversample=16, seed=1)
    assert np.array_equal(got, ok)
    assert np.array_equal(counts.cpu().numpy().astype(np.uint32), oc)
