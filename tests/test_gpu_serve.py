"""Serving loop on the GPU: every request's result in the mix is the same as
the result of sorting it alone (bit for bit), and matches the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import inputs
import oracle
import paper_1808_10292_gb300 as isort
from paper_1808_10292_gb300 import serve

pytestmark = pytest.mark.gpu


def make_fill(rid, n, pay):
    def fill(keys, vals, stream):
        inputs.device_keys(n, 32, "uniform", seed=3, stream=inputs.STREAM_REQUEST_BASE + rid,
                           out=keys, cuda_stream=stream)
        if vals is not None:
            inputs.device_iota(n, 32, out=vals, cuda_stream=stream)
    return fill


def collect():
    got = {}

    def done(r, keys, vals):
        got[r.rid] = (keys.cpu().numpy(), None if vals is None else vals.cpu().numpy())
    return got, done


@pytest.mark.parametrize("batching,rate", [(True, 20000.0), (False, 20000.0), (True, 400.0)])
def test_each_result_alone_equals_in_the_mix(batching, rate):
    """At 20,000 req/s requests queue up and share batches (segmented sorts);
    at 400 req/s most arrive to an idle server and run alone (plain sorts)."""
    count = 300 if rate > 1000 else 80
    arrivals, sizes, payload = inputs.requests(count, seed=2, rate=rate, min_log2=10,
                                               max_log2=17)
    got, done = collect()
    srv = serve.SortServer(budget_bytes=256 << 20, num_streams=3, max_batch_keys=1 << 20,
                           max_batch_requests=64, batching=batching)
    reqs = serve.drive(srv, arrivals, sizes, payload, make_fill, duration_s=1e9, done=done)
    srv.close()
    assert not srv.errors
    assert len(got) == len(reqs) == count
    if batching and rate > 1000:
        assert srv.batches < len(reqs)  # requests really were batched
    for r in reqs:
        k, v = got[r.rid]
        alone_k = torch.empty(r.n, dtype=torch.uint32, device="cuda")
        alone_v = torch.empty(r.n, dtype=torch.uint32, device="cuda") if r.payload else None
        make_fill(r.rid, r.n, r.payload)(alone_k, alone_v, torch.cuda.current_stream())
        if r.payload:
            isort.sort_pairs(alone_k, alone_v, 8)
            assert np.array_equal(v, alone_v.cpu().numpy())
        else:
            isort.sort_keys(alone_k, 8)
        assert np.array_equal(k, alone_k.cpu().numpy())
        if r.rid % 37 == 0:  # and a sample against the oracle
            host = inputs.keys(r.n, 32, "uniform", seed=3, stream=inputs.STREAM_REQUEST_BASE + r.rid)
            if r.payload:
                ok, ov = oracle.radix_sort(host, inputs.iota(r.n))
                assert np.array_equal(k, ok) and np.array_equal(v, ov)
            else:
                assert np.array_equal(k, oracle.radix_sort(host))


def test_admission_budget_refuses_what_can_never_fit_and_serves_the_rest():
    arrivals = np.array([0.0, 0.0, 0.0, 0.0])
    sizes = np.array([1 << 12, 1 << 22, 1 << 13, 1 << 12])  # 16 MiB request > 8 MiB budget
    payload = np.array([False, False, True, False])
    got, done = collect()
    srv = serve.SortServer(budget_bytes=8 << 20, num_streams=2, max_batch_keys=1 << 20,
                           max_batch_requests=8)
    reqs = serve.drive(srv, arrivals, sizes, payload, make_fill, duration_s=1.0, done=done)
    srv.close()
    assert not srv.errors
    assert [r.rid for r in srv.rejected] == [1]
    assert sorted(got) == [0, 2, 3] and len(reqs) == 3
    for rid in got:
        k, _ = got[rid]
        assert (k[1:] >= k[:-1]).all()


def test_cancelled_requests_never_run_and_the_rest_are_exact():
    """A tight budget keeps most requests queued; the second half is withdrawn
    right after submission. Withdrawn requests never reach the GPU or their done
    callback; every request that ran gives the result of sorting it alone."""
    got, done = collect()
    n = 1 << 18
    srv = serve.SortServer(budget_bytes=2 * n * 4, num_streams=1, max_batch_keys=n,
                           max_batch_requests=1)
    reqs = []
    import time
    for rid in range(24):
        r = serve.Request(rid=rid, n=n, payload=False, arrival=time.perf_counter(),
                          fill=make_fill(rid, n, False), done=done)
        assert srv.submit(r)
        reqs.append(r)
    withdrawn = {r.rid for r in reqs[12:] if srv.cancel(r)}
    srv.close()
    assert not srv.errors
    assert len(withdrawn) > 0  # the budget held them in the queue
    assert set(got) == {r.rid for r in reqs} - withdrawn
    assert {r.rid for r in srv.cancelled} == withdrawn
    for rid, (k, _) in got.items():
        alone = inputs.keys(n, 32, "uniform", seed=3, stream=inputs.STREAM_REQUEST_BASE + rid)
        assert np.array_equal(k, oracle.radix_sort(alone))
