"""The autotuner on the GPU: it times the kernel variants and radix widths on a
small sort, its choice is loaded into the library (radix_bits = 0 resolves to
it) and the sort with that choice stays bit-exact with the oracle."""
import json

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import inputs
import oracle
import paper_1808_10292_gb300 as isort
from paper_1808_10292_gb300 import _lib, tune

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("key_bits,val_bits", [(32, 0), (32, 32), (64, 0)])
def test_tuned_choice_is_applied_and_exact(tmp_path, key_bits, val_bits):
    n = (1 << 18) + 77
    try:
        res = tune.tune_plain(n, key_bits, val_bits, reps=1)
        best = res["best"]
        assert {r["radix_bits"] for r in res["all"]} == {8, 11, 16}
        assert best["ms"] == min(r["ms"] for r in res["all"])
        path = tmp_path / "cache.json"
        path.write_text(json.dumps({torch.cuda.get_device_name():
                                    {tune.plain_key(key_bits, val_bits, n): res}}))
        tune.apply_all(path=str(path))
        assert isort.resolve(n, key_bits, val_bits, 0) == (best["radix_bits"],
                                                           best.get("variant", 0))
        k = inputs.keys(n, key_bits, "and4", seed=7)
        dk = torch.from_numpy(k).cuda()
        if val_bits:
            v = inputs.iota(n)
            dv = torch.from_numpy(v).cuda()
            isort.sort_pairs(dk, dv, 0)
            ok, ov = oracle.radix_sort(k, v, radix_bits=8)
            assert isort.stream_status() == _lib.OK
            assert np.array_equal(dv.cpu().numpy(), ov)
        else:
            isort.sort_keys(dk, 0)
            ok = oracle.radix_sort(k, radix_bits=8)
            ok = ok[0] if isinstance(ok, tuple) else ok
            assert isort.stream_status() == _lib.OK
        assert np.array_equal(dk.cpu().numpy(), ok)
    finally:
        isort.tune_auto(key_bits, val_bits, -1, -1)
