"""GPU parity: the CUDA sort (through the C-ABI) against the serial C oracle,
element by element on the same seeded inputs. Integer work: bit-exact."""
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
TORCH_DT = {32: torch.uint32, 64: torch.uint64}


def to_dev(a: np.ndarray):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def to_host(t) -> np.ndarray:
    return t.cpu().numpy()


def gpu_sort(keys_np, vals_np=None, radix_bits=8):  # noqa: D401
    k = to_dev(keys_np)
    if vals_np is None:
        isort.sort_keys(k, radix_bits)
        assert isort.stream_status() == _lib.OK
        return to_host(k)
    v = to_dev(vals_np)
    isort.sort_pairs(k, v, radix_bits)
    assert isort.stream_status() == _lib.OK
    return to_host(k), to_host(v)


def edge_sizes(tile):
    # tile edges, and several look-back rows
    return sorted({0, 1, 2, 3, 31, 32, 33, 255, 257, tile - 1, tile, tile + 1, 2 * tile + 5,
                   5 * tile - 3, 8 * tile - 1, 8 * tile + 1, 17 * tile + 3})


def test_device_generator_matches_host_generator():
    for bits in (32, 64):
        for dist in inputs.DISTS:
            for n in (1, 1000, 65_537):
                d = to_host(inputs.device_keys(n, bits, dist, seed=5))
                assert np.array_equal(d, inputs.keys(n, bits, dist, seed=5)), (bits, dist, n)
    assert np.array_equal(to_host(inputs.device_iota(777)), inputs.iota(777))


def test_config1_uniform_2p20_seed1():
    """n = 2^20 uniform u32 keys, seed 1, radix 256, keys only: bit-exact vs the oracle."""
    k = inputs.keys(1 << 20, 32, "uniform", seed=1)
    assert np.array_equal(gpu_sort(k), oracle.radix_sort(k, radix_bits=8))


@pytest.mark.parametrize("key_bits", [32, 64])
@pytest.mark.parametrize("dist", inputs.DISTS)
def test_distributions_keys_only(key_bits, dist):
    n = 1_000_003  # several hundred tiles and a ragged tail
    k = inputs.keys(n, key_bits, dist, seed=9)
    assert np.array_equal(gpu_sort(k), oracle.radix_sort(k, radix_bits=8))


@pytest.mark.parametrize("key_bits,val_bits", [(32, 32), (32, 64), (64, 32), (64, 64)])
@pytest.mark.parametrize("dist", ["uniform", "and4", "equal", "u16"])
def test_pairs_stable(key_bits, val_bits, dist):
    n = 654_321
    k = inputs.keys(n, key_bits, dist, seed=4)
    v = inputs.iota(n, val_bits)
    gk, gv = gpu_sort(k, v)
    ok, ov = oracle.radix_sort(k, v, radix_bits=8)
    assert np.array_equal(gk, ok)
    assert np.array_equal(gv, ov)


@pytest.mark.parametrize("key_bits,val_bits", [(32, 0), (32, 32), (32, 64), (64, 0), (64, 32),
                                               (64, 64)])
def test_every_variant_edge_sizes(key_bits, val_bits):
    variants = isort.tune_variants(key_bits, val_bits, 8)
    assert variants
    try:
        for vi, (threads, kpt) in enumerate(variants):
            isort.tune_set(key_bits, val_bits, 8, vi)
            for n in edge_sizes(threads * kpt):
                k = inputs.keys(n, key_bits, "and4", seed=n + 1)
                if val_bits:
                    v = inputs.iota(n, val_bits)
                    gk, gv = gpu_sort(k, v)
                    ok, ov = oracle.radix_sort(k, v, radix_bits=8)
                    assert np.array_equal(gv, ov), (vi, n)
                else:
                    gk, ok = gpu_sort(k), oracle.radix_sort(k, radix_bits=8)
                assert np.array_equal(gk, ok), (vi, n)
    finally:
        isort.tune_set(key_bits, val_bits, 8, -1)


def test_unaligned_view_and_offsets():
    base = inputs.keys(100_001, 32, "uniform", seed=2)
    t = to_dev(base)
    view = t[1:]  # 4-byte aligned, not 16-byte aligned
    isort.sort_keys(view, 8)
    assert isort.stream_status() == _lib.OK
    got = to_host(t)
    assert got[0] == base[0]
    assert np.array_equal(got[1:], oracle.radix_sort(base[1:], radix_bits=8))


def test_bound_workspace_and_enomem():
    n = 300_000
    k = to_dev(inputs.keys(n, 32, "uniform", seed=3))
    need = isort.workspace_size(n, 32, 0, 8)
    s = torch.cuda.Stream()
    small = torch.empty(need // 2, dtype=torch.uint8, device="cuda")
    isort.set_workspace(small, stream=s)
    with pytest.raises(isort.IsortError) as e:
        isort.sort_keys(k, 8, stream=s)
    assert e.value.status == _lib.ENOMEM
    big = torch.empty(need, dtype=torch.uint8, device="cuda")
    isort.set_workspace(big, stream=s)
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        isort.sort_keys(k, 8)
    assert isort.stream_status(s) == _lib.OK
    assert np.array_equal(to_host(k), np.sort(inputs.keys(n, 32, "uniform", seed=3)))
    isort.set_workspace(None, stream=s)


def test_concurrent_streams_give_the_same_results():
    streams = [torch.cuda.Stream() for _ in range(4)]
    data = [inputs.keys(200_000 + 1000 * i, 32, "and4", seed=20 + i) for i in range(4)]
    ts = [to_dev(d) for d in data]
    torch.cuda.synchronize()
    for s, t in zip(streams, ts):
        with torch.cuda.stream(s):
            isort.sort_keys(t, 8)
    for s, t, d in zip(streams, ts, data):
        assert isort.stream_status(s) == _lib.OK
        assert np.array_equal(to_host(t), oracle.radix_sort(d, radix_bits=8))


@pytest.mark.parametrize("variant", [0, -1])
def test_bounded_wait_reports_timeout_and_context_survives(variant):
    """A tile that never publishes makes its successors' bounded waits give up:
    the error is latched and reported, no GPU hang, and the next sort is fine."""
    n = 64 * 4096  # many look-back rows
    k = to_dev(inputs.keys(n, 32, "uniform", seed=6))
    nv = len(isort.tune_variants(32, 0, 8))
    isort.tune_set(32, 0, 8, variant % nv)  # the default and the last variant
    isort.debug_set(_lib.DEBUG_SPIN_LIMIT, 2000)
    isort.debug_set(_lib.DEBUG_STALL_TILE, 1)
    try:
        isort.sort_keys(k, 8)
        assert isort.stream_status() == _lib.ETIMEOUT
        assert isort.stream_status() == _lib.OK  # cleared once reported
    finally:
        isort.debug_set(_lib.DEBUG_STALL_TILE, -1)
        isort.debug_set(_lib.DEBUG_SPIN_LIMIT, 0)
        isort.tune_set(32, 0, 8, -1)
    d = inputs.keys(n, 32, "uniform", seed=7)
    assert np.array_equal(gpu_sort(d), np.sort(d))


R16_TILE = 8192  # keys per tile of the radix-65536 steps (32-bit keys alone)


@pytest.mark.parametrize("key_bits", [32, 64])
@pytest.mark.parametrize("dist", inputs.DISTS)
def test_radix65536_distributions(key_bits, dist):
    n = 1_234_567  # 256 buckets of a few tiles each, ragged bucket ends
    k = inputs.keys(n, key_bits, dist, seed=12)
    assert np.array_equal(gpu_sort(k, radix_bits=16), oracle.radix_sort(k, radix_bits=16))


@pytest.mark.parametrize("key_bits,val_bits", [(32, 32), (32, 64), (64, 32), (64, 64)])
@pytest.mark.parametrize("dist", ["uniform", "and4", "u16"])
def test_radix65536_pairs_stable(key_bits, val_bits, dist):
    n = 700_001
    k = inputs.keys(n, key_bits, dist, seed=13)
    v = inputs.iota(n, val_bits)
    gk, gv = gpu_sort(k, v, radix_bits=16)
    ok, ov = oracle.radix_sort(k, v, radix_bits=16)
    assert np.array_equal(gk, ok)
    assert np.array_equal(gv, ov)


def test_radix65536_edge_sizes():
    for n in sorted({0, 1, 2, 3, 4095, 4096, 4097, 9000, R16_TILE - 1, R16_TILE, R16_TILE + 1,
                     256 * R16_TILE + 3, 600_001}):
        k = inputs.keys(n, 32, "and4", seed=n + 3)
        v = inputs.iota(n)
        gk, gv = gpu_sort(k, v, radix_bits=16)
        ok, ov = oracle.radix_sort(k, v, radix_bits=16)
        assert np.array_equal(gk, ok), n
        assert np.array_equal(gv, ov), n


R11_BLOCK = 1 << 16  # a size scale of the radix-2048 tests (tiles, buckets, ragged ends)


@pytest.mark.parametrize("key_bits", [32, 64])
@pytest.mark.parametrize("dist", inputs.DISTS)
def test_radix2048_distributions(key_bits, dist):
    """Radix 2048: 11-bit digits, the last one narrower (11, 11, 10 bits on
    32-bit keys; five of 11 and one of 9 on 64-bit keys)."""
    n = 1_234_567  # 19 count blocks, a ragged last block and sub-tile
    k = inputs.keys(n, key_bits, dist, seed=14)
    assert np.array_equal(gpu_sort(k, radix_bits=11), oracle.radix_sort(k, radix_bits=11))


@pytest.mark.parametrize("key_bits,val_bits", [(32, 32), (32, 64), (64, 32), (64, 64)])
@pytest.mark.parametrize("dist", ["uniform", "and4", "u16"])
def test_radix2048_pairs_stable(key_bits, val_bits, dist):
    n = 300_007
    k = inputs.keys(n, key_bits, dist, seed=15)
    v = inputs.iota(n, val_bits)
    gk, gv = gpu_sort(k, v, radix_bits=11)
    ok, ov = oracle.radix_sort(k, v, radix_bits=11)
    assert np.array_equal(gk, ok)
    assert np.array_equal(gv, ov)


def test_radix2048_edge_sizes():
    for n in sorted({0, 1, 2, 3, 4095, 4096, 4097, R11_BLOCK - 1, R11_BLOCK, R11_BLOCK + 1,
                     3 * R11_BLOCK + 4097}):
        k = inputs.keys(n, 32, "and4", seed=n + 5)
        v = inputs.iota(n)
        gk, gv = gpu_sort(k, v, radix_bits=11)
        ok, ov = oracle.radix_sort(k, v, radix_bits=11)
        assert np.array_equal(gk, ok), n
        assert np.array_equal(gv, ov), n


@pytest.mark.slow
@pytest.mark.parametrize("dist", ["uniform", "and4"])
def test_full_size_2p28_u32_radix2048(dist):
    """n = 2^28 u32 keys at radix 2048 (three passes), element by element."""
    n = 1 << 28
    t = inputs.device_keys(n, 32, dist, seed=1)
    host_in = to_host(t)
    isort.sort_keys(t, 11)
    assert isort.stream_status() == _lib.OK
    got = to_host(t)
    del t
    torch.cuda.empty_cache()
    assert np.array_equal(got, oracle.radix_sort(host_in, radix_bits=11))


@pytest.mark.slow
@pytest.mark.parametrize("dist", inputs.DISTS)
def test_full_size_2p28_u32_radix65536(dist):
    """n = 2^28 u32 keys at radix 65536 (two passes), element by element."""
    n = 1 << 28
    t = inputs.device_keys(n, 32, dist, seed=1)
    host_in = to_host(t)
    isort.sort_keys(t, 16)
    assert isort.stream_status() == _lib.OK
    got = to_host(t)
    del t
    torch.cuda.empty_cache()
    assert np.array_equal(got, oracle.radix_sort(host_in, radix_bits=16))


@pytest.mark.slow
@pytest.mark.parametrize("dist", inputs.DISTS)
def test_full_size_2p28_u32_radix256(dist):
    """The benchmark workload: n = 2^28 u32 keys, radix 256, launched exactly as
    bench.py launches it (default variant, device-generated keys); compared with
    the oracle element by element."""
    n = 1 << 28
    t = inputs.device_keys(n, 32, dist, seed=1)
    host_in = to_host(t)
    isort.sort_keys(t, 8)
    assert isort.stream_status() == _lib.OK
    got = to_host(t)
    del t
    torch.cuda.empty_cache()
    assert np.array_equal(got, oracle.radix_sort(host_in, radix_bits=8))


@pytest.mark.slow
def test_full_size_pairs_2p27_and_u64_2p26():
    n = 1 << 27
    k = inputs.device_keys(n, 32, "uniform", seed=1)
    v = inputs.device_iota(n, 32)
    kin = to_host(k)
    isort.sort_pairs(k, v, 8)
    assert isort.stream_status() == _lib.OK
    ok, ov = oracle.radix_sort(kin, inputs.iota(n), radix_bits=8)
    assert np.array_equal(to_host(k), ok)
    assert np.array_equal(to_host(v), ov)
    del k, v
    n = 1 << 26
    k = inputs.device_keys(n, 64, "uniform", seed=1)
    kin = to_host(k)
    isort.sort_keys(k, 8)
    assert isort.stream_status() == _lib.OK
    assert np.array_equal(to_host(k), oracle.radix_sort(kin, radix_bits=8))


@pytest.mark.slow
def test_max_size_2p30_u32():
    """n = 2^30, the largest n the 30-bit look-back counts allow: the output is
    non-decreasing and every digit histogram (each byte position) of the
    output equals the input's -- the paper's invariants, which hold at any size
    -- and the first and last 2^20 keys equal the oracle's sort of the whole
    input at those positions (the oracle sorts the 4 GiB input on the host)."""
    n = 1 << 30
    t = inputs.device_keys(n, 32, "uniform", seed=3)
    before = [torch.bincount(((t.view(torch.int32) >> (8 * b)) & 0xFF).to(torch.int64),
                             minlength=256) for b in range(4)]
    isort.sort_keys(t, 8)
    assert isort.stream_status() == _lib.OK
    sk = t.view(torch.int32) ^ (-(1 << 31))  # unsigned order as signed
    assert bool((sk[1:] >= sk[:-1]).all())
    del sk
    for b in range(4):
        after = torch.bincount(((t.view(torch.int32) >> (8 * b)) & 0xFF).to(torch.int64),
                               minlength=256)
        assert torch.equal(after, before[b]), b
    head, tail = to_host(t[: 1 << 20]), to_host(t[-(1 << 20):])
    del t
    torch.cuda.empty_cache()
    src = to_host(inputs.device_keys(n, 32, "uniform", seed=3))  # the same input, again
    want = oracle.radix_sort(src, radix_bits=8)
    assert np.array_equal(head, want[: 1 << 20]) and np.array_equal(tail, want[-(1 << 20):])


def kernels_of_one_sort(run):
    isort.debug_set(_lib.DEBUG_KERNEL_TIMING, 1)
    try:
        run()
        torch.cuda.synchronize()
        return [name for name, _ in isort.kernel_times()]
    finally:
        isort.debug_set(_lib.DEBUG_KERNEL_TIMING, 0)


@pytest.mark.parametrize("key_bits", [32, 64])
def test_keys_only_first_round_is_order_free_and_exact(key_bits):
    """Keys only: pass 0 runs the order-free first round (k_onesweep_first),
    the other passes the ordered round; pairs keep the stable round in pass 0.
    Either way the result is the oracle's, bit for bit."""
    n = 3 * 8192 * 5 + 77  # many tiles of every variant, a ragged tail
    k = inputs.keys(n, key_bits, "uniform", seed=31)
    want = oracle.radix_sort(k, radix_bits=8)
    for v in range(len(isort.tune_variants(key_bits, 0, 8))):
        isort.tune_set(key_bits, 0, 8, v)
        try:
            t = to_dev(k)
            names = kernels_of_one_sort(lambda: isort.sort_keys(t, 8))
            assert isort.stream_status() == _lib.OK
            assert np.array_equal(to_host(t), want), v
        finally:
            isort.tune_set(key_bits, 0, 8, -1)
        passes = key_bits // 8
        rounds = names.count("k_onesweep_first") + names.count("k_onesweep")
        assert rounds == passes, names
        assert names.index("k_onesweep_first") < names.index("k_onesweep"), names
    v = inputs.iota(n)
    t, tv = to_dev(k), to_dev(v)
    names = kernels_of_one_sort(lambda: isort.sort_pairs(t, tv, 8))
    assert "k_onesweep_first" not in names
    wk, wv = oracle.radix_sort(k, v, radix_bits=8)
    assert np.array_equal(to_host(t), wk) and np.array_equal(to_host(tv), wv)


@pytest.mark.parametrize("key_bits", [32, 64])
def test_keys_only_constant_low_digit(key_bits):
    """Digit 0 constant: pass 0 is skipped inside the order-free kernel, and the
    first executed round is the stable one. Digits 0 and 1 constant as well."""
    n = 100_003
    base = inputs.keys(n, key_bits, "uniform", seed=32)
    for shift in (8, 16):
        k = (base >> np.array(shift, dtype=base.dtype)) << np.array(shift, dtype=base.dtype)
        k = k | np.array(0x5A, dtype=base.dtype)  # digit 0 = 0x5A, not zero
        assert np.array_equal(gpu_sort(k), oracle.radix_sort(k, radix_bits=8)), shift


def crafted_runs(n, low_values, seed):
    """Keys whose low 8 (then 16) bits take few values, so that rounds 1 and 2
    see long runs of equal low bits next to warps that straddle a change of
    them, plus bursts of up to 31 consecutive distinct low bytes (several run
    starts in one 32-key row) and partial warps in the ragged last tile."""
    hi = inputs.keys(n, 32, "uniform", seed=seed) & np.uint32(0xFFFF0000)
    mid = (inputs.keys(n, 32, "uniform", seed=seed + 1) % np.uint32(low_values)) << np.uint32(8)
    lo = inputs.keys(n, 32, "uniform", seed=seed + 2) % np.uint32(low_values)
    k = hi | mid | lo
    for start in range(700, n - 64, 1500):
        burst = 1 + (start // 1500) % 31
        k[start:start + burst] = (k[start:start + burst] & np.uint32(0xFFFFFF00)) | \
            np.arange(burst, dtype=np.uint32)
    return k


@pytest.mark.parametrize("mode", [0, 2])
@pytest.mark.parametrize("low_values", [1, 3, 40])
def test_keys_only_ordered_rounds_crafted_runs(low_values, mode):
    """Keys only, rounds after the first: the ordered round's check compares
    every staged key with its successor in the key bits below the digit. Runs
    of equal low bits, bursts of distinct ones and ragged tiles, with the fast
    ranks as the hardware gives them (mode 0) and deliberately unstable (mode
    2, the check must repair every failing tile); every variant and the
    segmented form."""
    n = 5 * 8192 + 1234
    k = crafted_runs(n, low_values, 41)
    want = oracle.radix_sort(k, radix_bits=8)
    isort.debug_set(_lib.DEBUG_CHECK_MODE, mode)
    try:
        for v in range(len(isort.tune_variants(32, 0, 8))):
            isort.tune_set(32, 0, 8, v)
            try:
                assert np.array_equal(gpu_sort(k), want), v
            finally:
                isort.tune_set(32, 0, 8, -1)
        self_check_segmented(k, n)
    finally:
        isort.debug_set(_lib.DEBUG_CHECK_MODE, 0)


def self_check_segmented(k, n):
    # the segmented form on the same keys: ranges of mixed lengths
    off = np.array([0, 7, 4000, 4001, 20000, n], dtype=np.int64)
    t = to_dev(k)
    isort.sort_segmented(t, to_dev(off))
    assert isort.stream_status() == _lib.OK
    assert np.array_equal(to_host(t), oracle.segmented_sort(k, off))
