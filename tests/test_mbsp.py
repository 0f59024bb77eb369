"""The MBSP cost model (paper_1808_10292_gb300/mbsp.py) against the closed
forms and numbers the paper prints for g = 5G (tests/golden/mbsp_paper_values.txt),
and the GPU-round accounting against its own definitions. CPU only."""
import math
import os

import pytest

from paper_1808_10292_gb300 import mbsp

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "mbsp_paper_values.txt")
G = 1.0
g = 5 * G  # the paper's g = 5G
SIZES = [(8_192_000, 4), (32_768_000, 16), (131_072_000, 32), (1_000_000, 2)]


def golden_names():
    names = []
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            names.append(line.split("|")[0].strip())
    return names


def test_golden_file_lists_every_pinned_form():
    assert golden_names() == ["Ts_g5G", "Tp_r256_g5G", "Tp_r65536_g5G", "To_g5G", "Tb_g5G",
                              "obs5_ratio", "obs5_bounds", "obs6_bounds"]


@pytest.mark.parametrize("n,p", SIZES)
def test_general_formulas_reduce_to_the_printed_closed_forms(n, p):
    N = n / p
    assert mbsp.Ts(N, g, G) == pytest.approx(68 * N * G)                            # Eq. TsG
    assert mbsp.Tp(n, g, G, p) == pytest.approx((88 * n / p + 40 * 256 * p) * G)   # Eq. Tp4
    assert mbsp.Tp(n, g, G, p, r=65536) == pytest.approx(
        (44 * n / p + 20 * 256 ** 2 * p) * G)                                        # Eq. Tp2
    assert mbsp.To(n, g, G, p) == pytest.approx((68 * n / p + 20 * n) * G)          # Eq. ToG
    lg = math.log2(p)
    assert mbsp.Tb(n, g, G, p) == pytest.approx(
        (68 * n / p + 10 * n * lg * (lg + 1) / p) * G)                               # Eq. TbG


def test_observation_5_speedup_bounds():
    n = 10 ** 12  # "for large n"
    for p in (4, 8, 16):
        assert mbsp.Ts(n, g, G) / mbsp.Tp(n, g, G, p) == pytest.approx(
            mbsp.speedup_bound_pr4(p), rel=1e-4)
    assert [round(mbsp.speedup_bound_pr4(p)) for p in (4, 8, 16)] == [3, 6, 12]
    assert mbsp.speedup_bound_pr4(1) == pytest.approx(0.77, abs=0.005)


def test_observation_6_speedup_bounds():
    got = [mbsp.speedup_bound_gsd(p) for p in (4, 8, 16)]
    assert got[0] == pytest.approx(3.4, abs=0.005)
    assert got[1] == pytest.approx(6.3, abs=0.05)
    assert got[2] == pytest.approx(11.82, abs=0.01)
    # Theorem 1 with n_max = 1.2 n/p is the same expression
    n, p = 10 ** 9, 8
    Tg = mbsp.Ts(n / p, g, G) + 6 * G * n * math.log2(p) / p
    assert mbsp.Ts(n, g, G) / Tg == pytest.approx(mbsp.speedup_bound_gsd(p))


def test_gsd_bucket_expansion():
    # n_max = (1 + 1/ceil(w)) n/p + ceil(w) p; w = 4.2 -> ceil 5
    assert mbsp.n_max(1_000_000, 10, 4.2) == pytest.approx(1.2 * 100_000 + 50)
    assert mbsp.Tgsd(1_000_000, G, 8, 4) == pytest.approx(
        68 * 125_000 + 5 * mbsp.n_max(1_000_000, 8, 4) * 3)


def test_rounds_and_gpu_accounting():
    assert [mbsp.rounds(32, r) for r in (256, 2048, 65536)] == [4, 3, 2]
    assert mbsp.rounds(64, 256) == 8 and mbsp.rounds(64, 2048) == 6
    n, gg = 1 << 28, 4 / 6784e9
    # with free shared memory a radix-256 round costs its algorithmic HBM bytes
    assert mbsp.gpu_onesweep_round(n, 1, gg, 0.0) == pytest.approx(2 * n * 4 / 6784e9)
    assert mbsp.gpu_onesweep_round(n, 2, gg, 0.0) == pytest.approx(2 * n * 8 / 6784e9)
    # a wide round: its histogram read and two routing steps (3 reads, 2 writes)
    assert mbsp.gpu_wide_round(n, 1, 1, gg, 0.0) == pytest.approx(5 * n * gg)
    # radix 65536: two rounds plus the byte-histogram read of the buckets
    assert mbsp.gpu_sort(n, 32, 0, 65536, gg, 0.0) == pytest.approx(11 * n * gg)
    assert mbsp.gpu_sort(n, 32, 0, 2048, gg, 0.0) == pytest.approx(15 * n * gg)
    # a whole radix-256 sort: histogram read + 4 rounds
    assert mbsp.gpu_sort(n, 32, 0, 256, gg, 0.0) == pytest.approx(9 * n * gg)


def test_calibration_recovers_its_inputs():
    n, hbm = 1 << 28, 6784.2
    gg = 4 / (hbm * 1e9)
    GG = gg / 7.5
    t = mbsp.gpu_onesweep_round(n, 1, gg, GG)
    c = mbsp.calibrate(hbm, t, n)
    assert c["g"] == pytest.approx(gg) and c["G"] == pytest.approx(GG)
    assert c["g_over_G"] == pytest.approx(7.5)


def test_network_ratio_limits():
    # no local work: the ratio of q rounds to lg q (lg q + 1) / 2 stages
    assert mbsp.network_time_ratio(256, 0.0) == pytest.approx(256 / 36)
    assert mbsp.network_time_ratio(32, 0.0) == pytest.approx(32 / 15)
    assert mbsp.network_time_ratio(64, 1.0) == pytest.approx(1.0)


def test_gpu_sort_ordered_rounds():
    """Keys only at radix 256: the order-free first round saves the check's
    read (5 shared accesses per key against 6); pairs run the ordered round
    with the index and payload accesses (11) in every round."""
    n, g, G = 1 << 20, 2.0, 1.0
    ordered = mbsp.gpu_histogram(n, 1, 4, g, G) + 4 * mbsp.gpu_onesweep_round(n, 1, g, G)
    assert mbsp.gpu_sort(n, 32, 0, 256, g, G) == pytest.approx(ordered - n * G)
    pairs = mbsp.gpu_histogram(n, 1, 4, g, G) + 4 * mbsp.gpu_onesweep_round(n, 2, g, G, 11)
    assert mbsp.gpu_sort(n, 32, 32, 256, g, G) == pytest.approx(pairs)
    t64 = mbsp.gpu_sort(n, 64, 0, 256, g, G)
    assert t64 == pytest.approx(mbsp.gpu_histogram(n, 2, 8, g, G) +
                                8 * mbsp.gpu_onesweep_round(n, 2, g, G) - n * G)
