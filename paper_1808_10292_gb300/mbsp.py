"""The paper's MBSP cost model (Section "Implementations": "MBSP model" and
"SR4, PR2, PR4, BTN and OET under MBSP"; Theorem 1 for GSD), and the same
accounting applied to this library's GPU rounds.

MBSP charges g per word moved to or from main memory and G per word accessed
in fast memory; latency terms (l, L) are ignored, as in the paper. Words are
32-bit. The paper's formulas for sorting n 32-bit keys on p workers (N = n/p
per worker, radix r, 32 / lg r rounds):

  Ts(N)       = (32/lg r) (3Ng + 2NG)                      Eq. Ts  (SR4, serial)
  Tp(n, p)    = (32/lg r) (4Ng + 2NG + 2prg)               Eq. Tp  (PR4, PR2)
  To(n, p)    = Ts(n/p) + p (4n/p) g                       Eq. To  (OET)
  Tb(n, p)    = Ts(n/p) + lg p (lg p + 1)/2 (4n/p) g       Eq. Tb  (BTN)
  Tgsd(n, p)  = Ts(n/p) + 5 G n_max lg p,
                n_max = (1 + 1/ceil(w)) n/p + ceil(w) p    Theorem 1 (GSD)

On the GPU the worker of a round is a tile (one CTA), the main memory is HBM
and the fast memory is shared memory. A round of this library moves each key
(and payload) once in and once out of HBM -- the upfront histogram and the
decoupled look-back replace the paper's second read -- and touches shared
memory a fixed number of times per key; the wide radixes keep the paper's
count-sort structure (two reads, one write) and its 2prg count-matrix exchange
with p = count-matrix blocks. gpu_* below give those costs in the same (g, G)
currency; calibrate() derives g from a measured copy bandwidth and G from one
measured round, and predict() turns the model into times for other rounds.

Host-side arithmetic only: nothing here launches GPU work.
"""
from __future__ import annotations

import math


# ---- the paper's formulas ---------------------------------------------------
def rounds(key_bits: int, r: int) -> int:
    """32 / lg r rounds for 32-bit keys (Eqs. Ts, Tp); ceil(key_bits / lg r) in general."""
    return -(-key_bits // int(math.log2(r)))


def Ts(N: float, g: float, G: float, r: int = 256, key_bits: int = 32) -> float:
    """Eq. Ts: serial radix-r sort of N keys (each round reads twice, writes once)."""
    return rounds(key_bits, r) * (3 * N * g + 2 * N * G)


def Tp(n: float, g: float, G: float, p: int, r: int = 256, key_bits: int = 32) -> float:
    """Eq. Tp: parallel radix-r sort (PR4 for r = 2^8, PR2 for r = 2^16) on p workers."""
    N = n / p
    return rounds(key_bits, r) * (4 * N * g + 2 * N * G + 2 * p * r * g)


def To(n: float, g: float, G: float, p: int) -> float:
    """Eq. To: local SR4 of n/p keys, then p rounds of odd-even transposition merge-splits."""
    return Ts(n / p, g, G) + p * (4 * n / p) * g


def Tb(n: float, g: float, G: float, p: int) -> float:
    """Eq. Tb: local SR4, then lg p (lg p + 1) / 2 bitonic merge-split stages."""
    lg = math.log2(p)
    return Ts(n / p, g, G) + (lg * (lg + 1) / 2) * (4 * n / p) * g


def n_max(n: float, p: int, omega: float) -> float:
    """Theorem 1: the largest output sequence of GSD (bucket expansion 1 + 1/ceil(w))."""
    w = math.ceil(omega)
    return (1 + 1 / w) * (n / p) + w * p


def Tgsd(n: float, G: float, p: int, omega: float) -> float:
    """Theorem 1 (g = 5G): GSD's time, Ts(n/p, G) + 5 G n_max lg p."""
    return Ts(n / p, 5 * G, G) + 5 * G * n_max(n, p, omega) * math.log2(p)


def speedup_bound_pr4(p: int) -> float:
    """Observation 5: Ts(n) / Tp(n) for large n with g = 5G, r = 256: 68p / 88."""
    return 68 * p / 88


def speedup_bound_gsd(p: int) -> float:
    """Observation 6: Ts(n) / (Ts(n/p) + 6 G n lg p / p) = 68p / (68 + 6 lg p)."""
    return 68 * p / (68 + 6 * math.log2(p))


# ---- the same accounting for this library's rounds --------------------------
# Shared-memory word accesses per key of one radix-256 round (early counts):
# count, mark, mask read, counter update (by one lane per digit group, counted
# per key), key store, mask clear, staged read, offset read.
SHARED_ACCESSES_ONESWEEP = 8
# The first round of a keys-only sort keeps no order among equal digits:
# count add, slot add (its return value is the tile slot), key store, staged
# read, offset read.
SHARED_ACCESSES_FIRST = 5
# Per key of a wide-radix scatter: two stable 8-bit partitions (mark, mask read,
# counter, store of key and index each), the run pass (read key and index, run
# edges) and the offset update.
SHARED_ACCESSES_WIDE = 16


def gpu_onesweep_round(n: float, words_per_item: float, g: float, G: float,
                       shared: float = SHARED_ACCESSES_ONESWEEP) -> float:
    """One radix-256 round: one read and one write of every key (and payload)
    word in HBM, `shared` shared-memory accesses per key."""
    return 2 * n * words_per_item * g + shared * n * G


def gpu_histogram(n: float, key_words: float, passes: int, g: float, G: float) -> float:
    """The upfront histogram: one read of every key, one shared atomic per key and pass."""
    return n * key_words * g + passes * n * G


def gpu_wide_round(n: float, words_per_item: float, key_words: float, g: float, G: float,
                   r: int, blocks: int, shared: float = SHARED_ACCESSES_WIDE) -> float:
    """One wide-radix round: the count read (n key words + one shared add per
    key), the count-matrix exchange 2 * blocks * r words (the paper's 2prg), and
    the scatter (read and write every item, `shared` accesses per key)."""
    return (n * key_words * g + n * G + 2 * blocks * r * g +
            2 * n * words_per_item * g + shared * n * G)


def relaxed_share(n: float, j: int, radix_bits: int = 8, warp_keys: int = 1024) -> float:
    """Keys only, uniform keys: the share of warps of round j that place keys
    in any order. Round 0 is order-free; round j >= 1 reads input sorted by the
    j*radix_bits low bits, which come in runs of n / 2^(j*radix_bits) equal
    values, and a warp of warp_keys consecutive keys relaxes when no run ends
    inside it."""
    if j == 0:
        return 1.0
    run = n / 2.0 ** (radix_bits * j)
    return max(0.0, 1.0 - (warp_keys - 1) / run) if run >= warp_keys else 0.0


def gpu_sort(n: float, key_bits: int, val_bits: int, r: int, g: float, G: float,
             block_keys: int | None = None) -> float:
    """Model time of one whole sort of n keys at radix r (all rounds executed).
    Keys only at radix 256: the first round is order-free, and for 32-bit
    keys the warps of later rounds that share their low bits (relaxed_share,
    uniform keys) cost what the order-free round costs."""
    kw = key_bits / 32
    w = kw + val_bits / 32
    P = rounds(key_bits, r)
    if r == 256:
        t = gpu_histogram(n, kw, P, g, G)
        for j in range(P):
            f = 0.0
            if val_bits == 0 and (j == 0 or key_bits == 32):
                f = relaxed_share(n, j)
            shared = f * SHARED_ACCESSES_FIRST + (1 - f) * SHARED_ACCESSES_ONESWEEP
            t += gpu_onesweep_round(n, w, g, G, shared)
        return t
    blocks = -(-int(n) // (block_keys or (1 << 19 if r == 65536 else 1 << 16)))
    return P * gpu_wide_round(n, w, kw, g, G, r, blocks)


def calibrate(hbm_gbs: float, onesweep_round_s: float, n: float, words_per_item: float = 1.0,
              shared: float = SHARED_ACCESSES_ONESWEEP) -> dict:
    """g from the measured copy bandwidth (seconds per 4-byte word, whole GPU);
    G from one measured radix-256 round, charging it the paper's additive cost
    2 n w g + shared n G. Returns {"g": g, "G": G, "g_over_G": g / G}."""
    g = 4.0 / (hbm_gbs * 1e9)
    G = (onesweep_round_s - 2 * n * words_per_item * g) / (shared * n)
    return {"g": g, "G": G, "g_over_G": g / G if G > 0 else float("inf")}


def network_time_ratio(q: int, local_share: float) -> float:
    """OET over BTN time for q-thread networks when the local sort and the
    loads and stores take `local_share` of BTN's time (Eqs. To and Tb: the
    network parts are q rounds against lg q (lg q + 1) / 2 stages)."""
    lg = math.log2(q)
    stages = lg * (lg + 1) / 2
    return local_share + (1 - local_share) * q / stages
