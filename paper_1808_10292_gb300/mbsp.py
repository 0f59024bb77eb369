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
and the fast memory is shared memory. A radix-256 round of this library moves
each key (and payload) once in and once out of HBM -- the upfront histogram
and the decoupled look-back replace the paper's second read -- and touches
shared memory a fixed number of times per key; a wide-radix round reads the
keys for its digit histogram and then routes them in two such rounds (at
radix 65536 after one more read of the keys before round 0, for the buckets). gpu_*
below give those costs in the same (g, G) currency; calibrate() derives g from
a measured copy bandwidth and G from one measured round.

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
# Shared-memory accesses per key of one ordered round (keys only): count add,
# slot add (its return value is the key's tile slot), key store, staged read,
# digit-offset read, and the check's read of the next staged key.
SHARED_ACCESSES_ORDERED = 6
# With payloads, in addition: the input-index store and read, the check's read
# of the next index, the payload's copy into shared memory and its gather.
SHARED_ACCESSES_PAYLOAD = 5
# The first round of a keys-only sort keeps no order among equal digits and
# is not checked: count add, slot add, key store, staged read, offset read.
SHARED_ACCESSES_FIRST = 5


def gpu_onesweep_round(n: float, words_per_item: float, g: float, G: float,
                       shared: float = SHARED_ACCESSES_ORDERED) -> float:
    """One radix-256 round: one read and one write of every key (and payload)
    word in HBM, `shared` shared-memory accesses per key."""
    return 2 * n * words_per_item * g + shared * n * G


def gpu_histogram(n: float, key_words: float, passes: int, g: float, G: float) -> float:
    """The upfront histogram: one read of every key, one shared atomic per key and pass."""
    return n * key_words * g + passes * n * G


def gpu_wide_round(n: float, words_per_item: float, key_words: float, g: float, G: float,
                   shared: float = SHARED_ACCESSES_ORDERED) -> float:
    """One wide-radix round: the digit histogram (a read of the keys, one shared
    add per key) and its two routing steps (high part over all keys, low byte
    inside each bucket), each an ordered round that reads and writes every item.
    The paper's count exchange (2prg) is the steps' look-back, not charged, as
    for radix 256."""
    return n * key_words * g + n * G + 2 * gpu_onesweep_round(n, words_per_item, g, G, shared)


def gpu_sort(n: float, key_bits: int, val_bits: int, r: int, g: float, G: float) -> float:
    """Model time of one whole sort of n keys at radix r (all rounds executed).
    Keys only at radix 256, the first round is the order-free one."""
    kw = key_bits / 32
    w = kw + val_bits / 32
    P = rounds(key_bits, r)
    shared = SHARED_ACCESSES_ORDERED + (SHARED_ACCESSES_PAYLOAD if val_bits else 0)
    if r == 256:
        t = gpu_histogram(n, kw, P, g, G)
        for j in range(P):
            first = j == 0 and val_bits == 0
            t += gpu_onesweep_round(n, w, g, G, SHARED_ACCESSES_FIRST if first else shared)
        return t
    # radix 65536: the buckets of every round (the digits' high bytes) come
    # from one byte-histogram read of the keys before round 0
    t = gpu_histogram(n, kw, key_bits // 8, g, G) if r == 65536 else 0.0
    return t + P * gpu_wide_round(n, w, kw, g, G, shared)


def calibrate(hbm_gbs: float, onesweep_round_s: float, n: float, words_per_item: float = 1.0,
              shared: float = SHARED_ACCESSES_ORDERED) -> dict:
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
