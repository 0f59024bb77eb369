"""Host-side logic of the serving loop (no GPU): the arena allocator."""
import random

import pytest

torch = pytest.importorskip("torch")

from paper_1808_10292_gb300.serve import Arena


def test_arena_first_fit_and_coalescing():
    a = Arena(1 << 16, device="cpu")
    x = a.alloc(1000)
    y = a.alloc(5000)
    z = a.alloc(300)
    assert x == (0, 1024) and y == (1024, 5120) and z == (6144, 512)
    assert a.alloc(1 << 16) is None  # over budget: refused
    a.release(*y)
    assert a.alloc(5000) == (1024, 5120)  # first fit reuses the hole
    a.release(1024, 5120)
    a.release(*x)
    a.release(*z)
    assert a.free == [(0, 1 << 16)] and a.used == 0  # fully coalesced


def test_arena_random_workload_never_overlaps():
    rng = random.Random(5)
    a = Arena(1 << 20, device="cpu")
    live = []
    for _ in range(5000):
        if live and rng.random() < 0.45:
            a.release(*live.pop(rng.randrange(len(live))))
        else:
            r = a.alloc(rng.randint(1, 40_000))
            if r is not None:
                live.append(r)
        spans = sorted(live + a.free)
        for (o1, s1), (o2, _) in zip(spans, spans[1:]):
            assert o1 + s1 <= o2  # live blocks and holes never overlap
        assert a.used == sum(s for _, s in live)
    for r in live:
        a.release(*r)
    assert a.free == [(0, 1 << 20)]
