"""Host logic of the serving layer: the range allocator of the site and
pixel pools (checked against a brute-force occupancy array)."""
import random

import pytest

serve = pytest.importorskip("paper_2604_21984_gb300.serve")


def test_range_pool_first_fit_and_coalescing():
    p = serve.RangePool(100)
    a = p.alloc(30)
    b = p.alloc(30)
    c = p.alloc(30)
    assert (a, b, c) == (0, 30, 60)
    assert p.alloc(11) is None
    p.release(b, 30)
    assert p.alloc(31) is None
    assert p.alloc(30) == 30
    p.release(a, 30)
    p.release(30, 30)
    p.release(c, 30)
    assert p.free == [(0, 100)]
    with pytest.raises(ValueError):
        p.release(0, 10)


def test_range_pool_random_against_bitmap():
    rng = random.Random(7)
    cap = 1000
    p = serve.RangePool(cap, align=4)
    used = [False] * cap
    live = []
    for _ in range(3000):
        if live and rng.random() < 0.45:
            o, n = live.pop(rng.randrange(len(live)))
            p.release(o, n)
            nn = -(-n // 4) * 4
            for i in range(o, o + nn):
                assert used[i]
                used[i] = False
        else:
            n = rng.randint(1, 120)
            o = p.alloc(n)
            nn = -(-n // 4) * 4
            # first fit: no earlier free run of length nn
            run, first = 0, None
            for i in range(cap):
                run = run + 1 if not used[i] else 0
                if run == nn:
                    first = i - nn + 1
                    break
            assert o == first
            if o is not None:
                assert o % 4 == 0
                for i in range(o, o + nn):
                    assert not used[i]
                    used[i] = True
                live.append((o, n))
        assert p.free_total() == used.count(False)
        # free list sorted, disjoint and coalesced
        for (o1, l1), (o2, _) in zip(p.free, p.free[1:]):
            assert o1 + l1 < o2


def test_pool_bytes_counts_every_array():
    # params, m, v (3 x 11 floats), prepared table (48 B), accumulators (80 B)
    # per site; target (12 B) and two K-entry maps per pixel
    assert serve.pool_bytes(1, 0, 16) == 132 + 48 + 80
    assert serve.pool_bytes(0, 1, 16) == 12 + 128
    assert serve.pool_bytes(0, 1, 8) == 12 + 64
