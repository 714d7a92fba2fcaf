"""Target-BPP schedule simulator (Sec. 4.5): counts follow the event
schedule exactly, and the scale search lands on the target when it is
reachable."""
import math

from paper_2604_21984_gb300 import budget


def test_target_sites():
    assert budget.target_sites(4.0, 512, 768) == 12288      # 4 bits/px, 128 bits/site
    assert budget.target_sites(0.001, 4, 4) == 1


def test_simulation_replays_the_schedule():
    # hand-computed: 100 -> +10 -> 110 - 3 = 107 at t=10; 107 + 10 -> 117 - 3 = 114 at t=20
    trace, n = budget.simulate_counts(100, 25, 10, 10, 20, 0.1, 0.03, 1000)
    assert trace == [(10, 107), (20, 114)] and n == 114
    # capacity caps the densify step
    _, n = budget.simulate_counts(100, 10, 10, 10, 10, 0.5, 0.0, 120)
    assert n == 120
    # no events outside the window or without a frequency
    assert budget.simulate_counts(100, 50, 0, 0, 50, 0.5, 0.5, 1000)[1] == 100
    assert budget.simulate_counts(100, 9, 10, 10, 20, 0.5, 0.5, 1000)[1] == 100


def test_scale_search_hits_reachable_targets():
    n0, iters, every, start, end, cap = 32768, 2000, 200, 200, 1800, 65536
    for target, d, p in ((40000, 0.05, 0.01), (20000, 0.01, 0.033), (32768, 0.01, 0.033)):
        lam, n = budget.scale_for_target(n0, target, iters, every, start, end, d, p, cap)
        assert abs(n - target) <= 0.01 * target, (target, lam, n)
        assert budget.simulate_counts(n0, iters, every, start, end, d, p, cap, lam)[1] == n
    # target = n0 with a shrinking schedule: lam = 0 (no events) is exact
    lam, n = budget.scale_for_target(n0, n0, iters, every, start, end, 0.01, 0.033, cap)
    assert n == n0 and lam == 0.0
