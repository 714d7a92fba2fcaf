"""Site-budget schedule for a target bit rate (Sec. 4.5: "When a target BPP
is specified, we scale the base densify/prune percentiles with a schedule
simulator to match the expected final site count under the iteration
budget, via a 1D search over a shared scale factor").

Readings (the paper gives no more):
  * one site costs one packed 16-byte evaluation record (App. "Data Layout
    and Packing"), so a target of b bits per pixel means
    N* = round(b * H * W / 128) sites;
  * the simulator replays the encoder's event schedule: at every event
    t = every, 2 every, ... inside [start, end], first densify n += floor(lam
    d n) (capped by the capacity), then prune n -= floor(lam p n);
  * the shared scale factor lam multiplies both base percentiles, each
    scaled percentile capped at 0.95 (Sec. 6.1); lam is found by scanning
    [0, lam_max] and refining the best interval by ternary search on
    |n_final - N*| (n_final is piecewise constant and need not be monotone
    in lam).  With base percentiles that shrink the budget (densify < prune)
    targets above the initial count are out of reach and lam = 0 is
    returned (no events).
"""
from __future__ import annotations

import math


def target_sites(bpp: float, H: int, W: int) -> int:
    return max(1, int(round(bpp * H * W / 128.0)))


def simulate_counts(n0: int, iters: int, every: int, start: int, end: int, densify_pct: float,
                    prune_pct: float, capacity: int, lam: float = 1.0):
    """Active-site count after each densify-then-prune event; returns the
    list of (iteration, count) and the final count."""
    n = n0
    trace = []
    if every <= 0:
        return trace, n
    d, p = min(0.95, lam * densify_pct), min(0.95, lam * prune_pct)
    for t in range(1, iters + 1):
        if start <= t <= end and t % every == 0:
            n = min(capacity, n + int(math.floor(d * n)))
            n = max(0, n - int(math.floor(p * n)))
            trace.append((t, n))
    return trace, n


def scale_for_target(n0: int, target: int, iters: int, every: int, start: int, end: int,
                     densify_pct: float, prune_pct: float, capacity: int, lam_max: float = 20.0,
                     steps: int = 2001):
    """Shared percentile scale lam whose simulated final count is closest
    to `target` (ties: the smaller lam).  Returns (lam, final count)."""
    def err(lam):
        return abs(simulate_counts(n0, iters, every, start, end, densify_pct, prune_pct, capacity,
                                   lam)[1] - target)
    grid = [lam_max * i / (steps - 1) for i in range(steps)]
    errs = [err(l) for l in grid]
    k = min(range(steps), key=lambda i: (errs[i], i))
    lo = grid[max(0, k - 1)]
    hi = grid[min(steps - 1, k + 1)]
    best, best_e = grid[k], errs[k]
    for _ in range(40):                 # refine inside the neighbouring interval
        mid_l, mid_h = lo + (hi - lo) / 3, hi - (hi - lo) / 3
        el, eh = err(mid_l), err(mid_h)
        for l, e in ((mid_l, el), (mid_h, eh)):
            if e < best_e or (e == best_e and l < best):
                best, best_e = l, e
        if el <= eh:
            hi = mid_h
        else:
            lo = mid_l
    return best, simulate_counts(n0, iters, every, start, end, densify_pct, prune_pct, capacity,
                                 best)[1]
