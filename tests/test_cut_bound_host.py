"""The bound the fused training step relies on when it ends a pixel's list
early: with the list sorted by logit (descending), stopping at the first
entry whose exponential is below 1e-7 of the running sum leaves out at most
(K - 1) * 1e-7 of the kept sum, so the blend moves by at most that fraction
of the colour range.  Checked in float32, the step's own precision, on
random and adversarial lists."""
import numpy as np


def _cut(ell):
    """Entries kept by the rule, in list order (ell sorted descending)."""
    m = ell[0]
    z = np.float32(0.0)
    kept = []
    for k, lk in enumerate(ell):
        e = np.exp(np.float32(lk - m), dtype=np.float32)
        if e < np.float32(1e-7) * z:
            break
        kept.append(k)
        z = np.float32(z + e)
    return kept


def test_dropped_weight_is_bounded():
    rng = np.random.default_rng(0)
    K = 16
    worst = 0.0
    for trial in range(20000):
        scale = 10.0 ** rng.uniform(-1, 2.5)
        ell = np.sort(rng.normal(0, scale, K).astype(np.float32))[::-1]
        if trial % 4 == 0:   # adversarial: one leader, the rest tied just below the cut
            ell = np.concatenate([[0.0], np.full(K - 1, np.log(1e-7) - 1e-3)]).astype(np.float32)
        kept = _cut(ell)
        e = np.exp(ell.astype(np.float64) - ell[0])
        dropped = e.sum() - e[kept].sum()
        worst = max(worst, dropped / e[kept].sum())
        assert kept == list(range(len(kept)))            # a prefix of the list
        assert dropped <= (K - 1) * 1.0000001e-7 * e[kept].sum()
    assert worst > 1e-6       # the adversarial lists reach the bound's order


def test_blend_error_within_bound():
    """Colours in [0, 1]: the cut blend differs from the full blend by at
    most (K - 1) * 1e-7."""
    rng = np.random.default_rng(1)
    K = 16
    for _ in range(2000):
        ell = np.sort(rng.normal(0, 30, K))[::-1].astype(np.float32)
        col = rng.uniform(0, 1, (K, 3))
        kept = _cut(ell)
        e = np.exp(ell.astype(np.float64) - ell[0])
        full = (e[:, None] * col).sum(0) / e.sum()
        part = (e[kept, None] * col[kept]).sum(0) / e[kept].sum()
        assert np.abs(full - part).max() <= (K - 1) * 1.0000001e-7
