"""Pins of the adaptive-budget oracle (Sec. 4.5): statistics, selection,
split geometry and the densify/prune event."""
import math

import numpy as np
import pytest

from paper_2604_21984_gb300 import inputs as gen

INV = 0xFFFFFFFF


def _setup(H=20, W=24, n=40, K=6, seed=3):
    img = gen.image_noise_polygons_lines(H, W, seed=seed, n_polygons=3, n_lines=2)
    p = gen.sites_isotropic(img, n, seed=seed + 1, scale_px=2.0, tau=40.0, capacity=n + 10).astype(np.float64)
    ids = gen.knn_map(p.astype(np.float32), H, W, K, seed=seed + 2)
    return img, p, ids


def test_mass_and_energy_totals(oracle):
    img, p, ids = _setup()
    H, W = img.shape[:2]
    st = oracle.site_stats(p, H, W, ids, img)
    assert st[0].sum() == pytest.approx(H * W, rel=1e-12)               # weights sum to 1 per pixel
    L, _ = oracle.mse_loss_and_grad_rgb(oracle.render(p, H, W, ids), img)
    assert st[1].sum() == pytest.approx(L * H * W, rel=1e-12)           # sum of energies = total SSE


def test_moments_brute_force(oracle):
    img, p, ids = _setup(H=10, W=12, n=15, K=4, seed=9)
    H, W = img.shape[:2]
    st = oracle.site_stats(p, H, W, ids, img)
    c = oracle.render(p, H, W, ids)
    i = int(ids[37, 0])
    acc = np.zeros(5)
    for q in range(H * W):
        row, col = divmod(q, W)
        lst = [int(v) for v in ids[q]]
        if i not in lst:
            continue
        l = [(-math.exp(p[2, j]) * (math.hypot(col + 0.5 - p[0, j], row + 0.5 - p[1, j]) * math.exp(p[10, j] / 2)
              - p[3, j]) / max(H, W)) for j in lst]
        mx = max(l)
        w = math.exp(l[lst.index(i)] - mx) / sum(math.exp(v - mx) for v in l)
        om = w * ((c[q] - img.reshape(-1, 3)[q].astype(np.float64)) ** 2).sum()
        dx, dy = col + 0.5 - p[0, i], row + 0.5 - p[1, i]
        acc += om * np.array([dx, dy, dx * dx, dx * dy, dy * dy])
    np.testing.assert_allclose(st[2:7, i], acc, rtol=1e-9, atol=1e-15)


def test_selection_brute_force(oracle):
    rng = np.random.default_rng(4)
    n = 60
    p = np.zeros((11, n))
    p[0] = rng.uniform(0, 10, n)
    p[0, ::7] = -1                                                       # inactive
    st = np.zeros((8, n))
    st[0] = rng.uniform(0.5, 5, n)
    st[1] = rng.uniform(0, 1, n)
    st[7] = rng.uniform(-1, 1, n)
    st[7, 5] = st[7, 6]                                                  # a tie
    d, pr = oracle.densify_prune_select(p, st, 0.1, 0.2, alpha=0.7)
    act = [i for i in range(n) if p[0, i] >= 0]
    cand = [i for i in act if st[0, i] > 1]
    ranked = sorted(cand, key=lambda i: (-st[1, i] / max(st[0, i], 1e-8) ** 0.7, i))
    assert list(d) == sorted(ranked[:int(0.1 * len(act))])
    rest = [i for i in act if i not in d]
    assert list(pr) == sorted(sorted(rest, key=lambda i: (st[7, i], i))[:int(0.2 * len(act))])


def test_split_axis_follows_elongated_residual(oracle):
    """Residual spread along angle t around the site: the children sit on
    that line, symmetric about the centroid, with a = -log(l1/l2)/2 and
    u along the axis."""
    H = W = 64
    t = 0.7
    d = np.array([math.cos(t), math.sin(t)])
    p = np.zeros((11, 1))
    p[:, 0] = [30, 30, 5.0, 2.0, .5, .5, .5, 1, 0, 0.3, 0]
    tt = np.linspace(-6, 6, 25)
    off = 0.2 * (-1.0) ** np.arange(25)          # uncorrelated with tt: axis exactly d
    pts = np.outer(tt, d) + np.outer(off, [-d[1], d[0]])
    om = np.ones(len(pts))
    st = np.zeros((8, 1))
    st[0, 0] = 36.0
    st[1, 0] = om.sum()
    st[2, 0], st[3, 0] = pts[:, 0].sum(), pts[:, 1].sum()
    st[4, 0], st[5, 0], st[6, 0] = (pts[:, 0] ** 2).sum(), (pts[:, 0] * pts[:, 1]).sum(), (pts[:, 1] ** 2).sum()
    img = np.zeros((H, W, 3), np.float32)
    plus, minus = oracle.split_site(p, st, img, 0, H, W)
    mid = (plus[:2] + minus[:2]) / 2
    np.testing.assert_allclose(mid, p[:2, 0] + pts.mean(0), atol=1e-9)
    sep = plus[:2] - minus[:2]
    assert np.linalg.norm(sep) == pytest.approx(2 * min(max(0.5 * 6.0, 1.5), 48), rel=1e-9)
    assert abs(abs(sep @ d) / np.linalg.norm(sep) - 1) < 1e-6
    C = np.cov(pts.T, bias=True)
    l2, l1 = np.linalg.eigvalsh(C)
    assert plus[9] == pytest.approx(max(-2.0, -0.5 * math.log(l1 / l2)))
    assert abs(abs(plus[7] * d[0] + plus[8] * d[1]) - 1) < 1e-6
    assert plus[2] == pytest.approx(4.75) and plus[3] == pytest.approx(1.7)


def test_split_fallback_uses_sobel_gradient(oracle):
    H = W = 16
    img = np.zeros((H, W, 3), np.float32)
    img[:, 8:] = 1.0                                   # vertical edge: gradient along +x
    p = np.zeros((11, 1))
    p[:, 0] = [7.5, 8.2, 5.0, 2.0, .5, .5, .5, 0, 1, 1.0, 0]
    st = np.zeros((8, 1))
    st[0, 0] = 4.0                                     # energy 0 -> insufficient statistics
    plus, minus = oracle.split_site(p, st, img, 0, H, W)
    assert plus[1] == pytest.approx(8.2) and minus[1] == pytest.approx(8.2)
    assert plus[0] - minus[0] == pytest.approx(2 * 1.5)
    assert plus[9] == pytest.approx(0.8) and plus[7] == 0 and plus[8] == 1
    assert tuple(plus[4:7]) == (1.0, 1.0, 1.0) and tuple(minus[4:7]) == (0.0, 0.0, 0.0)


def test_densify_prune_event_counts(oracle):
    img, p, ids = _setup(n=40, seed=5)
    H, W = img.shape[:2]
    st = oracle.site_stats(p, H, W, ids, img)
    m = np.ones_like(p)
    v = np.ones_like(p)
    d, pr = oracle.densify_prune_select(p, st, 0.1, 0.05)
    q, m2, v2, n_act = oracle.densify_prune(p, m, v, st, img, H, W, 0.1, 0.05)
    free = np.nonzero(p[0] < 0)[0]
    ns = min(len(d), len(free))
    assert n_act == 40 + ns - len(pr)
    for k, i in enumerate(d[:ns]):
        j = free[k]
        assert np.all(m2[:, i] == 0) and np.all(m2[:, j] == 0) and np.all(v2[:, j] == 0)
        assert q[2, i] == pytest.approx(p[2, i] - 0.25) and q[2, j] == pytest.approx(p[2, i] - 0.25)
    assert np.all(q[0, pr] == -1) and np.all(q[1, pr] == -1)
