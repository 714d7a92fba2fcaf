"""Pins of the oracle's fp64 definitions against closed forms and textbook
geometry (Sec. 3 "Preliminaries", Sec. 4.1-4.2).  CPU only."""
import math

import numpy as np
import pytest
from scipy.spatial import cKDTree

from paper_2604_21984_gb300 import inputs as gen

INV = 0xFFFFFFFF


def _sites(xy, log_tau=0.0, r=0.0, a=0.0, b=0.0, theta=0.0, colours=None):
    xy = np.asarray(xy, dtype=np.float64)
    n = len(xy)
    p = np.zeros((11, n))
    p[0], p[1] = xy[:, 0], xy[:, 1]
    p[2] = log_tau
    p[3] = r
    if colours is None:
        colours = np.eye(3)[np.arange(n) % 3]
    p[4:7] = np.asarray(colours, dtype=np.float64).T
    p[7], p[8] = math.cos(theta), math.sin(theta)
    p[9], p[10] = a, b
    return p


def test_metric_closed_form(oracle):
    g = np.random.default_rng(1)
    n = 50
    p = np.zeros((11, n))
    th = g.uniform(0, 2 * np.pi, n)
    raw = g.uniform(0.2, 3.0, n)
    p[7], p[8] = raw * np.cos(th), raw * np.sin(th)      # unnormalised direction
    p[9] = g.uniform(-2, 2, n)
    p[10] = g.uniform(-3, 3, n)
    G00, G01, G11 = oracle.metric(p)
    det = G00 * G11 - G01 ** 2
    np.testing.assert_allclose(det, np.exp(2 * p[10]), rtol=1e-12)   # det = 1 when b = 0
    u = np.stack([np.cos(th), np.sin(th)])
    v = np.stack([-np.sin(th), np.cos(th)])
    Gu = np.stack([G00 * u[0] + G01 * u[1], G01 * u[0] + G11 * u[1]])
    Gv = np.stack([G00 * v[0] + G01 * v[1], G01 * v[0] + G11 * v[1]])
    np.testing.assert_allclose(Gu, np.exp(p[10] + p[9]) * u, atol=1e-12, rtol=1e-12)
    np.testing.assert_allclose(Gv, np.exp(p[10] - p[9]) * v, atol=1e-12, rtol=1e-12)


def test_weights_sum_to_one_and_empty_lists(oracle):
    img = gen.image_sinusoid_polygons(16, 16, seed=3)
    p = gen.sites_random_spd(16, 16, 40, seed=4, capacity=48)
    ids = gen.knn_map(p, 16, 16, 8, seed=5, truncate_frac=0.3, shuffle=True,
                      include_inactive_frac=0.2)
    ids[7, :] = INV                                    # an empty list
    w, _, valid, _ = oracle.weights(p, 16, 16, ids)
    sums = w.sum(1)
    has = valid.any(1)
    np.testing.assert_allclose(sums[has], 1.0, atol=1e-12)
    assert np.all(sums[~has] == 0)
    assert np.all(w[~valid] == 0)
    c = oracle.render(p, 16, 16, ids)
    assert np.all(c[7] == 0)
    del img


def test_nearer_site_gets_larger_weight(oracle):
    # two isotropic sites, equal tau and radius: the nearer one dominates
    p = _sites([[2.0, 2.0], [10.0, 2.0]], log_tau=math.log(50.0))
    ids = np.array([[0, 1]] * 3, dtype=np.uint32)
    px = np.array([3.0, 6.0, 9.0])
    py = np.array([2.0, 2.0, 2.0])
    w, _, _, _ = oracle.weights(p, 16, 16, ids, px, py)
    assert w[0, 0] > 0.5 > w[2, 0]
    assert abs(w[1, 0] - 0.5) < 1e-12                  # equidistant


def test_permutation_invariance_and_k_equals_n(oracle):
    p = gen.sites_random_spd(12, 10, 9, seed=11)
    full = np.tile(np.arange(9, dtype=np.uint32), (120, 1))
    g = np.random.default_rng(0)
    shuf = np.array([g.permutation(row) for row in full])
    np.testing.assert_allclose(oracle.render(p, 10, 12, full), oracle.render(p, 10, 12, shuf), atol=1e-14)
    # exact top-K with K = N lists every active site
    ex, _ = oracle.exact_topk(p, 10, 12, 9)
    assert all(sorted(row.tolist()) == list(range(9)) for row in ex)


def test_hard_limit_is_ordinary_voronoi(oracle):
    """K=1 (any tau), a=b=0, r=0: label = Euclidean nearest site (Eq. Voronoi cell)."""
    H, W = 40, 56
    g = np.random.default_rng(7)
    xy = g.uniform(0, [W, H], (30, 2))
    p = _sites(xy)
    lab, _ = oracle.exact_topk(p, H, W, 1)
    row, col = np.divmod(np.arange(H * W), W)
    _, nn = cKDTree(xy).query(np.stack([col + 0.5, row + 0.5], 1))
    assert np.array_equal(lab[:, 0].astype(np.int64), nn)


def test_square_lattice_gives_square_cells(oracle):
    H = W = 32
    cell = 8
    cy, cx = np.mgrid[0:H // cell, 0:W // cell]
    xy = np.stack([(cx.ravel() + 0.5) * cell, (cy.ravel() + 0.5) * cell], 1)
    # sub-pixel offset breaks exact ties on the cell borders
    xy = xy + 0.01
    p = _sites(xy)
    lab, _ = oracle.exact_topk(p, H, W, 1)
    row, col = np.divmod(np.arange(H * W), W)
    expect = (row // cell) * (W // cell) + col // cell
    assert np.array_equal(lab[:, 0].astype(np.int64), expect)


def test_anisotropic_hard_partition_is_nearest_in_warped_space(oracle):
    """All sites share one metric G: |x-p|_G = |L(x-p)| with L = G^(1/2), so the
    K=1 partition is the Euclidean Voronoi diagram of the warped points (Sec. 3,
    anisotropic norm).  Catches a transposed or sign-flipped metric."""
    H, W = 48, 48
    g = np.random.default_rng(9)
    xy = g.uniform(0, W, (25, 2))
    a, b, th = 1.3, 0.4, 0.6
    p = _sites(xy, a=a, b=b, theta=th)
    R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    L = R @ np.diag([math.exp((b + a) / 2), math.exp((b - a) / 2)]) @ R.T   # G^(1/2)
    row, col = np.divmod(np.arange(H * W), W)
    q = np.stack([col + 0.5, row + 0.5], 1)
    _, nn = cKDTree(xy @ L.T).query(q @ L.T)
    lab, _ = oracle.exact_topk(p, H, W, 1)
    assert np.array_equal(lab[:, 0].astype(np.int64), nn)


def test_apollonius_boundary_is_hyperbola_branch(oracle):
    """Two isotropic sites with radii r1 > r2, equal tau, K=1: the boundary of
    the additively weighted cells is the branch |x-p1| - |x-p2| = r1 - r2 of the
    hyperbola with foci p1, p2 (Sec. 3, Apollonius diagram).  Points built
    from the hyperbola's parametric form must flip label across the branch."""
    c, A = 6.0, 2.0                    # half focal distance, semi-major axis
    Bh = math.sqrt(c * c - A * A)
    centre = np.array([30.0, 30.0])
    p1, p2 = centre + [-c, 0.0], centre + [c, 0.0]
    r1, r2 = 3.0, 3.0 - 2 * A          # r1 - r2 = 2A
    p = np.zeros((11, 2))
    p[0], p[1] = [p1[0], p2[0]], [p1[1], p2[1]]
    p[3] = [r1, r2]
    p[4:7] = np.eye(3)[:, :2]
    p[7] = 1.0
    # branch closer to p2 (d1 - d2 = 2A > 0): x = +A cosh t, y = B sinh t
    t = np.linspace(-1.5, 1.5, 25)
    on = np.stack([A * np.cosh(t), Bh * np.sinh(t)], 1) + centre
    outward = np.stack([np.cosh(t) / A, -np.sinh(t) / Bh], 1)   # gradient of x^2/A^2 - y^2/B^2
    outward /= np.linalg.norm(outward, axis=1, keepdims=True)
    eps = 1e-3
    for sign, expect in ((+1, 1), (-1, 0)):     # beyond the branch: site 2 (nearer p2) wins
        q = on + sign * eps * outward
        ids = np.array([[0, 1]] * len(q), dtype=np.uint32)
        _, ell, _, _ = oracle.weights(p, 64, 64, ids, q[:, 0], q[:, 1])
        assert np.all(np.argmax(ell, axis=1) == expect)


def test_large_tau_limit_matches_k1(oracle):
    """Uniform, very large tau (per-pixel slope >> 1): the K=8 soft render equals
    the colour of the hard K=1 cell away from cell boundaries."""
    H = W = 32
    p = gen.sites_random_spd(H, W, 60, seed=21)
    p = p.astype(np.float64)
    p[2] = math.log(1e4 * max(H, W))
    top8, ell8 = oracle.exact_topk(p, H, W, 8)
    soft = oracle.render(p, H, W, top8)
    hard = np.stack([p[4:7][:, i] for i in top8[:, 0].astype(np.int64)])
    margin = ell8[:, 0] - ell8[:, 1]
    far = margin > 30.0
    assert far.mean() > 0.5
    np.testing.assert_allclose(soft[far], hard[far], atol=1e-10)


def test_two_site_colour_derivative_closed_form(oracle):
    """1 pixel, 2 sites: c = w1 c1 + w2 c2 with w1 = sigma(l1 - l2), so
    dc/dr1 = w1 w2 tau1 s (c1 - c2) and dc/dlog_tau1 = w1 w2 l1 (c1 - c2)."""
    H = W = 20
    s = 1.0 / 20
    p = _sites([[4.3, 5.1], [7.9, 6.2]], log_tau=[math.log(30.0), math.log(12.0)],
               r=[0.7, -0.4], a=[0.3, -0.5], b=[0.2, 0.1], theta=0.4,
               colours=[[0.9, 0.1, 0.2], [0.2, 0.6, 0.8]])
    ids = np.array([[0, 1]], dtype=np.uint32)
    px, py = np.array([5.5]), np.array([6.5])
    w, ell, _, _ = oracle.weights(p, H, W, ids, px, py)
    g = np.array([[0.3, -1.1, 0.7]])
    grads = oracle.render_backward(p, H, W, ids, g, px, py)
    c1, c2 = p[4:7, 0], p[4:7, 1]
    w1, w2 = w[0]
    tau1 = 30.0
    assert grads[3, 0] == pytest.approx(w1 * w2 * tau1 * s * float(g[0] @ (c1 - c2)), rel=1e-12)
    assert grads[2, 0] == pytest.approx(w1 * w2 * ell[0, 0] * float(g[0] @ (c1 - c2)), rel=1e-12)
    np.testing.assert_allclose(grads[4:7, 0], w1 * g[0], rtol=1e-12)
