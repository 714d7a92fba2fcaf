"""Pins of the oracle's gradient-weighted initialisation (Sec. 4.4)."""
import math

import numpy as np
import pytest

from paper_2604_21984_gb300 import inputs as gen


def test_log32_accuracy(oracle):
    xs = np.exp(np.linspace(-80, 80, 300001)).astype(np.float32)
    xs = xs[xs > 1e-37]
    got = oracle.log32(xs).astype(np.float64)
    ref = np.log(xs.astype(np.float64))
    ulp = np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)
    assert np.max(np.abs(got - ref) / ulp) <= 2.0
    assert oracle.log32(np.float32(1.0)) == 0.0
    assert np.all(np.diff(oracle.log32(np.sort(xs))) >= 0)


def test_gradient_of_a_ramp_is_its_slope(oracle):
    H, W = 9, 13
    a = np.array([0.01, -0.02, 0.005])
    b = np.array([0.03, 0.0, -0.01])
    yy, xx = np.mgrid[0:H, 0:W]
    img = (0.5 + xx[..., None] * a + yy[..., None] * b).astype(np.float32)
    g = oracle.grad_magnitude_fp32(img).astype(np.float64)
    np.testing.assert_allclose(g, math.sqrt((a ** 2).sum() + (b ** 2).sum()), rtol=2e-5)
    flat = np.full((4, 5, 3), 0.3, np.float32)
    assert np.all(oracle.grad_magnitude_fp32(flat) == 0)


def test_init_weights(oracle):
    img = gen.image_noise_polygons_lines(48, 64, seed=5, n_polygons=4, n_lines=2)
    w = oracle.init_weights_fp32(img, 0.3).astype(np.float64)
    assert abs(w.sum() - 1.0) < 1e-4
    assert np.all(oracle.init_weights_fp32(img, 1.0) == np.float32(1.0 / (48 * 64)))
    g = oracle.grad_magnitude_fp32(img).ravel().astype(np.float64)
    np.testing.assert_allclose(oracle.init_weights_fp32(img, 0.0), g / g.sum(), rtol=1e-5, atol=1e-9)


def test_single_draw_probability_is_the_weight(oracle):
    """Efraimidis-Spirakis keys: with n = 1 the selected index has probability
    w_x exactly; Monte Carlo over seeds, chi-square."""
    w = np.array([0.05, 0.1, 0.15, 0.2, 0.5], np.float32)
    counts = np.zeros(5)
    trials = 20000
    for s in range(trials):
        counts[oracle.init_select(oracle.init_keys_fp32(w, s), 1)[0]] += 1
    expect = w.astype(np.float64) * trials
    chi2 = ((counts - expect) ** 2 / expect).sum()
    assert chi2 < 25                                    # 4 dof, p ~ 5e-5


def test_init_sites_invariants(oracle):
    H, W = 40, 56
    img = gen.image_noise_polygons_lines(H, W, seed=7, n_polygons=5, n_lines=3)
    n, cap = 300, 320
    p = oracle.init_sites(img, n, cap, 0.3, seed=11, log_tau0=6.5)
    x, y = p[0, :n], p[1, :n]
    col, row = np.floor(x).astype(int), np.floor(y).astype(int)
    assert np.all(np.abs(x - (col + 0.5)) <= 0.25) and np.all(np.abs(y - (row + 0.5)) <= 0.25)
    assert len(set((row * W + col).tolist())) == n                     # without replacement
    np.testing.assert_array_equal(p[4:7, :n].T, img[row, col])
    assert np.all(p[2, :n] == np.float32(6.5)) and np.all(p[3] == 0) and np.all(p[9:11] == 0)
    assert np.all(p[7] == 1) and np.all(p[8] == 0)
    assert np.all(p[0, n:] == -1) and np.all(p[1, n:] == -1)
    # more sites land where the gradient is large
    g = oracle.grad_magnitude_fp32(img)
    assert g[row, col].mean() > 1.5 * g.mean()
    # n = P selects every pixel once
    small = img[:6, :7]
    q = oracle.init_sites(small, 42, 42, 0.3, seed=1, log_tau0=5.0)
    assert sorted((np.floor(q[1]) * 7 + np.floor(q[0])).astype(int).tolist()) == list(range(42))
