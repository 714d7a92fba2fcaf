"""Pins of the oracle Adam step (Sec. 6.1) against hand-computed values."""
import math

import numpy as np
import pytest


def _one_site(x=10.0, y=5.0, log_tau=3.0, r=2.0, a=0.5):
    p = np.zeros((11, 1))
    p[:, 0] = [x, y, log_tau, r, 0.5, 0.5, 0.5, 1.0, 0.0, a, 0.0]
    return p


def test_first_step_moves_by_learning_rate(oracle):
    H, W = 40, 80                                   # s = 1/80
    p = _one_site()
    g = np.zeros_like(p)
    g[0, 0] = 3e-4                                  # dL/dx > 0 -> x decreases
    g[2, 0] = -2.0                                  # dL/dlog_tau < 0 -> increases
    g[4, 0] = 1e-3
    z = np.zeros_like(p)
    q, m, v = oracle.adam_step(p, g, z, z, 1, H, W)
    # bias-corrected first step = lr * g / (|g| + eps); x steps in units of 1/s
    gx = 3e-4 * 80
    assert q[0, 0] == pytest.approx(10.0 - 1e-3 * 80 * gx / (gx + 1e-8), rel=1e-12)
    assert q[2, 0] == pytest.approx(3.0 + 1e-2 * 2.0 / (2.0 + 1e-8), rel=1e-12)
    assert q[4, 0] == pytest.approx(0.5 - 5e-3 * 1e-3 / (1e-3 + 1e-8), rel=1e-12)
    assert q[1, 0] == 5.0                           # zero gradient: no motion
    assert m[0, 0] == pytest.approx(0.1 * 3e-4 * 80)
    assert v[0, 0] == pytest.approx(0.001 * (3e-4 * 80) ** 2)


def test_second_step_hand_computed(oracle):
    H, W = 64, 64
    p = _one_site(log_tau=5.0)
    z = np.zeros_like(p)
    g1 = np.zeros_like(p); g1[2, 0] = 1.0
    g2 = np.zeros_like(p); g2[2, 0] = -3.0
    p1, m1, v1 = oracle.adam_step(p, g1, z, z, 1, H, W)
    p2, m2, v2 = oracle.adam_step(p1, g2, m1, v1, 2, H, W)
    m_ = 0.9 * 0.1 * 1.0 + 0.1 * -3.0               # -0.21
    v_ = 0.999 * 0.001 * 1.0 + 0.001 * 9.0          # 0.009999
    mhat = m_ / (1 - 0.81)
    vhat = v_ / (1 - 0.999 ** 2)
    expect = (5.0 - 1e-2 / (1.0 + 1e-8)) - 1e-2 * mhat / (math.sqrt(vhat) + 1e-8)
    assert p2[2, 0] == pytest.approx(expect, rel=1e-12)


def test_clamps_and_direction_renormalised(oracle):
    H, W = 32, 32
    p = _one_site(x=0.001, log_tau=2.0, r=1.0, a=1.999)
    p[7, 0], p[8, 0] = 3.0, 4.0                     # unnormalised direction
    g = np.zeros_like(p)
    g[0, 0] = 1.0                                   # pushes x below 0
    g[2, 0] = 1.0                                   # pushes log_tau below 2
    g[3, 0] = 1.0                                   # pushes r below 1
    g[9, 0] = -1.0                                  # pushes a above 2
    g[4, 0] = -1.0                                  # colour towards > 1 (0.5 + 5e-3 ok)
    z = np.zeros_like(p)
    q, _, _ = oracle.adam_step(p, g, z, z, 1, H, W)
    assert q[0, 0] == 0.0 and q[2, 0] == 2.0 and q[3, 0] == 1.0 and q[9, 0] == 2.0
    assert q[7, 0] == pytest.approx(0.6) and q[8, 0] == pytest.approx(0.8)


def test_inactive_sites_untouched(oracle):
    p = _one_site()
    p[0, 0], p[1, 0] = -1.0, -1.0
    g = np.ones_like(p)
    z = np.zeros_like(p)
    q, m, v = oracle.adam_step(p, g, z, z, 1, 16, 16)
    assert np.array_equal(q, p) and not m.any() and not v.any()
