"""Pins of the oracle's packed evaluation format (App. "Data Layout and
Packing", Packed storage for evaluation): hand-built words, quantisation
error bounds from the bit widths, exact endpoint round trips, inactive
sites, and the exactness of folding b into (log tau, r)."""
import math

import numpy as np
import pytest

from paper_2604_21984_gb300 import inputs as gen


def _sites(n=400, H=64, W=96, seed=3):
    p = gen.sites_random_spd(H, W, n, seed=seed)
    return p, H, W


def test_hand_built_words(oracle):
    o = oracle
    H, W = 50, 80
    p = np.zeros((11, 2), np.float32)
    p[o.PX] = [80.0, 0.0]
    p[o.PY] = [0.0, 50.0]
    p[o.PLOGTAU] = [1.0, 3.0]
    p[o.PR] = [2.0, -2.0]
    p[o.PCR:o.PCB + 1] = [[0.25, 1.0], [0.0, 0.5], [1.0, 0.0]]
    p[o.PUX] = [1.0, 0.0]
    p[o.PUY] = [0.0, 2.0]
    p[o.PA] = [1.0, -0.5]
    w, q = o.pack_eval(p, H, W)
    np.testing.assert_array_equal(q, np.float32([1, 3, -2, 2, 0.25, 1, 0, 0.5, 0, 1]))
    # site 0: x = W (code 32767), y = 0, active; colour r at its min (0), g at
    # its min, b at its max (1023); log tau min, r max; angle 0 -> code
    # round(0.5 * 65535) = 32768 (half to even); a = 1.0 -> float16 0x3C00
    assert w[0, 0] == 32767 | (1 << 31)
    assert w[0, 1] == 0 | (0 << 11) | (1023 << 22)
    assert w[0, 2] == 0 | (65535 << 16)
    assert w[0, 3] == 32768 | (0x3C00 << 16)
    # site 1: x = 0, y = H; colour r max, g max, b min; log tau max, r min;
    # u = (0, 2): angle pi/2 -> round(0.75 * 65535) = 49151; a = -0.5 -> 0xB800
    assert w[1, 0] == 0 | (32767 << 15) | (1 << 31)
    assert w[1, 1] == 2047 | (2047 << 11) | (0 << 22)
    assert w[1, 2] == 65535 | (0 << 16)
    assert w[1, 3] == 49151 | (0xB800 << 16)


def test_quantisation_error_bounds(oracle):
    o = oracle
    p, H, W = _sites()
    p[o.PB] = 0.0
    w, q = o.pack_eval(p, H, W)
    u = o.unpack_eval(w, q, H, W)
    tol32 = 1e-6
    assert np.abs(u[o.PX] - np.clip(p[o.PX], 0, W)).max() <= W / 32767 / 2 + tol32 * W
    assert np.abs(u[o.PY] - np.clip(p[o.PY], 0, H)).max() <= H / 32767 / 2 + tol32 * H
    for i, (plane, bits) in enumerate(((o.PLOGTAU, 16), (o.PR, 16), (o.PCR, 11), (o.PCG, 11), (o.PCB, 10))):
        lo, hi = q[2 * i], q[2 * i + 1]
        step = (hi - lo) / ((1 << bits) - 1)
        assert np.abs(u[plane] - p[plane]).max() <= step / 2 + tol32 * max(abs(lo), abs(hi), 1.0), plane
    th = np.arctan2(p[o.PUY], p[o.PUX])
    th2 = np.arctan2(u[o.PUY], u[o.PUX])
    d = np.abs(np.angle(np.exp(1j * (th - th2))))
    assert d.max() <= math.pi / 65535 + 1e-6
    assert np.allclose(np.hypot(u[o.PUX], u[o.PUY]), 1.0, atol=1e-6)
    assert np.all(np.abs(u[o.PA] - p[o.PA]) <= np.abs(p[o.PA]) * 2.0 ** -11 + 2.0 ** -24)
    assert np.all(u[o.PB] == 0)


def test_endpoints_round_trip_exactly(oracle):
    o = oracle
    p, H, W = _sites(seed=5)
    p[o.PB] = 0.0
    w, q = o.pack_eval(p, H, W)
    u = o.unpack_eval(w, q, H, W)
    for plane in (o.PLOGTAU, o.PR, o.PCR, o.PCG, o.PCB):
        for pick in (np.argmin, np.argmax):
            i = pick(p[plane])
            assert u[plane, i] == p[plane, i]


def test_inactive_sites(oracle):
    o = oracle
    p, H, W = _sites(seed=7)
    p = gen.deactivate_random(p, 0.3, seed=8)
    act = p[o.PX] >= 0
    # ranges cover the active sites only
    p[o.PCR, ~act] = 5.0
    w, q = o.pack_eval(p, H, W)
    assert np.all(w[~act] == 0)
    assert q[5] <= 1.0
    u = o.unpack_eval(w, q, H, W)
    assert np.all(u[o.PX, ~act] < 0) and np.all(u[o.PX, act] >= 0)


def test_folding_b_is_exact_for_the_logits(oracle):
    """tau s (r - e^{b/2} n0) = (tau e^{b/2}) s (r e^{-b/2} - n0)."""
    o = oracle
    p, H, W = _sites(n=50, seed=9)
    lt, rr = o._fold_b(p)
    f = p.astype(np.float64).copy()
    f[o.PLOGTAU] = lt
    f[o.PR] = rr
    f[o.PB] = 0.0
    g = np.random.default_rng(0)
    pts_x, pts_y = g.uniform(0, W, 200), g.uniform(0, H, 200)
    ids = np.tile(np.arange(50, dtype=np.uint32), (200, 1))
    a = o.logits(p.astype(np.float64), H, W, ids, pts_x, pts_y)
    b = o.logits(f, H, W, ids, pts_x, pts_y)
    # folded values are rounded to float32: relative 1e-6
    np.testing.assert_allclose(a, b, rtol=2e-6, atol=2e-5)
