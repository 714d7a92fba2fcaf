"""Pins of the oracle adjoint (App. "Gradient Computation and Reduction", Per-pixel gradients) and removal
delta (Sec. 4.5) against central finite differences and brute force.  CPU."""
import math

import numpy as np
import pytest

from paper_2604_21984_gb300 import inputs as gen

INV = 0xFFFFFFFF


def _setup(seed, H=10, W=12, n=14, K=5):
    p = gen.sites_random_spd(H, W, n, seed=seed).astype(np.float64)
    # make the blend sharper than the workload default so every term matters
    p[2] += 2.5
    # break exact pixel-centre hits (gradient undefined there)
    p[0] += 0.123
    p[1] += 0.071
    # unnormalised directions exercise the (ux, uy) -> theta mapping
    p[7] *= 1.7
    p[8] *= 1.7
    ids = gen.knn_map(p.astype(np.float32), H, W, K, seed=seed + 1, shuffle=True,
                      truncate_frac=0.2)
    g = gen.grad_image(H, W, seed=seed + 2).reshape(-1, 3).astype(np.float64)
    return p, ids, g, H, W


def _loss(oracle, p, H, W, ids, g):
    return float((oracle.render(p, H, W, ids) * g).sum())


def _fd(oracle, p, H, W, ids, g, i, j, h):
    """Fourth-order central difference of L = sum_x g(x) . c(x) in p[j, i],
    accumulated as per-pixel colour differences to limit cancellation."""
    def c_at(d):
        q = p.copy()
        q[j, i] += d
        return oracle.render(q, H, W, ids)
    diff = (8.0 * (c_at(h) - c_at(-h)) - (c_at(2 * h) - c_at(-2 * h))) / (12.0 * h)
    return float((diff * g).sum())


@pytest.mark.parametrize("seed", [31, 32])
def test_adjoint_matches_central_differences(oracle, seed):
    p, ids, g, H, W = _setup(seed)
    grads = oracle.render_backward(p, H, W, ids, g)
    used = np.unique(ids[ids != INV]).astype(np.int64)
    rng = np.random.default_rng(seed)
    floor = 1e-7 * np.abs(grads).max(axis=1)
    for i in rng.choice(used, size=min(6, len(used)), replace=False):
        for j in range(11):
            h = 1e-4 * max(1.0, abs(p[j, i]))
            fd = _fd(oracle, p, H, W, ids, g, i, j, h)
            an = grads[j, i]
            assert abs(fd - an) <= 1e-7 * abs(fd) + floor[j], (i, j, fd, an)


def test_unlisted_sites_get_zero_gradient(oracle):
    p, ids, g, H, W = _setup(40)
    grads = oracle.render_backward(p, H, W, ids, g)
    listed = np.zeros(p.shape[1], bool)
    listed[np.unique(ids[ids != INV]).astype(np.int64)] = True
    assert np.all(grads[:, ~listed] == 0)


def test_rotation_gradient_matches_theta_derivative(oracle):
    """dL/dtheta = -uy dL/dux + ux dL/duy for unit u; check against a finite
    difference in the angle itself (rotating u), independent of the raw map."""
    p, ids, g, H, W = _setup(41)
    p[7], p[8] = np.cos(np.arctan2(p[8], p[7])), np.sin(np.arctan2(p[8], p[7]))
    grads = oracle.render_backward(p, H, W, ids, g)
    dth = -p[8] * grads[7] + p[7] * grads[8]
    i = int(np.argmax(np.abs(dth)))                   # the most rotation-sensitive site
    th = math.atan2(p[8, i], p[7, i])
    h = 1e-4

    def c_at(d):
        q = p.copy()
        q[7, i], q[8, i] = math.cos(th + d), math.sin(th + d)
        return oracle.render(q, H, W, ids)
    fd = float(((8 * (c_at(h) - c_at(-h)) - (c_at(2 * h) - c_at(-2 * h))) / (12 * h) * g).sum())
    assert dth[i] == pytest.approx(fd, rel=1e-7)


@pytest.mark.parametrize("sharp", [2.0, 14.0])
def test_removal_delta_matches_brute_force(oracle, sharp):
    """Delete site k from each list, renormalise, recompute the loss (Sec. 4.5).
    The sharp case makes 1 - w of the dominant site underflow in fp64."""
    H, W = 8, 9
    p = gen.sites_random_spd(H, W, 12, seed=50).astype(np.float64)
    p[2] += sharp
    ids = gen.knn_map(p.astype(np.float32), H, W, 4, seed=51)
    img = gen.image_sinusoid_polygons(H, W, seed=52).reshape(-1, 3).astype(np.float64)
    ids[3, 1:] = INV                                  # a single-site pixel
    rd = oracle.removal_delta(p, H, W, ids, img)
    base = ((oracle.render(p, H, W, ids) - img) ** 2).sum(1)
    expect = np.zeros(p.shape[1])
    for k in range(ids.shape[1]):
        cut = ids.copy()
        cut[:, k] = INV
        after = ((oracle.render(p, H, W, cut) - img) ** 2).sum(1)
        has = ids[:, k] != INV
        np.add.at(expect, ids[has, k].astype(np.int64), (after - base)[has])
    np.testing.assert_allclose(rd, expect, atol=1e-12)


def test_mse_gradient_is_loss_derivative(oracle):
    g = np.random.default_rng(3)
    c = g.random((20, 3))
    t = g.random((20, 3))
    L, dc = oracle.mse_loss_and_grad_rgb(c, t)
    assert L == pytest.approx(((c - t) ** 2).sum() / 20)
    h = 1e-7
    c2 = c.copy()
    c2[4, 1] += h
    L2, _ = oracle.mse_loss_and_grad_rgb(c2, t)
    assert (L2 - L) / h == pytest.approx(dc[4, 1], rel=1e-5)
