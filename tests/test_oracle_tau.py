"""Pins of the oracle's tau diffusion (App. "Tau Diffusion")."""
import numpy as np

from paper_2604_21984_gb300 import inputs as gen


def _setup(seed=1):
    H, W, K = 20, 30, 8
    p = gen.sites_random_spd(H, W, 60, seed=seed)
    p = gen.deactivate_random(p, 0.2, seed=seed + 1)
    ids = gen.knn_map(p, H, W, K, seed=seed + 2)
    g = np.random.default_rng(seed).normal(size=60)
    return p, H, W, ids, g


def test_lambda_zero_and_constant_gradients(oracle):
    p, H, W, ids, g = _setup()
    np.testing.assert_array_equal(oracle.tau_diffusion(p, H, W, ids, 0.0, g), g)
    c = np.full(60, 2.5)
    np.testing.assert_allclose(oracle.tau_diffusion(p, H, W, ids, 0.7, c), c, rtol=0, atol=1e-15)


def test_lambda_one_is_the_neighbour_mean(oracle):
    p, H, W, ids, g = _setup(seed=5)
    out = oracle.tau_diffusion(p, H, W, ids, 1.0, g)
    for i in range(60):
        if p[0, i] < 0:
            assert out[i] == g[i]
            continue
        col = min(max(int(np.floor(p[0, i])), 0), W - 1)
        row = min(max(int(np.floor(p[1, i])), 0), H - 1)
        nb = sorted({int(j) for j in ids[row * W + col] if j != oracle.INVALID and j != i and p[0, j] >= 0})
        if nb:
            assert abs(out[i] - sum(g[j] for j in nb) / len(nb)) < 1e-12
        else:
            assert out[i] == g[i]


def test_mixing_is_affine_in_lambda(oracle):
    p, H, W, ids, g = _setup(seed=9)
    a = oracle.tau_diffusion(p, H, W, ids, 0.0, g)
    b = oracle.tau_diffusion(p, H, W, ids, 1.0, g)
    m = oracle.tau_diffusion(p, H, W, ids, 0.3, g)
    np.testing.assert_allclose(m, 0.7 * a + 0.3 * b, rtol=0, atol=1e-12)
