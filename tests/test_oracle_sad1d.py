"""Pins of the 1-D oracle (Sec. "1D Signal Fitting"): every function is held
to something other than itself -- partition of unity, the logistic two-site
closed form, the hard Apollonius partition of the line in the large-tau limit
(and plain nearest-site labels for zero radii), brute-force top-K, central
finite differences of the loss for all four parameter planes, and a
hand-computed Adam step."""
import math

import numpy as np
import pytest

from oracle import sad_oracle as o


def _sites(N, L, seed, tau=None):
    g = np.random.default_rng(seed)
    p = np.zeros((4, N))
    p[o.P1_P] = np.sort(g.uniform(0, L, N))
    p[o.P1_C] = g.uniform(-1, 1, N)
    p[o.P1_LOGTAU] = np.log(tau if tau is not None else g.uniform(2 * N, 8 * N, N))
    p[o.P1_R] = g.uniform(0, 3, N)
    return p


@pytest.mark.parametrize("K", [1, 3, 8, 64])
def test_weights_are_a_partition_of_unity(K):
    """A constant value c on every site renders c everywhere (the weights sum
    to one over each top-K set)."""
    p = _sites(64, 256, 1)
    p[o.P1_C] = 0.375
    assert np.abs(o.sad1d_render(p, 256, K) - 0.375).max() < 1e-12


def test_two_sites_blend_is_logistic():
    p = _sites(2, 100, 2)
    xs = np.linspace(0.5, 99.5, 37)
    ell = o.sad1d_logits(p, 100, xs)
    w1 = 1.0 / (1.0 + np.exp(-(ell[:, 0] - ell[:, 1])))
    ref = w1 * p[o.P1_C, 0] + (1 - w1) * p[o.P1_C, 1]
    assert np.abs(o.sad1d_render(p, 100, 2, xs) - ref).max() < 1e-12


def test_logit_is_the_normalised_additively_weighted_distance():
    """l = -tau (|x - p| - r) / L, written out for one site and a few points."""
    L = 40
    p = np.array([[12.0], [0.0], [math.log(7.0)], [1.5]])
    xs = np.array([0.5, 12.0, 12.5, 39.5])
    want = [-7.0 * (abs(x - 12.0) - 1.5) / L for x in xs]
    assert np.allclose(o.sad1d_logits(p, L, xs)[:, 0], want, rtol=0, atol=1e-15)


def test_large_tau_gives_the_apollonius_partition_of_the_line():
    """Sites at 10 (r = 2) and 20 (r = 0): the hard boundary is where
    |x - 10| - 2 = |x - 20|, i.e. x = 16, not the midpoint 15."""
    L = 32
    p = np.array([[10.0, 20.0], [1.0, 2.0], [math.log(1e5), math.log(1e5)], [2.0, 0.0]])
    xs = o.sad1d_samples(L)
    vals = o.sad1d_render(p, L, 2)
    left = xs < 16.0
    assert np.abs(vals[left] - 1.0).max() < 1e-9
    assert np.abs(vals[~left] - 2.0).max() < 1e-9


def test_zero_radii_equal_tau_gives_nearest_site_labels():
    L = 200
    p = _sites(17, L, 3, tau=1e6)
    p[o.P1_R] = 0.0
    p[o.P1_C] = np.arange(17, dtype=np.float64)
    xs = o.sad1d_samples(L)
    nearest = np.argmin(np.abs(xs[:, None] - p[o.P1_P][None, :]), axis=1)
    vals = o.sad1d_render(p, L, 1)
    assert np.array_equal(np.rint(vals).astype(int), nearest)
    assert np.array_equal(o.sad1d_topk(p, L, 1)[:, 0], nearest)


def test_topk_matches_a_sorted_brute_force():
    L = 64
    p = _sites(23, L, 4)
    p[o.P1_P, 5] = p[o.P1_P, 9]        # a tie: equal logits everywhere for 5 and 9
    p[o.P1_R, 5] = p[o.P1_R, 9]
    p[o.P1_LOGTAU, 5] = p[o.P1_LOGTAU, 9]
    ids = o.sad1d_topk(p, L, 6)
    ell = o.sad1d_logits(p, L)
    for k in range(L):
        order = sorted(range(23), key=lambda i: (-ell[k, i], i))[:6]
        assert list(ids[k]) == order


@pytest.mark.parametrize("K", [4, 16])
def test_adjoint_matches_finite_differences(K):
    """dL/dtheta of L = mean (c - y)^2 against 4th-order central differences,
    with sites placed so that no sample sits on a site and no top-K set
    changes under the step (checked)."""
    L = 96
    p = _sites(16, L, 5)
    p[o.P1_P] = np.arange(16) * 6.0 + 3.2       # off the sample centres
    y = np.sin(np.arange(L) / 7.0)
    vals = o.sad1d_render(p, L, K)
    _, g = o.sad1d_loss_and_grad(vals, y)
    grads = o.sad1d_backward(p, L, K, g)
    ids0 = np.sort(o.sad1d_topk(p, L, K), axis=1)

    def loss(q):
        assert np.array_equal(np.sort(o.sad1d_topk(q, L, K), axis=1), ids0)   # same sets
        return o.sad1d_loss_and_grad(o.sad1d_render(q, L, K), y)[0]
    for j in range(4):
        for i in range(16):
            h = 1e-4 * max(1.0, abs(p[j, i]))
            q = p.copy()
            f = []
            for d in (2, 1, -1, -2):
                q[j, i] = p[j, i] + d * h
                f.append(loss(q))
            fd = (8 * (f[1] - f[2]) - (f[0] - f[3])) / (12 * h)
            assert abs(grads[j, i] - fd) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(grads[j]).max()), (j, i)


def test_adjoint_position_gradient_is_zero_at_the_kink():
    """A sample exactly at a site's position contributes no position gradient
    (|x - p| has no derivative there); the other planes are unaffected."""
    L = 8
    p = np.array([[3.5, 6.0], [0.0, 1.0], [math.log(20.0)] * 2, [1.0, 0.0]])
    xs = np.array([3.5])
    g = np.array([1.0])
    out = o.sad1d_backward(p, L, 2, g, xs)
    assert out[o.P1_P, 0] == 0.0 and out[o.P1_P, 1] != 0.0
    assert out[o.P1_C, 0] > 0 and out[o.P1_LOGTAU, 0] != 0.0


def test_adam_first_step_by_hand():
    """Step 1: m = (1 - b1) g, v = (1 - b2) g^2, so the bias-corrected step is
    lr g / (|g| + eps) ~ lr sign(g); p and r move in normalised units."""
    L = 50
    p = np.array([[10.0], [0.5], [4.0], [1.0]])
    g = np.array([[0.02], [-0.3], [0.1], [0.004]])
    p1, m1, v1 = o.sad1d_adam_step(p, g, np.zeros_like(p), np.zeros_like(p), 1, L)
    s = 1.0 / L
    for j, name in enumerate(o.SAD1D_PLANES):
        unit = s if j in (o.P1_P, o.P1_R) else 1.0
        gj = g[j, 0] / unit
        assert math.isclose(m1[j, 0], 0.1 * gj, rel_tol=1e-12)
        assert math.isclose(v1[j, 0], 0.001 * gj * gj, rel_tol=1e-12)
        step = o.SAD1D_LR[name] * gj / (abs(gj) + 1e-8) / unit
        assert math.isclose(p1[j, 0], p[j, 0] - step, rel_tol=1e-12)


def test_adam_clamps():
    L = 20
    p = np.array([[0.01, 19.99], [5.0, -5.0], [2.0, 20.0], [0.0, 19.99]])
    g = np.array([[1.0, -1.0], [0.0, 0.0], [1.0, -1.0], [1.0, -1.0]])
    lr = {"p": 10.0, "c": 0.0, "log_tau": 10.0, "r": 10.0}
    p1, _, _ = o.sad1d_adam_step(p, g, np.zeros_like(p), np.zeros_like(p), 1, L, lr=lr)
    assert p1[o.P1_P, 0] == 0.0 and p1[o.P1_P, 1] == 20.0
    assert p1[o.P1_R, 0] == 0.0 and p1[o.P1_R, 1] == 20.0
    assert p1[o.P1_LOGTAU, 0] == 2.0 and p1[o.P1_LOGTAU, 1] == 20.0
    assert p1[o.P1_C, 0] == 5.0 and p1[o.P1_C, 1] == -5.0   # values are not clamped


def test_train_step_lowers_the_loss():
    """Repeated steps on a step-plus-sine target reduce the loss (the steps
    follow the adjoint, which the FD test pins)."""
    L, N = 256, 16
    xs = o.sad1d_samples(L)
    y = np.where(xs < 100, 0.2, 0.8) + 0.1 * np.sin(xs / 9.0)
    p = np.zeros((4, N))
    p[o.P1_P] = (np.arange(N) + 0.5) * L / N
    p[o.P1_C] = np.interp(p[o.P1_P], xs, y)
    p[o.P1_LOGTAU] = math.log(4.0 * N)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    losses = []
    for t in range(1, 61):
        p, m, v, loss, _ = o.sad1d_train_step(p, m, v, t, y, 8)
        losses.append(loss)
    assert losses[-1] < 0.5 * losses[0]
