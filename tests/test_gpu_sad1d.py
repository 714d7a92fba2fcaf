"""1-D SAD on the GPU (Sec. "1D Signal Fitting") against the fp64 oracle:
render, the fused training step's gradients, loss and Adam update, batch
independence, ragged sample chunks and the wide-site path."""
import math

import numpy as np
import pytest

from paper_2604_21984_gb300 import inputs as gen
from tests.gpu_util import dev, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    return require_gpu()


def _batch(B, N, L, seed, jitter=True):
    y = gen.signals_1d(B, L, seed)
    p = gen.sites_1d(y, N).astype(np.float64).reshape(4, B, N)
    if jitter:   # move the sites off the uniform grid, vary tau and r
        g = np.random.default_rng(seed + 1)
        p[0] += g.uniform(-0.3, 0.3, p[0].shape) * (L / N)
        p[0] = np.clip(p[0], 0, L)
        p[2] += g.uniform(-0.5, 0.5, p[2].shape)
        p[3] = g.uniform(0.0, 2.0, p[3].shape)
    return y, p.reshape(4, B * N).astype(np.float32)


def _sig(p, B, N, b):
    return p.reshape(4, B, N)[:, b, :].astype(np.float64)


def _near_tie_ok(oracle, ps, L, K, k):
    """Sample k's K-th and (K+1)-th oracle logits are within float32 rounding."""
    ell = np.sort(oracle.sad1d_logits(ps, L)[k])[::-1]
    return K < len(ell) and abs(ell[K - 1] - ell[K]) < 1e-5 * max(1.0, abs(ell[K - 1]))


@pytest.mark.parametrize("N,L,K", [(64, 1024, 64), (64, 700, 8), (16, 1500, 4), (300, 400, 16), (1, 50, 1)])
def test_render_matches_oracle(capi, oracle, N, L, K):
    B = 5
    y, p = _batch(B, N, L, seed=N + L + K)
    got = capi.sad1d_render(dev(p), B, N, L, K).cpu().numpy()
    for b in range(B):
        ref = oracle.sad1d_render(_sig(p, B, N, b), L, K)
        err = np.abs(got[b] - ref)
        for k in np.nonzero(err > 1e-5)[0]:
            assert _near_tie_ok(oracle, _sig(p, B, N, b), L, K, k), (b, k, err[k])


@pytest.mark.parametrize("N,L,K", [(64, 1024, 64), (32, 1300, 8), (300, 257, 300)])
def test_train_step_matches_oracle(capi, oracle, N, L, K):
    """Gradients (norm-relative 1e-4 per plane, elementwise with a 1e-4 of max
    floor), the per-signal loss and one Adam step (t = 1)."""
    torch = pytest.importorskip("torch")
    B = 3
    y, p = _batch(B, N, L, seed=7 * N + L)
    pt = dev(p)
    m = torch.zeros_like(pt)
    v = torch.zeros_like(pt)
    loss = torch.empty(B, dtype=torch.float32, device="cuda")
    grads = torch.empty_like(pt)
    hp = capi.sad1d_hparams()
    capi.sad1d_train_step(pt, m, v, B, N, L, K, dev(y), loss, hp, 1, grads)
    got_g = grads.cpu().numpy().reshape(4, B, N)
    got_p = pt.cpu().numpy().reshape(4, B, N)
    for b in range(B):
        ps = _sig(p, B, N, b)
        p1, _, _, L_ref, g_ref = oracle.sad1d_train_step(ps, np.zeros_like(ps), np.zeros_like(ps), 1,
                                                          y[b].astype(np.float64), K)
        assert abs(loss[b].item() - L_ref) <= 1e-5 * max(L_ref, 1e-12)
        for j in range(4):
            r, gj = g_ref[j], got_g[j, b]
            scale = np.abs(r).max()
            assert np.all(np.abs(gj - r) <= 1e-4 * np.abs(r) + 1e-4 * scale), (b, j)
            assert np.linalg.norm(gj - r) <= 1e-4 * max(np.linalg.norm(r), 1e-30), (b, j)
        # Adam at t = 1 moves each parameter by about lr sign(g) (p, r scaled by
        # 1/s): compare where the gradient is not negligible
        s = 1.0 / L
        for j, lr in enumerate(oracle.SAD1D_LR.values()):
            unit = s if j in (0, 3) else 1.0
            ok = np.abs(g_ref[j]) > 1e-3 * np.abs(g_ref[j]).max()
            np.testing.assert_allclose(got_p[j, b][ok], p1[j][ok], rtol=1e-5, atol=1e-3 * lr / unit)


def test_signal_alone_equals_signal_in_a_batch(capi):
    """One block per signal: a signal's trajectory does not depend on the rest
    of the batch (bitwise, over several steps)."""
    torch = pytest.importorskip("torch")
    B, N, L, K = 6, 48, 900, 8
    y, p = _batch(B, N, L, seed=3)
    hp = capi.sad1d_hparams()

    def run(pp, yy, BB):
        pt = dev(pp)
        m = torch.zeros_like(pt)
        v = torch.zeros_like(pt)
        loss = torch.empty(BB, dtype=torch.float32, device="cuda")
        for t in range(1, 6):
            capi.sad1d_train_step(pt, m, v, BB, N, L, K, dev(yy), loss, hp, t)
        return pt.cpu().numpy().reshape(4, BB, N), loss.cpu().numpy()
    allp, alll = run(p, y, B)
    b = 4
    onep, onel = run(np.ascontiguousarray(p.reshape(4, B, N)[:, b:b + 1, :].reshape(4, N)), y[b:b + 1], 1)
    assert np.array_equal(allp[:, b, :], onep[:, 0, :]) and alll[b] == onel[0]


def test_training_fits_the_step_target(capi):
    """Training lowers the loss of step-plus-sine targets (the fused step
    follows the pinned adjoint)."""
    torch = pytest.importorskip("torch")
    B, N, L, K = 8, 64, 1024, 64
    y, p = _batch(B, N, L, seed=11, jitter=False)
    pt = dev(p)
    m = torch.zeros_like(pt)
    v = torch.zeros_like(pt)
    loss = torch.empty(B, dtype=torch.float32, device="cuda")
    hp = capi.sad1d_hparams()
    capi.sad1d_train_step(pt, m, v, B, N, L, K, dev(y), loss, hp, 1)
    first = loss.cpu().numpy().copy()
    for t in range(2, 301):
        capi.sad1d_train_step(pt, m, v, B, N, L, K, dev(y), loss, hp, t)
    last = loss.cpu().numpy()
    psnr = 10 * np.log10(1.0 / np.maximum(last, 1e-12))
    print("PSNR after 300 steps", np.round(psnr, 1))
    assert np.all(last < 0.5 * first) and np.median(psnr) > 30.0


def test_bad_arguments(capi):
    L_ = capi.lib()
    q = __import__("ctypes").c_void_p(256)
    assert L_.sad1d_render(q, 2, 64, 100, 20, q, None) == 1          # K < N must be <= 16
    assert L_.sad1d_render(q, 2, 2000, 100, 2000, q, None) == 1      # N above 1024
    assert L_.sad1d_render(q, 0, 64, 100, 64, q, None) == 1
    hp = capi.sad1d_hparams()
    assert L_.sad1d_train_step(q, q, q, 2, 8, 10, 8, q, q, __import__("ctypes").byref(hp), 0, None, None) == 1
