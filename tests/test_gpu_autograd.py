"""torch.autograd wrapper of render/render_backward: gradients vs the oracle's
fp64 adjoint (small) and vs fp64 central finite differences on 64 random
sites of the 2048x2048, 262144-site, K=16 differentiation workload."""
import numpy as np
import pytest

from paper_2604_21984_gb300 import inputs as gen
from tests.gpu_util import dev, require_gpu

pytestmark = pytest.mark.gpu
INV = 0xFFFFFFFF


@pytest.fixture(scope="module")
def capi():
    return require_gpu()


def _autograd_grads(capi, p, ids, H, W, g):
    torch = pytest.importorskip("torch")
    from paper_2604_21984_gb300.autograd import sad_render_fn
    params = dev(p).requires_grad_(True)
    rgb = sad_render_fn(params, capi.map_from_ids(ids), H, W)
    (rgb * dev(g)).sum().backward()
    return rgb.detach().cpu().numpy(), params.grad.cpu().numpy().astype(np.float64)


def test_autograd_matches_oracle_adjoint(capi, oracle):
    H, W, K = 48, 40, 16
    p = gen.sites_random_spd(H, W, 300, seed=5)
    p[2] += 2.0
    ids = gen.knn_map(p, H, W, K, seed=6)
    g = gen.grad_image(H, W, seed=7)
    rgb, grads = _autograd_grads(capi, p, ids, H, W, g)
    assert np.abs(rgb.reshape(-1, 3) - oracle.render(p, H, W, ids)).max() <= 1e-5
    ref = oracle.render_backward(p, H, W, ids, g.reshape(-1, 3))
    from tests.gpu_util import assert_grads_close
    assert_grads_close(grads, ref)


def test_autograd_vs_finite_differences_config3(capi, oracle):
    H = W = 2048
    K = 16
    p = gen.sites_random_spd(H, W, 262144, seed=3000)
    ids = gen.knn_map(p, H, W, K, seed=3001)
    g = gen.grad_image(H, W, seed=3002) / (H * W)
    _, grads = _autograd_grads(capi, p, ids, H, W, g)
    rng = np.random.default_rng(17)
    sites = rng.choice(262144, 64, replace=False)
    p64 = p.astype(np.float64)
    g2 = g.reshape(-1, 3).astype(np.float64)
    fds = np.zeros((11, len(sites)))
    for si, s in enumerate(sites):
        rows = np.nonzero((ids == np.uint32(s)).any(axis=1))[0]
        r, c = np.divmod(rows, W)
        sub, gs = ids[rows], g2[rows]
        for j in range(11):
            # positions/radius in pixels: absolute step; others relative
            h = 1e-3 if j in (0, 1, 3) else 1e-4 * max(1.0, abs(p64[j, s]))

            def col_at(d):
                q = p64.copy()
                q[j, s] += d
                return oracle.render(q, H, W, sub, c + 0.5, r + 0.5)
            diff = (8 * (col_at(h) - col_at(-h)) - (col_at(2 * h) - col_at(-2 * h))) / (12 * h)
            fds[j, si] = (diff * gs).sum()
    got = grads[:, sites]
    # tolerance per parameter plane: norm-relative 1e-4 and elementwise
    # 1e-4 |fd| + 1e-4 max|fd| of the plane
    for j in range(11):
        scale = np.abs(fds[j]).max()
        err = np.abs(got[j] - fds[j])
        ratio = (err / (1e-4 * np.abs(fds[j]) + 1e-4 * scale + 1e-300)).max()
        nrel = np.linalg.norm(got[j] - fds[j]) / max(np.linalg.norm(fds[j]), 1e-300)
        print(f"plane {j:2d}: max err/tol {ratio:.3f}, norm-relative {nrel:.2e}")
        assert ratio <= 1.0 and nrel <= 1e-4, j


@pytest.mark.parametrize("worst_case_bytes", [8 << 30, 0])
def test_autograd_overflowing_map_gives_complete_gradients(capi, monkeypatch, worst_case_bytes):
    """A spatially incoherent map needs far more per-tile records than the
    default workspace holds.  With the worst-case workspace allowed, autograd
    allocates that one (no status read); with it forbidden, the backward must
    notice the overflow, grow the workspace and run again.  Either way the
    gradients equal those of a call whose workspace fits everything."""
    torch = pytest.importorskip("torch")
    from paper_2604_21984_gb300 import autograd
    monkeypatch.setattr(autograd, "WORST_CASE_BYTES", worst_case_bytes)
    monkeypatch.setattr(autograd, "_WS", autograd._Workspaces())
    H = W = 128
    K, n = 16, 20000
    p = gen.sites_random_spd(H, W, n, seed=31)
    ids = gen.random_map(H * W, K, n, seed=32, invalid_frac=0.05)
    g = gen.grad_image(H, W, seed=33)
    m = capi.map_from_ids(ids)
    pt = dev(p)
    prep = capi.empty_prep(n)
    capi.sad_prepare_sites(pt, H, W, prep)
    rgb = torch.empty((H, W, 3), dtype=torch.float32, device="cuda")
    fwd = torch.empty((2, H * W), dtype=torch.float32, device="cuda")
    capi.sad_render_save(prep, n, H, W, K, m, rgb, fwd)
    gd = dev(g)
    small = capi.backward_workspace(H, W, K, n)
    out = torch.empty((11, n), dtype=torch.float32, device="cuda")
    capi.sad_render_backward_saved(pt, prep, H, W, K, m, gd, rgb, fwd, out, small)
    st, used = capi.sad_workspace_status(small)
    assert st == capi.SAD_EWORKSPACE          # the default size really overflows
    big = capi.backward_workspace(H, W, K, n, max_records=used)
    ref = torch.empty_like(out)
    capi.sad_render_backward_saved(pt, prep, H, W, K, m, gd, rgb, fwd, ref, big)
    assert capi.sad_workspace_status(big)[0] == 0
    _, grads = _autograd_grads(capi, p, ids, H, W, g)
    assert np.array_equal(grads, ref.cpu().numpy().astype(np.float64))
    (_, n, exact), = autograd._WS._ws.values()
    assert exact == (worst_case_bytes > 0)
    assert n == (capi.sad_backward_max_records(H, W, K, p.shape[1]) if exact else used)
