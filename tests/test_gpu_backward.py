"""GPU adjoint (App. "Gradient Computation and Reduction") vs the oracle's fp64 adjoint: gradients within 1e-4
norm-relative per parameter plane (floor 1e-4 max|grad|); bitwise determinism;
the fused MSE training gradient and loss."""
import numpy as np
import pytest

from paper_2604_21984_gb300 import inputs as gen
from tests.gpu_util import assert_grads_close, dev, prepare, require_gpu

pytestmark = pytest.mark.gpu
INV = 0xFFFFFFFF


@pytest.fixture(scope="module")
def capi():
    return require_gpu()


def _backward(capi, p, H, W, ids, g, max_records=0, saved=False):
    """The adjoint by sad_render_backward, or (saved) by sad_render_save then
    sad_render_backward_saved."""
    torch = pytest.importorskip("torch")
    K = ids.shape[1]
    cap = p.shape[1]
    pt, prep = prepare(capi, p, H, W)
    grads = torch.empty((11, cap), dtype=torch.float32, device="cuda")
    ws = capi.backward_workspace(H, W, K, cap, max_records)
    m = capi.map_from_ids(ids)
    if saved:
        rgb = torch.empty((H, W, 3), dtype=torch.float32, device="cuda")
        fwd = torch.empty((2, H * W), dtype=torch.float32, device="cuda")
        capi.sad_render_save(prep, cap, H, W, K, m, rgb, fwd)
        capi.sad_render_backward_saved(pt, prep, H, W, K, m, dev(g.astype(np.float32)), rgb, fwd, grads, ws)
    else:
        capi.sad_render_backward(pt, prep, H, W, K, m, dev(g.astype(np.float32)), grads, ws)
    st, used = capi.sad_workspace_status(ws)
    assert st == 0, used
    return grads.cpu().numpy().astype(np.float64), used


@pytest.mark.parametrize("saved", [False, True])
def test_config1_backward(capi, oracle, saved):
    H = W = 64
    img = gen.image_sinusoid_polygons(H, W, seed=1000)
    p = gen.sites_isotropic(img, 256, seed=1001)
    p[0] += 0.01                                           # keep sites off pixel centres
    ids = oracle.propagate_fp32(p, H, W, 8, passes=6, J=2, seed=77)
    g = gen.grad_image(H, W, seed=1002) / (H * W)
    got, used = _backward(capi, p, H, W, ids, g, saved=saved)
    ref = oracle.render_backward(p, H, W, ids, g)
    assert_grads_close(got, ref)
    assert used > 0


@pytest.mark.parametrize("saved", [False, True])
@pytest.mark.parametrize("K", [4, 8, 16])
@pytest.mark.parametrize("H,W", [(40, 56), (17, 33), (1, 1)])
def test_backward_edge_cases(capi, oracle, K, H, W, saved):
    n = max(K + 4, 60)
    p = gen.sites_random_spd(H, W, n, seed=H * 7 + W + K, capacity=n + 5)
    p[2] += 2.0
    p = gen.deactivate_random(p, 0.1, seed=3)
    ids = gen.knn_map(p, H, W, K, seed=4, truncate_frac=0.3, shuffle=True, include_inactive_frac=0.2)
    ids[0, :] = INV
    g = gen.grad_image(H, W, seed=5)
    got, _ = _backward(capi, p, H, W, ids, g, saved=saved)
    ref = oracle.render_backward(p, H, W, ids, g)
    assert_grads_close(got, ref)


@pytest.mark.parametrize("saved", [False, True])
def test_incoherent_map_uses_extra_rounds(capi, oracle, saved):
    """Random, spatially incoherent lists: far more distinct sites per tile
    than the per-round table holds, so the multi-round path runs."""
    H, W, K = 32, 48, 16
    p = gen.sites_random_spd(H, W, 3000, seed=51)
    ids = gen.random_map(H * W, K, 3000, seed=52, invalid_frac=0.05)
    g = gen.grad_image(H, W, seed=53)
    got, used = _backward(capi, p, H, W, ids, g, max_records=H * W * K, saved=saved)
    ref = oracle.render_backward(p, H, W, ids, g)
    assert_grads_close(got, ref)
    assert used > 128 * ((H + 15) // 16) * ((W + 15) // 16)


def test_deterministic_bitwise(capi):
    H, W, K = 200, 150, 16
    p = gen.sites_random_spd(H, W, 2500, seed=61)
    ids = gen.knn_map(p, H, W, K, seed=62)
    g = gen.grad_image(H, W, seed=63)
    a, _ = _backward(capi, p, H, W, ids, g)
    b, _ = _backward(capi, p, H, W, ids, g)
    assert np.array_equal(a.view(np.uint64), b.view(np.uint64))


def test_workspace_overflow_is_reported(capi):
    torch = pytest.importorskip("torch")
    H, W, K = 64, 64, 16
    p = gen.sites_random_spd(H, W, 500, seed=71)
    ids = gen.knn_map(p, H, W, K, seed=72)
    pt, prep = prepare(capi, p, H, W)
    grads = torch.empty((11, 500), dtype=torch.float32, device="cuda")
    ws = capi.backward_workspace(H, W, K, 500, max_records=10)
    capi.sad_render_backward(pt, prep, H, W, K, capi.map_from_ids(ids),
                             dev(gen.grad_image(H, W, 73)), grads, ws)
    st, used = capi.sad_workspace_status(ws)
    assert st == 3 and used > 10


def test_train_grads_and_loss(capi, oracle):
    torch = pytest.importorskip("torch")
    H, W, K = 48, 64, 8
    img = gen.image_noise_polygons_lines(H, W, seed=81, n_polygons=5, n_lines=3)
    p = gen.sites_isotropic(img, 200, seed=82, tau=60.0)
    ids = gen.knn_map(p, H, W, K, seed=83)
    pt, prep = prepare(capi, p, H, W)
    grads = torch.empty((11, 200), dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    rgb = torch.empty((H, W, 3), dtype=torch.float32, device="cuda")
    ws = capi.backward_workspace(H, W, K, 200)
    capi.sad_train_grads(pt, prep, H, W, K, capi.map_from_ids(ids), dev(img), grads, loss, ws, rgb)
    ref_rgb = oracle.render(p, H, W, ids)
    L, g = oracle.mse_loss_and_grad_rgb(ref_rgb, img)
    assert abs(float(loss.item()) - L) <= 1e-5 * max(L, 1e-3)
    assert np.abs(rgb.cpu().numpy().reshape(-1, 3) - ref_rgb).max() <= 1e-5
    assert_grads_close(grads.cpu().numpy().astype(np.float64), oracle.render_backward(p, H, W, ids, g))


@pytest.mark.parametrize("saved", [False, True])
def test_full_size_sampled_sites(capi, oracle, saved):
    """2048^2, 262144 sites, K=16 (config 3, both adjoint forms): 64 sampled
    sites' gradients, each from every pixel that lists it (oracle restricted
    to those pixels)."""
    H = W = 2048
    K = 16
    p = gen.sites_random_spd(H, W, 262144, seed=3000)
    ids = gen.knn_map(p, H, W, K, seed=3001)
    g = gen.grad_image(H, W, seed=3002) / (H * W)
    got, _ = _backward(capi, p, H, W, ids, g, saved=saved)
    rng = np.random.default_rng(3)
    sites = rng.choice(262144, 64, replace=False)
    rows = np.nonzero(np.isin(ids, sites.astype(np.uint32)).any(axis=1))[0]
    r, c = np.divmod(rows, W)
    ref = oracle.render_backward(p, H, W, ids[rows], g.reshape(-1, 3)[rows], c + 0.5, r + 0.5)
    assert_grads_close(got[:, sites], ref[:, sites])


def test_render_save_state(capi, oracle):
    """sad_render_save: the same image as sad_render bit for bit, and per
    pixel the max listed logit and 1/Z of the oracle's softmax (a black pixel
    with no valid site: both 0)."""
    torch = pytest.importorskip("torch")
    H, W, K = 37, 53, 16
    p = gen.sites_random_spd(H, W, 400, seed=61)
    p = gen.deactivate_random(p, 0.15, seed=62)
    ids = gen.knn_map(p, H, W, K, seed=63, truncate_frac=0.3, shuffle=True, include_inactive_frac=0.2)
    ids[5, :] = INV
    cap = p.shape[1]
    _, prep = prepare(capi, p, H, W)
    m = capi.map_from_ids(ids)
    a = torch.empty((H, W, 3), dtype=torch.float32, device="cuda")
    b = torch.empty_like(a)
    fwd = torch.empty((2, H * W), dtype=torch.float32, device="cuda")
    capi.sad_render(prep, cap, H, W, K, m, a)
    capi.sad_render_save(prep, cap, H, W, K, m, b, fwd)
    assert torch.equal(a, b)
    f = fwd.cpu().numpy().astype(np.float64)
    valid, safe = oracle._valid_entries(p, ids)
    px, py = oracle.pixel_centres(H, W)
    l = oracle.logits(p, H, W, safe, px, py)
    lm = np.where(valid, l, -np.inf)
    mx = lm.max(axis=1)
    has = valid.any(axis=1)
    mx_safe = np.where(has, mx, 0.0)
    z = np.where(valid, np.exp(np.where(valid, l, 0.0) - mx_safe[:, None]), 0.0).sum(axis=1)
    np.testing.assert_allclose(f[0][has], mx[has], rtol=1e-5, atol=1e-5)
    np.testing.assert_allclose(f[1][has], 1.0 / z[has], rtol=1e-5)
    assert np.all(f[:, ~has] == 0.0) and (~has).any()

