"""GPU render / decode vs the oracle's fp64 blend (Sec. 4.2): |err| <= 1e-5."""
import numpy as np
import pytest

from paper_2604_21984_gb300 import inputs as gen
from tests.gpu_util import dev, prepare, require_gpu

pytestmark = pytest.mark.gpu
TOL = 1e-5
INV = 0xFFFFFFFF


@pytest.fixture(scope="module")
def capi():
    return require_gpu()


def _render(capi, p, H, W, ids):
    torch = pytest.importorskip("torch")
    K = ids.shape[1]
    _, prep = prepare(capi, p, H, W)
    rgb = torch.empty((H, W, 3), dtype=torch.float32, device="cuda")
    capi.sad_render(prep, p.shape[1], H, W, K, capi.map_from_ids(ids), rgb)
    return rgb.cpu().numpy().reshape(-1, 3)


def test_config1_render(capi, oracle):
    H = W = 64
    img = gen.image_sinusoid_polygons(H, W, seed=1000)
    p = gen.sites_isotropic(img, 256, seed=1001)
    ids = oracle.propagate_fp32(p, H, W, 8, passes=6, J=2, seed=77)
    got = _render(capi, p, H, W, ids)
    ref = oracle.render(p, H, W, ids)
    assert np.abs(got - ref).max() <= TOL


@pytest.mark.parametrize("K", [4, 8, 16])
@pytest.mark.parametrize("H,W", [(33, 47), (16, 16), (1, 1), (5, 130)])
def test_render_edge_cases(capi, oracle, K, H, W):
    p = gen.sites_random_spd(H, W, max(K + 4, 40), seed=H * 131 + W, capacity=max(K + 4, 40) + 6)
    p = gen.deactivate_random(p, 0.1, seed=7)
    ids = gen.knn_map(p, H, W, K, seed=8, truncate_frac=0.3, shuffle=True, include_inactive_frac=0.2)
    ids[0, :] = INV                                        # an empty list renders black
    ids[-1, 1] = 10 ** 6                                   # beyond capacity: skipped
    got = _render(capi, p, H, W, ids)
    ref = oracle.render(p, H, W, ids)
    assert np.abs(got - ref).max() <= TOL
    assert np.all(got[0] == 0)


def test_sharp_temperatures(capi, oracle):
    """Trained-like sharpness: tau * s * |dl| up to ~30 across a list."""
    H, W = 96, 80
    p = gen.sites_random_spd(H, W, 600, seed=31)
    p[2] = np.random.default_rng(1).uniform(3.0, 7.5, 600)
    ids = gen.knn_map(p, H, W, 16, seed=32)
    got = _render(capi, p, H, W, ids)
    assert np.abs(got - oracle.render(p, H, W, ids)).max() <= TOL


def test_full_size_sampled(capi, oracle):
    H = W = 2048
    p = gen.sites_random_spd(H, W, 262144, seed=3000)
    ids = gen.knn_map(p, H, W, 16, seed=3001)
    got = _render(capi, p, H, W, ids)
    sample = np.random.default_rng(9).choice(H * W, 4096, replace=False)
    row, col = np.divmod(sample, W)
    ref = oracle.render(p, H, W, ids[sample], col + 0.5, row + 0.5)
    assert np.abs(got[sample] - ref).max() <= TOL


def test_decode_points(capi, oracle):
    torch = pytest.importorskip("torch")
    H, W, K = 120, 90, 16
    p = gen.sites_random_spd(H, W, 700, seed=41)
    ids = gen.knn_map(p, H, W, K, seed=42)
    xy = gen.uniform_points(5000, H, W, seed=43)
    xy[:3] = [[0.0, 0.0], [W - 1e-3, H - 1e-3], [-3.0, H + 5.0]]   # borders and outside
    _, prep = prepare(capi, p, H, W)
    rgb = torch.empty((len(xy), 3), dtype=torch.float32, device="cuda")
    capi.sad_decode_points(prep, p.shape[1], H, W, K, capi.map_from_ids(ids), dev(xy), rgb)
    cx = np.clip(np.floor(xy[:, 0]).astype(int), 0, W - 1)
    cy = np.clip(np.floor(xy[:, 1]).astype(int), 0, H - 1)
    ref = oracle.render(p, H, W, ids[cy * W + cx], xy[:, 0].astype(np.float64), xy[:, 1].astype(np.float64))
    assert np.abs(rgb.cpu().numpy() - ref).max() <= TOL
