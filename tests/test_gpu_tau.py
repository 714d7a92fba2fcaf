"""Tau diffusion on the GPU (App. "Tau Diffusion") vs the oracle, and an
encode that uses it."""
import numpy as np
import pytest

from paper_2604_21984_gb300 import inputs as gen
from tests.gpu_util import dev, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    return require_gpu()


@pytest.mark.parametrize("K,lam", [(8, 0.5), (16, 1.0), (4, 0.0)])
def test_tau_diffusion_matches_oracle(capi, oracle, K, lam):
    torch = pytest.importorskip("torch")
    H, W = 70, 90
    p = gen.sites_random_spd(H, W, 800, seed=K)
    p = gen.deactivate_random(p, 0.15, seed=K + 1)
    p[0, :5] = [-3.0, W + 9.0, 0.0, W - 1e-3, 10.5]     # clamped into the image
    p[1, 1] = H + 4.0
    ids = gen.random_map(H * W, K, 820, seed=K + 2, invalid_frac=0.2)
    g = np.random.default_rng(K).normal(size=800).astype(np.float32)
    out = torch.empty(800, dtype=torch.float32, device="cuda")
    capi.sad_tau_diffusion(dev(p), H, W, K, capi.map_from_ids(ids), lam, dev(g), out)
    ref = oracle.tau_diffusion(p, H, W, ids, lam, g.astype(np.float64))
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-5, atol=1e-6)
    with pytest.raises(capi.SadError):
        gg = dev(g)
        capi.sad_tau_diffusion(dev(p), H, W, K, capi.map_from_ids(ids), lam, gg, gg)


def test_encode_with_tau_diffusion(capi):
    from paper_2604_21984_gb300.encode import EncodeConfig, Encoder
    H, W = 128, 192
    img = dev(gen.image_noise_polygons_lines(H, W, seed=47, n_polygons=10, n_lines=6))
    enc = Encoder(img, EncodeConfig(n_sites=1536, K=16, J=4, iters=200, densify_every=0, seed=5,
                                    tau_diffusion=0.3))
    enc.init()
    p0 = enc.psnr()
    enc.run()
    p1 = enc.psnr()
    print(f"PSNR with tau diffusion {p0:.2f} -> {p1:.2f}")
    assert p1 > p0 + 3.0
