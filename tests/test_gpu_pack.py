"""Packed 16-byte evaluation sites on the GPU: pack and unpack equal the
oracle bit for bit; the decode that reads the packed records matches the
oracle's fp64 blend of the unpacked sites; packing a trained encode barely
moves its PSNR."""
import numpy as np
import pytest

from paper_2604_21984_gb300 import inputs as gen
from tests.gpu_util import dev, require_gpu

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def capi():
    return require_gpu()


@pytest.mark.parametrize("n,H,W,frac", [(700, 120, 90, 0.0), (5000, 256, 384, 0.2), (1, 7, 5, 0.0)])
def test_pack_unpack_bit_exact(capi, oracle, n, H, W, frac):
    p = gen.sites_random_spd(H, W, n, seed=n)
    if frac:
        p = gen.deactivate_random(p, frac, seed=n + 1)
    pt = dev(p)
    words, q = capi.sad_pack_sites(pt, H, W)
    w_ref, q_ref = oracle.pack_eval(p, H, W)
    np.testing.assert_array_equal(q.cpu().numpy(), q_ref)
    np.testing.assert_array_equal(words.cpu().numpy().view(np.uint32)[:n], w_ref)
    u = capi.sad_unpack_sites(words, q, n, H, W)
    u_ref = oracle.unpack_eval(w_ref, q_ref, H, W)
    np.testing.assert_array_equal(u.cpu().numpy(), u_ref)


def test_all_inactive(capi, oracle):
    H, W = 16, 16
    p = gen.sites_random_spd(H, W, 10, seed=2)
    p[0] = -1.0
    words, q = capi.sad_pack_sites(dev(p), H, W)
    assert not words.any().item() and not q.any().item()


def test_decode_packed_matches_oracle(capi, oracle):
    torch = pytest.importorskip("torch")
    H, W, K = 120, 90, 16
    p = gen.sites_random_spd(H, W, 700, seed=41)
    p = gen.deactivate_random(p, 0.1, seed=44)
    ids = gen.knn_map(p, H, W, K, seed=42)
    xy = gen.uniform_points(5000, H, W, seed=43)
    xy[:3] = [[0.0, 0.0], [W - 1e-3, H - 1e-3], [-3.0, H + 5.0]]
    words, q = capi.sad_pack_sites(dev(p), H, W)
    rgb = torch.empty((len(xy), 3), dtype=torch.float32, device="cuda")
    capi.sad_decode_packed(words, q.cpu(), p.shape[1], H, W, K, capi.map_from_ids(ids), dev(xy), rgb)
    w_ref, q_ref = oracle.pack_eval(p, H, W)
    u = oracle.unpack_eval(w_ref, q_ref, H, W)
    cx = np.clip(np.floor(xy[:, 0]).astype(int), 0, W - 1)
    cy = np.clip(np.floor(xy[:, 1]).astype(int), 0, H - 1)
    ref = oracle.render(u, H, W, ids[cy * W + cx], xy[:, 0].astype(np.float64), xy[:, 1].astype(np.float64))
    assert np.abs(rgb.cpu().numpy() - ref).max() <= TOL


def test_packed_render_keeps_psnr(capi):
    """A trained encode rendered from its unpacked 16-byte records: the PSNR
    moves by less than 0.05 dB."""
    torch = pytest.importorskip("torch")
    from paper_2604_21984_gb300.encode import EncodeConfig, Encoder
    H, W = 128, 192
    img = dev(gen.image_noise_polygons_lines(H, W, seed=42, n_polygons=10, n_lines=6))
    enc = Encoder(img, EncodeConfig(n_sites=1536, K=16, J=4, iters=300, densify_every=100,
                                    densify_start=100, densify_end=200, seed=3)).run()
    full = enc.render()
    words, q = capi.sad_pack_sites(enc.params, H, W)
    u = capi.sad_unpack_sites(words, q, enc.cap, H, W)
    prep = capi.empty_prep(enc.cap)
    capi.sad_prepare_sites(u, H, W, prep)
    rgb = torch.empty_like(full)
    capi.sad_render(prep, enc.cap, H, W, 16, enc.maps[0], rgb)

    def psnr(x):
        mse = ((x - img) ** 2).mean().item()
        return 10 * np.log10(1.0 / mse)
    d = psnr(full) - psnr(rgb)
    print("PSNR full %.3f packed %.3f" % (psnr(full), psnr(rgb)))
    assert abs(d) < 0.05


def test_render_packed_matches_oracle(capi, oracle):
    torch = pytest.importorskip("torch")
    H, W, K = 96, 128, 16
    p = gen.sites_random_spd(H, W, 900, seed=51)
    ids = gen.knn_map(p, H, W, K, seed=52)
    words, q = capi.sad_pack_sites(dev(p), H, W)
    rgb = torch.empty((H, W, 3), dtype=torch.float32, device="cuda")
    capi.sad_render_packed(words, q.cpu(), p.shape[1], H, W, K, capi.map_from_ids(ids), rgb)
    w_ref, q_ref = oracle.pack_eval(p, H, W)
    u = oracle.unpack_eval(w_ref, q_ref, H, W)
    ref = oracle.render(u, H, W, ids).reshape(H, W, 3)
    assert np.abs(rgb.cpu().numpy() - ref).max() <= TOL
