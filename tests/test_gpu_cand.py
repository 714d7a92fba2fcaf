"""Half2 candidate sites on the GPU (App. "Data Layout and Packing", Packed
candidate sites) against the oracle: the packed records bit for bit
(saturation, ties to even, subnormals, NaN), and candidate passes scored
from them bit for bit (ragged sizes, every K, long and unit jumps, inactive
sites, the 2048^2 workload on sampled pixels, degenerate inputs).  Calls go
through the C-ABI binding."""
import numpy as np
import pytest

from paper_2604_21984_gb300 import inputs as gen
from tests.gpu_util import dev, prep_to_oracle_dict, prepare, require_gpu

pytestmark = pytest.mark.gpu
INV = 0xFFFFFFFF


@pytest.fixture(scope="module")
def capi():
    return require_gpu()


def _pack(capi, prep, cap):
    torch = pytest.importorskip("torch")
    cand = torch.empty((cap, 4), dtype=torch.int32, device="cuda")
    capi.sad_pack_candidates(prep, cap, cand)
    return cand


def test_pack_bit_exact_with_edge_values(capi, oracle):
    torch = pytest.importorskip("torch")
    H, W = 61, 47
    p = gen.sites_random_spd(H, W, 700, seed=21, capacity=777)
    _, prep = prepare(capi, p, H, W)
    # edge values written straight into the prepared table: above the
    # largest half, ties at 2049 / 2051, a subnormal half, NaN, -0
    edge = torch.tensor([1e6, -1e6, 2049.0, 2051.0, 1e-7, float("nan"), -0.0, 65519.0, 65520.0],
                        dtype=torch.float32, device="cuda")
    n = edge.numel()
    prep[0, :n, 0] = edge
    prep[0, n:2 * n, 2] = edge
    prep[1, :n, 1] = edge.flip(0)
    cand = _pack(capi, prep, p.shape[1])
    ref = oracle.candidate_words(prep_to_oracle_dict(prep, p.shape[1]))
    got = cand.cpu().numpy().view(np.uint32)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("K,J,H,W,t", [(4, 2, 37, 53, 0), (8, 4, 70, 45, 3), (16, 2, 64, 80, 9),
                                       (16, 0, 33, 33, 1), (8, 16, 1, 40, 2)])
def test_h2_pass_bit_exact(capi, oracle, K, J, H, W, t):
    p = gen.sites_random_spd(H, W, max(1, H * W // 6), seed=K + J + t)
    p = gen.deactivate_random(p, 0.2, seed=t + 1)
    cap = p.shape[1]
    _, prep = prepare(capi, p, H, W)
    cand = _pack(capi, prep, cap)
    ids = gen.knn_map(p, H, W, K, seed=3)
    mi, mo = capi.map_from_ids(ids), capi.empty_map(H, W, K)
    code = oracle.step_code(t, H, W)
    capi.sad_update_topk_h2(cand, cap, H, W, K, mi, mo, code, J, 77)
    table = oracle.candidate_table_fp32(oracle.prepare_fp32(p, H, W))
    ref = oracle.topk_pass_fp32(table, ids, H, W, K, code, J, 77)
    assert np.array_equal(capi.ids_from_map(mo), ref)


def test_h2_propagation_from_seed(capi, oracle):
    """Seed + 6 passes at the jump schedule, every pass on the half2 table."""
    H, W, K, J = 64, 64, 8, 2
    img = gen.image_sinusoid_polygons(H, W, seed=1000)
    p = gen.sites_isotropic(img, 256, seed=1001)
    cap = p.shape[1]
    _, prep = prepare(capi, p, H, W)
    cand = _pack(capi, prep, cap)
    a, b = capi.empty_map(H, W, K), capi.empty_map(H, W, K)
    capi.sad_topk_seed(prep, cap, H, W, K, a)
    prep32 = oracle.prepare_fp32(p, H, W)
    table = oracle.candidate_table_fp32(prep32)
    ids = oracle.topk_seed_fp32(prep32, H, W, K)
    for t in range(6):
        code = oracle.step_code(t, H, W)
        capi.sad_update_topk_h2(cand, cap, H, W, K, a, b, code, J, 5)
        a, b = b, a
        ids = oracle.topk_pass_fp32(table, ids, H, W, K, code, J, 5)
    assert np.array_equal(capi.ids_from_map(a), ids)


def test_h2_full_size_sampled_pixels(capi, oracle):
    """2048x2048, 262144 anisotropic sites, K=16, J=2, at jump 1 and at a
    long jump: 2048 sampled pixels bit-exact."""
    H = W = 2048
    K, J = 16, 2
    p = gen.sites_random_spd(H, W, 262144, seed=3000)
    ids = gen.knn_map(p, H, W, K, seed=3001)
    _, prep = prepare(capi, p, H, W)
    cand = _pack(capi, prep, p.shape[1])
    table = oracle.candidate_table_fp32(oracle.prepare_fp32(p, H, W))
    mi, mo = capi.map_from_ids(ids), capi.empty_map(H, W, K)
    sample = np.random.default_rng(5).choice(H * W, 2048, replace=False)
    for t in (11, 2):
        code = oracle.step_code(t, H, W)
        capi.sad_update_topk_h2(cand, p.shape[1], H, W, K, mi, mo, code, J, 99)
        ref = oracle.topk_pass_fp32(table, ids, H, W, K, code, J, 99, sample)
        assert np.array_equal(capi.ids_from_map(mo)[sample], ref), t


def test_h2_degenerate(capi, oracle):
    torch = pytest.importorskip("torch")
    # capacity 0: every list empties
    m, m2 = capi.empty_map(6, 6, 8), capi.empty_map(6, 6, 8)
    capi.sad_topk_seed(capi.empty_prep(0), 0, 6, 6, 8, m)
    cand = torch.empty((0, 4), dtype=torch.int32, device="cuda")
    capi.sad_pack_candidates(capi.empty_prep(0), 0, cand)
    capi.sad_update_topk_h2(cand, 0, 6, 6, 8, m, m2, 0x10000, 2, 1)
    assert np.all(capi.ids_from_map(m2) == INV)
    # 1x1 image, all sites inactive but one
    p = gen.sites_random_spd(1, 1, 3, seed=2)
    p[0, 1:] = -1.0
    _, prep = prepare(capi, p, 1, 1)
    cand = _pack(capi, prep, 3)
    ids = np.full((1, 4), INV, np.uint32)
    ids[0, 0] = 2
    mi, mo = capi.map_from_ids(ids), capi.empty_map(1, 1, 4)
    capi.sad_update_topk_h2(cand, 3, 1, 1, 4, mi, mo, 0x10000, 4, 3)
    ref = oracle.topk_pass_fp32(oracle.candidate_table_fp32(oracle.prepare_fp32(p, 1, 1)), ids, 1, 1, 4,
                                0x10000, 4, 3)
    assert np.array_equal(capi.ids_from_map(mo), ref)
    assert np.all(capi.ids_from_map(mo)[0, 1:] == INV)   # one active site at most
    # a misaligned table is refused on the host
    with pytest.raises(capi.SadError):
        capi.sad_update_topk_h2(cand.view(-1)[1:], 2, 1, 1, 4, mi, mo, 0x10000, 4, 3)


def test_h2_encode_trains_like_float32(capi):
    """Encodes whose refresh passes score from the half2 table land, on
    average over three seeds, within 0.5 dB of the float32-table encodes
    (one seed alone moves by a few tenths of a dB under any change of
    rounding: training is chaotic)."""
    from paper_2604_21984_gb300.encode import EncodeConfig, Encoder
    H, W = 128, 192
    img = dev(gen.image_noise_polygons_lines(H, W, seed=42, n_polygons=10, n_lines=6))
    p16, p32 = [], []
    for seed in (3, 4, 5):
        kw = dict(n_sites=1536, K=16, J=4, iters=300, densify_every=100, densify_start=100,
                  densify_end=200, seed=seed, fused=False)
        p16.append(Encoder(img, EncodeConfig(cand_half2=True, **kw)).run().psnr())
        p32.append(Encoder(img, EncodeConfig(**kw)).run().psnr())
    m16, m32 = float(np.mean(p16)), float(np.mean(p32))
    print(f"PSNR half2 candidates {np.round(p16, 3)} mean {m16:.3f}, float32 {np.round(p32, 3)} mean {m32:.3f}")
    assert m16 > m32 - 0.5


def test_hybrid_warm_up_bit_exact(capi, oracle):
    """Seed + the jump schedule with the passes at jump >= 4 on the half2
    table and the rest on the float32 table (encode.propagate), against the
    oracle running the same mix."""
    from paper_2604_21984_gb300.encode import jump_code, propagate
    H, W, K, J = 72, 100, 16, 4
    img = gen.image_noise_polygons_lines(H, W, seed=12, n_polygons=6, n_lines=3)
    p = gen.sites_isotropic(img, 900, seed=13)
    cap = p.shape[1]
    _, prep = prepare(capi, p, H, W)
    a, b = capi.empty_map(H, W, K), capi.empty_map(H, W, K)
    capi.sad_topk_seed(prep, cap, H, W, K, a)
    codes = [jump_code(t, H, W) for t in range(9)]
    a, b = propagate(prep, cap, H, W, K, J, 21, a, b, codes, half2_min_jump=4)
    prep32 = oracle.prepare_fp32(p, H, W)
    table = oracle.candidate_table_fp32(prep32)
    ids = oracle.topk_seed_fp32(prep32, H, W, K)
    for code in codes:
        ids = oracle.topk_pass_fp32(table if (code >> 16) >= 4 else prep32, ids, H, W, K, code, J, 21)
    assert np.array_equal(capi.ids_from_map(a), ids)
    assert [c >> 16 for c in codes][:3] == [64, 32, 16]
