"""Batched fused training step: equals the unfused single-image sequence,
an image's result does not depend on the batch, graph replay equals eager."""
import numpy as np
import pytest

from paper_2604_21984_gb300 import inputs as gen
from tests.gpu_util import assert_grads_close, dev, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    return require_gpu()


def _images(sizes, seed):
    return [dev(gen.image_noise_polygons_lines(H, W, seed=seed + i, n_polygons=6, n_lines=3))
            for i, (H, W) in enumerate(sizes)]


def test_fused_step_matches_unfused_sequence(capi, oracle):
    """One batched step on a single image == prepare, pass, train_grads, Adam."""
    torch = pytest.importorskip("torch")
    from paper_2604_21984_gb300.batch import BatchConfig, BatchTrainer
    imgs = _images([(40, 56)], 7)
    tr = BatchTrainer(imgs, BatchConfig(K=8, J=2, graph=False, seed=3))
    H, W = 40, 56
    n = tr.total_cap
    p0 = tr.params.clone()
    map0 = capi.ids_from_map(tr.maps[0])
    t_pass = int(tr.state[0, 1].item())
    assert t_pass == tr.images[0]["n_pass"]
    seed = tr.images[0]["seed"]
    grads_fused = torch.empty_like(tr.params)
    capi.sad_train_step(tr.table, 8, 2, tr.params, tr.m, tr.v, tr.prep, tr.maps[0], tr.maps[1],
                        tr.total_pixels, tr.targets, tr.loss, tr.hp, tr.state, tr.ws, grads_out=grads_fused)
    torch.cuda.synchronize()
    # unfused reference on copies
    p = p0.clone()
    prep = capi.empty_prep(n)
    capi.sad_prepare_sites(p, H, W, prep)
    a = capi.map_from_ids(map0)
    b = capi.empty_map(H, W, 8)
    capi.sad_update_topk(prep, n, H, W, 8, a, b, (1 << 16) | t_pass, 2, seed)
    assert np.array_equal(capi.ids_from_map(b), capi.ids_from_map(tr.maps[1]))
    grads = torch.empty_like(p)
    loss = torch.empty(1, device="cuda")
    ws = capi.backward_workspace(H, W, 8, n)
    capi.sad_train_grads(p, prep, H, W, 8, b, imgs[0], grads, loss, ws)
    assert abs(loss.item() - tr.loss[0].item()) <= 1e-6 * loss.item()
    assert_grads_close(grads_fused.cpu().numpy().astype(np.float64), grads.cpu().numpy().astype(np.float64))
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    capi.sad_adam_step(p, grads_fused, m, v, H, W, 1, tr.hp)
    np.testing.assert_allclose(tr.params.cpu().numpy(), p.cpu().numpy(), rtol=1e-6, atol=1e-6)
    # the prepared table was refreshed for the new parameters
    prep2 = capi.empty_prep(n)
    capi.sad_prepare_sites(tr.params, H, W, prep2)
    assert torch.equal(prep2[:5], tr.prep[:5])                       # the float4 planes
    assert torch.equal(prep2[5].reshape(-1)[:n], tr.prep[5].reshape(-1)[:n])   # the dense blue plane


def test_batch_results_do_not_depend_on_the_batch(capi):
    """Three uneven images trained together == each trained alone (bitwise)."""
    torch = pytest.importorskip("torch")
    from paper_2604_21984_gb300.batch import BatchConfig, BatchTrainer
    sizes = [(48, 80), (96, 64), (33, 47)]
    imgs = _images(sizes, 11)
    cfg = BatchConfig(K=16, J=4, graph=False, seed=5)
    tr = BatchTrainer(imgs, cfg)
    tr.run(12)
    for b, img in enumerate(imgs):
        solo = BatchTrainer([img], cfg, seeds=[tr.images[b]["user_seed"]])
        solo.run(12)
        lo, n = tr.images[b]["site_offset"], tr.images[b]["capacity"]
        assert torch.equal(tr.params[:, lo:lo + n], solo.params[:, :n]), b
        assert np.array_equal(tr.map_for(b), solo.map_for(0)), b
        assert tr.loss[b].item() == solo.loss[0].item()


def test_graph_replay_equals_eager(capi):
    torch = pytest.importorskip("torch")
    from paper_2604_21984_gb300.batch import BatchConfig, BatchTrainer
    imgs = _images([(64, 64), (40, 72)], 21)
    a = BatchTrainer(imgs, BatchConfig(K=8, J=4, graph=False, seed=2))
    b = BatchTrainer(imgs, BatchConfig(K=8, J=4, graph=True, seed=2))
    a.run(10)
    b.run(10)
    torch.cuda.synchronize()
    assert torch.equal(a.params, b.params)
    assert torch.equal(a.maps[0], b.maps[0])
    st = b.state.cpu().numpy()
    assert (st[:, 0] == 11).all() and (st[:, 2] == 0).all()
    assert [int(x) for x in st[:, 1]] == [im["n_pass"] + 10 for im in b.images]


def test_batch_training_improves_psnr(capi):
    from paper_2604_21984_gb300.batch import BatchConfig, BatchTrainer
    imgs = _images([(96, 128), (128, 96), (80, 80)], 31)
    tr = BatchTrainer(imgs, BatchConfig(K=16, J=4, seed=1))
    tr.run(2)
    p0 = tr.psnr()
    tr.run(300)
    p1 = tr.psnr()
    print("PSNR", p0, "->", p1)
    assert all(b > a + 3.0 for a, b in zip(p0, p1))


def test_state_rows_carry_each_images_counters(capi):
    """Any distinct state rows give the same training; an image left out of
    some calls resumes from its own row (Adam step, pass index, map parity)."""
    torch = pytest.importorskip("torch")
    from paper_2604_21984_gb300 import capi as C
    from paper_2604_21984_gb300.batch import BatchConfig, BatchTrainer
    imgs = _images([(48, 64), (40, 40)], 41)
    cfg = BatchConfig(K=8, J=3, graph=False, seed=9)
    a = BatchTrainer(imgs, cfg)
    a.run(7)
    b = BatchTrainer(imgs, cfg)
    rows = torch.zeros((5, 4), dtype=torch.int32, device="cuda")
    rows[3] = b.state[0]
    rows[1] = b.state[1]
    b.images[0]["state_index"], b.images[1]["state_index"] = 3, 1
    full = C.batch_table(b.images)
    only0 = C.batch_table([b.images[0]])

    def call(table, B):
        C.sad_train_step(table, 8, 3, b.params, b.m, b.v, b.prep, b.bufs[0], b.bufs[1], b.total_pixels,
                         b.targets, b.loss[:B], b.hp, rows, b.ws)

    for _ in range(3):
        call(full, 2)
    for _ in range(2):      # image 1 sits these out
        call(only0, 1)
    for _ in range(2):
        call(full, 2)
    for _ in range(2):      # image 1 catches up alone
        call(C.batch_table([b.images[1]]), 1)
    torch.cuda.synchronize()
    assert torch.equal(a.params, b.params)
    assert rows[3, 0].item() == 8 and rows[1, 0].item() == 8
    # 7 steps each: both current maps are in bufs[1]
    assert torch.equal(a.maps[0], b.bufs[1])


def test_decode_batch_matches_per_image_decode(capi):
    torch = pytest.importorskip("torch")
    from paper_2604_21984_gb300.batch import BatchConfig, BatchTrainer
    sizes = [(40, 72), (64, 48), (17, 29)]
    imgs = _images(sizes, 51)
    tr = BatchTrainer(imgs, BatchConfig(K=16, J=4, graph=False, seed=4))
    tr.run(6)
    rng = np.random.default_rng(3)
    n = 5000
    qimg = rng.integers(0, len(sizes), n).astype(np.int32)
    xy = np.empty((n, 2), np.float32)
    for b, (H, W) in enumerate(sizes):
        sel = qimg == b
        # include points slightly outside the image (clamped map cell)
        xy[sel, 0] = rng.uniform(-1.0, W + 1.0, sel.sum())
        xy[sel, 1] = rng.uniform(-1.0, H + 1.0, sel.sum())
    qimg[:7] = [-1, 3, 99, 0, 1, 2, 0]
    xy_d, q_d = torch.from_numpy(xy).cuda(), torch.from_numpy(qimg).cuda()
    out = torch.empty((n, 3), device="cuda")
    capi.sad_decode_batch(tr.table, 16, tr.prep, tr.total_cap, tr.maps[0], tr.total_pixels, xy_d, q_d, out)
    got = out.cpu().numpy()
    for b, (H, W) in enumerate(sizes):
        im = tr.images[b]
        lo, cap = im["site_offset"], im["capacity"]
        p = tr.params[:, lo:lo + cap].contiguous()
        prep = capi.empty_prep(cap)
        capi.sad_prepare_sites(p, H, W, prep)
        mp = capi.map_from_ids(tr.map_for(b))
        sel = np.nonzero(qimg == b)[0]
        ref = torch.empty((len(sel), 3), device="cuda")
        capi.sad_decode_points(prep, cap, H, W, 16, mp, xy_d[sel].contiguous(), ref)
        np.testing.assert_allclose(got[sel], ref.cpu().numpy(), rtol=0, atol=1e-6)
    bad = (qimg < 0) | (qimg >= len(sizes))
    assert np.all(got[bad] == 0.0)


def test_keep_lists_step_and_batch_update(capi, oracle):
    """A step flagged to keep its lists = train_grads on the current map +
    Adam; sad_batch_update = sad_update_topk per image (bit-exact)."""
    torch = pytest.importorskip("torch")
    from paper_2604_21984_gb300.batch import BatchConfig, BatchTrainer
    imgs = _images([(40, 56), (33, 47)], 61)
    tr = BatchTrainer(imgs, BatchConfig(K=16, J=4, graph=False, seed=6))
    tr.run(2)
    torch.cuda.synchronize()
    # propagation-only pass of both images vs the single-image pass
    before = [tr.map_for(b) for b in range(2)]
    pass_idx = tr.state[:, 1].cpu().numpy().copy()
    cur, other = tr.maps
    capi.sad_batch_update(tr.table, 16, 4, tr.prep, tr.total_cap, tr.bufs[0], tr.bufs[1], tr.total_pixels,
                          tr.state)
    torch.cuda.synchronize()
    tr.refreshes += 1
    for b, (H, W) in enumerate([(40, 56), (33, 47)]):
        im = tr.images[b]
        lo, n = im["site_offset"], im["capacity"]
        prep = capi.empty_prep(n)
        capi.sad_prepare_sites(tr.params[:, lo:lo + n].contiguous(), H, W, prep)
        a = capi.map_from_ids(before[b])
        out = capi.empty_map(H, W, 16)
        capi.sad_update_topk(prep, n, H, W, 16, a, out, (1 << 16) | int(pass_idx[b]), 4, im["seed"])
        assert np.array_equal(capi.ids_from_map(out), tr.map_for(b)), b
    assert (tr.state[:, 1].cpu().numpy() == pass_idx + 1).all()
    # a keep-lists step: gradients of the current lists, t advances only
    H, W = 40, 56
    im = tr.images[0]
    lo, n = im["site_offset"], im["capacity"]
    p_before = tr.params[:, lo:lo + n].contiguous()
    st_before = tr.state.clone()
    keep = capi.batch_table([dict(x, flags=capi.STEP_KEEP_LISTS) for x in tr.images])
    grads = torch.zeros_like(tr.params)
    capi.sad_train_step(keep, 16, 4, tr.params, tr.m, tr.v, tr.prep, tr.bufs[0], tr.bufs[1], tr.total_pixels,
                        tr.targets, tr.loss, tr.hp, tr.state, tr.ws, grads_out=grads)
    torch.cuda.synchronize()
    st = tr.state.cpu().numpy()
    assert (st[:, 0] == st_before.cpu().numpy()[:, 0] + 1).all()
    assert (st[:, 1:] == st_before.cpu().numpy()[:, 1:]).all()
    prep = capi.empty_prep(n)
    capi.sad_prepare_sites(p_before, H, W, prep)
    g_ref = torch.empty_like(p_before)
    loss = torch.empty(1, device="cuda")
    capi.sad_train_grads(p_before, prep, H, W, 16, capi.map_from_ids(tr.map_for(0)), imgs[0], g_ref, loss,
                         capi.backward_workspace(H, W, 16, n))
    assert abs(loss.item() - tr.loss[0].item()) <= 1e-6 * loss.item()
    assert_grads_close(grads[:, lo:lo + n].cpu().numpy().astype(np.float64), g_ref.cpu().numpy().astype(np.float64))


def test_candidate_period_graph_equals_eager(capi):
    torch = pytest.importorskip("torch")
    from paper_2604_21984_gb300.batch import BatchConfig, BatchTrainer
    imgs = _images([(48, 48), (32, 64)], 71)
    a = BatchTrainer(imgs, BatchConfig(K=8, J=2, graph=False, seed=3, cand_every=3))
    b = BatchTrainer(imgs, BatchConfig(K=8, J=2, graph=True, seed=3, cand_every=3))
    a.run(11)
    b.run(1)
    b.run(10)
    torch.cuda.synchronize()
    assert torch.equal(a.params, b.params)
    assert torch.equal(a.maps[0], b.maps[0])
    assert a.refreshes == b.refreshes == 4


def test_autotune_picks_fastest_within_tolerance_and_caches(capi, tmp_path):
    """The autotuner trains each candidate for the budget, picks the fastest
    whose mean PSNR is within the tolerance of the best, and a second call
    with the same key is served from its JSON cache without training."""
    import json
    import time
    from paper_2604_21984_gb300.batch import autotune
    imgs = _images([(64, 80), (48, 48), (96, 64)], 21)
    cands = ((16, 4, 16), (16, 4, 32), (8, 2))
    path = str(tmp_path / "tune.json")
    t0 = time.perf_counter()
    pick, rows = autotune(imgs, iters=20, candidates=cands, cache_path=path)
    t_first = time.perf_counter() - t0
    assert pick in ((16, 4, 16), (16, 4, 32), (8, 2, 16)) and len(rows) == 3
    assert all(np.isfinite(r[4]) and r[3] > 0 for r in rows)
    q = {}
    for r in rows:
        q.setdefault(r[:2], []).append(r[4])
    q = {kj: float(np.mean(v)) for kj, v in q.items()}
    ok = [r for r in rows if q[r[:2]] >= max(q.values()) - 0.05]
    assert pick == tuple(min(ok, key=lambda r: r[3])[:3])
    t0 = time.perf_counter()
    pick2, rows2 = autotune(imgs, iters=20, candidates=cands, cache_path=path)
    assert pick2 == pick and [tuple(r) for r in rows2] == [tuple(r) for r in rows]
    assert time.perf_counter() - t0 < 0.2 * t_first
    with open(path) as f:
        assert len(json.load(f)) == 1


def test_tile_shapes_agree(capi):
    """The batched step with 32x8 adjoint tiles equals the 16x16 step: the
    same new maps, losses and gradients up to the rounding of the per-tile
    partial sums, on uneven images with ragged tiles."""
    torch = pytest.importorskip("torch")
    from paper_2604_21984_gb300.batch import BatchConfig, BatchTrainer
    imgs = _images([(40, 56), (73, 29), (64, 96)], 31)
    out = {}
    for tw in (16, 32):
        tr = BatchTrainer(imgs, BatchConfig(K=16, J=4, seed=9, graph=False, tile_w=tw))
        grads = torch.empty_like(tr.params)
        capi.sad_train_step(tr.table, 16, 4, tr.params, tr.m, tr.v, tr.prep, tr.bufs[0], tr.bufs[1],
                            tr.total_pixels, tr.targets, tr.loss, tr.hp, tr.state, tr.ws, grads_out=grads,
                            tile_w=tw)
        torch.cuda.synchronize()
        out[tw] = (capi.ids_from_map(tr.bufs[1]), tr.loss.cpu().numpy().copy(), grads.cpu().numpy())
    assert np.array_equal(out[16][0], out[32][0])
    np.testing.assert_allclose(out[32][1], out[16][1], rtol=1e-5)
    g16, g32 = out[16][2].astype(np.float64), out[32][2].astype(np.float64)
    for j in range(11):
        scale = np.abs(g16[j]).max()
        if scale > 0:
            assert np.abs(g32[j] - g16[j]).max() <= 1e-5 * scale, j
    # a bad tile width is refused on the host
    with pytest.raises(capi.SadError):
        capi.sad_train_step(tr.table, 16, 4, tr.params, tr.m, tr.v, tr.prep, tr.bufs[0], tr.bufs[1],
                            tr.total_pixels, tr.targets, tr.loss, tr.hp, tr.state, tr.ws, tile_w=24)


def test_tile_shapes_agree_with_kept_lists(capi):
    """Candidate refresh every 2 iterations (the keep-lists tile kernel on
    the other iterations): 32x8 and 16x16 adjoint tiles train alike over a
    few iterations."""
    torch = pytest.importorskip("torch")
    from paper_2604_21984_gb300.batch import BatchConfig, BatchTrainer
    imgs = _images([(40, 56), (73, 29)], 41)
    losses = {}
    for tw in (16, 32):
        tr = BatchTrainer(imgs, BatchConfig(K=8, J=2, seed=4, graph=False, cand_every=2, tile_w=tw))
        tr.run(4)
        torch.cuda.synchronize()
        losses[tw] = tr.loss.cpu().numpy().copy()
    np.testing.assert_allclose(losses[32], losses[16], rtol=1e-3)
