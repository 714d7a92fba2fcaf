"""Serving layer on the GPU: an encode served in a changing mix of other
encodes returns bit-for-bit what it returns alone; batched decode answers
equal the plain per-request decode; a short real-time stream completes."""
import numpy as np
import pytest

from paper_2604_21984_gb300 import inputs as gen
from tests.gpu_util import dev, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    return require_gpu()


def _img(H, W, seed):
    return dev(gen.image_noise_polygons_lines(H, W, seed=seed, n_polygons=5, n_lines=2))


def _small_cfg(**kw):
    from paper_2604_21984_gb300.serve import ServeConfig
    return ServeConfig(K=16, J=4, site_pool=40000, pixel_pool=1 << 18, max_side=256,
                       max_decode_per_tick=1 << 16, **kw)


@pytest.mark.parametrize("pixels_per_call", [1 << 21, 1])
def test_encode_in_a_mix_equals_encode_alone(capi, pixels_per_call):
    """pixels_per_call=1 steps only the encode with the least remaining work
    in each call, so the others skip calls (their own counters and map
    buffer carry their state)."""
    torch = pytest.importorskip("torch")
    from paper_2604_21984_gb300.batch import BatchConfig, BatchTrainer
    from paper_2604_21984_gb300.serve import Request, Server
    srv = Server(_small_cfg(pixels_per_call=pixels_per_call))
    specs = [((48, 64), 11, 9), ((80, 40), 12, 14), ((33, 57), 13, 6), ((64, 64), 14, 10)]
    reqs = [Request("encode", image=_img(H, W, sd), iters=it, seed=1000 + sd) for (H, W), sd, it in specs]
    # staggered joins: 0 at tick 0, 1 at tick 2, 2 and 3 at tick 5
    joins = {0: [0], 2: [1], 5: [2, 3]}
    t = 0
    while t < 6 or srv.busy():
        for k in joins.get(t, []):
            srv.submit(reqs[k])
        srv.tick()
        t += 1
    torch.cuda.synchronize()
    for r, ((H, W), sd, it) in zip(reqs, specs):
        solo = BatchTrainer([r.image], BatchConfig(K=16, J=4, graph=False), seeds=[r.seed])
        solo.run(it)
        n = solo.total_cap
        assert r.result.shape == (11, n)
        assert torch.equal(r.result, solo.params[:, :n]), (H, W)
    # every range went back to the pools
    assert srv.sites.free_total() == srv.cfg.site_pool
    assert srv.pixels.free_total() == srv.cfg.pixel_pool


def test_batched_decode_equals_plain_decode(capi):
    torch = pytest.importorskip("torch")
    from paper_2604_21984_gb300.serve import PlainLoop, Request, Server
    cfg = _small_cfg()
    srv, plain = Server(cfg), PlainLoop(cfg)
    sets = [(96, 128, 700, 1), (200, 150, 1800, 2)]
    for H, W, N, sd in sets:
        p = dev(gen.sites_random_spd(H, W, N, seed=sd))
        srv.add_resident(p, H, W, passes=8)
        plain.add_resident(p, H, W, passes=8)
    # an encode in flight does not disturb the resident sets
    srv.submit(Request("encode", image=_img(64, 48, 3), iters=3, seed=5))
    rng = np.random.default_rng(0)
    reqs = []
    for k in range(6):
        b = k % 2
        H, W = sets[b][0], sets[b][1]
        n = int(rng.integers(1, 3000))
        xy = np.stack([rng.uniform(0, W, n), rng.uniform(0, H, n)], 1).astype(np.float32)
        reqs.append((Request("decode", resident=b, xy=torch.from_numpy(xy).pin_memory()),
                     Request("decode", resident=b, xy=torch.from_numpy(xy).pin_memory())))
    for a, _ in reqs[:3]:
        srv.submit(a)
    srv.tick()
    srv.tick()
    for a, _ in reqs[3:]:
        srv.submit(a)
    while srv.busy():
        srv.tick()
    for _, b in reqs:
        plain.submit(b)
        plain.run_one()
    torch.cuda.synchronize()
    for a, b in reqs:
        np.testing.assert_allclose(a.result.numpy(), b.result.numpy(), rtol=0, atol=1e-6)


def test_stream_replay_completes(capi):
    torch = pytest.importorskip("torch")
    from paper_2604_21984_gb300.serve import Request, Server, latency_summary, run_stream
    srv = Server(_small_cfg())
    p = dev(gen.sites_random_spd(64, 64, 240, seed=4))
    srv.add_resident(p, 64, 64, passes=6)
    rng = np.random.default_rng(1)
    reqs, t = [], 0.0
    for k in range(12):
        t += rng.exponential(0.01)
        if k % 3 == 0:
            reqs.append(Request("encode", arrival=t, image=_img(40 + k, 56, k), iters=20, seed=k))
        else:
            xy = torch.from_numpy(rng.uniform(0, 64, (500, 2)).astype(np.float32)).pin_memory()
            reqs.append(Request("decode", arrival=t, resident=0, xy=xy))
    wall = run_stream(srv, reqs)
    s = latency_summary(reqs)
    assert s["encode"]["n"] == 4 and s["decode"]["n"] == 8
    assert all(r.latency is not None and -1e-3 <= r.latency < wall + 1e-3 for r in reqs)
    assert all(np.isfinite(r.result.cpu().numpy()).all() for r in reqs)


def test_served_encode_trains_like_the_plain_loop(capi):
    """Same seed: the served (batched, in a mix) encode and the plain loop's
    one-image encode give the same sites bit for bit."""
    torch = pytest.importorskip("torch")
    from paper_2604_21984_gb300.encode import psnr_from_loss
    from paper_2604_21984_gb300.serve import PlainLoop, Request, Server
    cfg = _small_cfg()
    srv, plain = Server(cfg), PlainLoop(cfg)
    img = _img(72, 96, 21)
    a = Request("encode", image=img, iters=60, seed=77)
    b = Request("encode", image=img, iters=60, seed=77)
    srv.submit(Request("encode", image=_img(50, 40, 22), iters=25, seed=3))   # company
    srv.submit(a)
    while srv.busy():
        srv.train_tick(4)
    plain.submit(b)
    plain.run_one()
    torch.cuda.synchronize()
    assert torch.equal(a.result, b.result)
    assert a.loss.item() == b.loss.item()


def test_submit_rejects_what_cannot_be_served(capi):
    """Admission failures are raised at submit, on the host, before any work
    is queued: an encode above max_side, an encode that fits max_side but not
    the pools left beside a resident set, a decode of an unknown resident
    set, a decode above max_decode_per_tick."""
    torch = pytest.importorskip("torch")
    from paper_2604_21984_gb300.serve import Request, Server
    srv = Server(_small_cfg())
    with pytest.raises(ValueError, match="max_side"):
        srv.submit(Request("encode", image=_img(300, 200, 1), iters=5))
    ok = Request("encode", image=_img(256, 256, 2), iters=5)
    srv.submit(ok)                                  # fits while the pools are empty
    assert srv.cancel(ok) and not srv.busy()
    p = dev(gen.sites_random_spd(400, 500, 12000, seed=3))
    srv.add_resident(p, 400, 500, passes=4)        # 200000 of the 262144 pool pixels
    with pytest.raises(ValueError, match="pools left"):
        srv.submit(Request("encode", image=_img(256, 256, 2), iters=5))
    xy = torch.zeros((10, 2), dtype=torch.float32)
    with pytest.raises(ValueError, match="unknown resident"):
        srv.submit(Request("decode", resident=1, xy=xy))
    with pytest.raises(ValueError, match="unknown resident"):
        srv.submit(Request("decode", resident=-1, xy=xy))
    with pytest.raises(ValueError, match="max_decode_per_tick"):
        srv.submit(Request("decode", resident=0, xy=torch.zeros(((1 << 16) + 1, 2))))
    with pytest.raises(ValueError):
        srv.submit(Request("render"))
    assert not srv.busy()
    d = Request("decode", resident=0, xy=xy)
    srv.submit(d)
    assert srv.cancel(d) and not srv.busy() and d.cancelled


def test_cancel_hands_back_ranges_and_rows(capi):
    """Withdrawing a waiting and an admitted encode: the others finish with
    the same sites as when served without them, the cancelled ones never
    complete, and the allocator's free totals and the free state rows come
    back to their starting values."""
    torch = pytest.importorskip("torch")
    from paper_2604_21984_gb300.serve import Request, Server
    srv = Server(_small_cfg())
    free_s, free_p, rows = srv.sites.free_total(), srv.pixels.free_total(), len(srv.free_rows)
    specs = [((64, 64), 21, 30), ((48, 80), 22, 25), ((56, 40), 23, 20)]
    reqs = [Request("encode", image=_img(H, W, sd), iters=it, seed=sd) for (H, W), sd, it in specs]
    for r in reqs:
        srv.submit(r)
    srv.train_tick(1)                                # admits all three, one iteration each
    assert len(srv.active) == 3
    late = Request("encode", image=_img(32, 32, 24), iters=10, seed=24)
    srv.submit(late)
    assert srv.cancel(late) and late not in srv.waiting
    assert srv.cancel(reqs[1])                       # admitted, with work in flight
    assert not srv.cancel(reqs[1])                   # already withdrawn
    while srv.busy():
        srv.train_tick(4)
    torch.cuda.synchronize()
    assert reqs[1].cancelled and reqs[1].result is None and reqs[1].done_event is None
    assert srv.sites.free_total() == free_s
    assert srv.pixels.free_total() == free_p
    assert len(srv.free_rows) == rows
    # the survivors are unaffected by the withdrawal
    for k in (0, 2):
        (H, W), sd, it = specs[k]
        solo = Server(_small_cfg())
        r = Request("encode", image=_img(H, W, sd), iters=it, seed=sd)
        solo.submit(r)
        while solo.busy():
            solo.train_tick(4)
        torch.cuda.synchronize()
        assert torch.equal(r.result, reqs[k].result), k
