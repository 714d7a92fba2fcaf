"""Kernel stage tracing: per-kernel launch counts and device times of the
calls made while tracing is on; nothing is recorded while off or while a
stream is being captured; the fused encoder step equals the separate calls."""
import math

import numpy as np
import pytest

from paper_2604_21984_gb300 import inputs as gen
from tests.gpu_util import dev, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    return require_gpu()


def test_trace_counts_launches(capi):
    torch = pytest.importorskip("torch")
    from paper_2604_21984_gb300.encode import EncodeConfig, Encoder
    img = dev(gen.image_noise_polygons_lines(64, 96, seed=3, n_polygons=4, n_lines=2))
    enc = Encoder(img, EncodeConfig(n_sites=300, K=16, J=4, seed=1))
    enc.init()
    capi.sad_trace_collect()
    prev = capi.sad_trace_enable(True)
    try:
        for _ in range(3):
            enc.step()
        enc.render()
        tr = capi.sad_trace_collect()
    finally:
        capi.sad_trace_enable(prev)
    assert tr["k_step_tile"][0] == 3
    # the segmented reduce: one scan launch and the scatter per step
    assert tr["k_seg_scan"][0] == 3
    assert tr["k_rec_scatter"][0] == 3
    assert tr["k_site_step"][0] == 3
    assert "k_step_finish" not in tr        # the site step finishes the step
    assert tr["k_render"][0] == 1 and tr["k_prepare"][0] == 1
    assert all(ms >= 0.0 and math.isfinite(ms) for _, ms in tr.values())
    assert tr["k_step_tile"][1] > 0.0
    # off: nothing recorded
    enc.step()
    assert capi.sad_trace_collect() == {}


def test_trace_skips_graph_capture(capi):
    torch = pytest.importorskip("torch")
    from paper_2604_21984_gb300.batch import BatchConfig, BatchTrainer
    img = dev(gen.image_noise_polygons_lines(48, 48, seed=5, n_polygons=4, n_lines=2))
    tr = BatchTrainer([img], BatchConfig(K=8, J=2, graph=True))
    capi.sad_trace_collect()
    prev = capi.sad_trace_enable(True)
    try:
        tr.run(4)          # capture (not traced) + replays (graph nodes, not library calls)
        torch.cuda.synchronize()
        rec = capi.sad_trace_collect()
    finally:
        capi.sad_trace_enable(prev)
    assert "k_step_tile" not in rec


def test_fused_encoder_matches_separate_calls(capi):
    """The fused iteration and the four separate calls train alike: same
    active count after densify/prune, same PSNR to 0.02 dB, nearly the same
    field (Adam amplifies rounding-level gradient differences near zero)."""
    torch = pytest.importorskip("torch")
    from paper_2604_21984_gb300.encode import EncodeConfig, Encoder
    img = dev(gen.image_noise_polygons_lines(80, 72, seed=8, n_polygons=5, n_lines=3))
    cfg = dict(n_sites=350, K=16, J=4, seed=4, densify_every=5, densify_start=5, densify_end=10)
    a = Encoder(img, EncodeConfig(fused=True, **cfg)).run(12)
    b = Encoder(img, EncodeConfig(fused=False, **cfg)).run(12)
    torch.cuda.synchronize()
    assert a.n_active == b.n_active
    pa, pb = a.psnr(), b.psnr()
    assert abs(pa - pb) < 0.02, (pa, pb)
    same = (capi.ids_from_map(a.maps[0]) == capi.ids_from_map(b.maps[0])).mean()
    assert same > 0.95
