"""The workspace-free backward entry point.

Some callers cannot allocate device memory (they only receive device
pointers, or run where an allocation is not allowed); for them
sad_render_backward_noalloc uses a scratch buffer that lives inside the
library.  Its results must equal sad_render_backward's, also on a second call
in a row, after the first call has left its data in the shared buffer.  This
file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2604_21984_gb300 import inputs as gen
from tests.gpu_util import assert_grads_close, dev, prepare, require_gpu

pytestmark = pytest.mark.gpu


def test_noalloc_matches_workspace_backward_twice():
    torch = pytest.importorskip("torch")
    capi = require_gpu()
    cases = [(96, 160, 16, 1200, 11), (64, 64, 8, 300, 12)]   # second call: other sizes and data
    for H, W, K, n, seed in cases:
        p = gen.sites_random_spd(H, W, n, seed=seed)
        p[2] += 1.5
        ids = gen.knn_map(p, H, W, K, seed=seed + 1, truncate_frac=0.1)
        g = dev(gen.grad_image(H, W, seed=seed + 2))
        pt, prep = prepare(capi, p, H, W)
        m = capi.map_from_ids(ids)
        ref = torch.empty((11, n), dtype=torch.float32, device="cuda")
        ws = capi.backward_workspace(H, W, K, n)
        capi.sad_render_backward(pt, prep, H, W, K, m, g, ref, ws)
        got = torch.full((11, n), float("nan"), dtype=torch.float32, device="cuda")
        status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        capi.sad_render_backward_noalloc(pt, prep, H, W, K, m, g, got, status)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        assert_grads_close(got.cpu().numpy().astype(np.float64), ref.cpu().numpy().astype(np.float64))


def test_noalloc_rejects_oversize_problem():
    capi = require_gpu()
    L = capi.lib()
    p = __import__("ctypes").c_void_p(256)
    assert L.sad_render_backward_noalloc(p, p, 10, 4096, 2048, 16, p, p, p, None, None) == 1
    assert b"static limit" in L.sad_last_error()
    assert L.sad_render_backward_noalloc(p, p, 300000, 64, 64, 16, p, p, p, None, None) == 1


def test_noalloc_reports_record_overflow_within_the_limits():
    """Spatially incoherent lists (every pixel lists 16 random sites of
    262144) stay inside the size limits but need far more per-tile records
    than the fixed buffer holds: the call must say so through status_out."""
    torch = pytest.importorskip("torch")
    capi = require_gpu()
    H = W = 512
    K, n = 16, 262144
    p = gen.sites_random_spd(H, W, n, seed=21)
    ids = gen.random_map(H * W, K, n, seed=22, invalid_frac=0.0)
    g = dev(gen.grad_image(H, W, seed=23))
    pt, prep = prepare(capi, p, H, W)
    m = capi.map_from_ids(ids)
    got = torch.empty((11, n), dtype=torch.float32, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    capi.sad_render_backward_noalloc(pt, prep, H, W, K, m, g, got, status)
    torch.cuda.synchronize()
    assert int(status.item()) == capi.SAD_EWORKSPACE
    # the buffer keeps working for a problem that fits
    test_noalloc_matches_workspace_backward_twice()
