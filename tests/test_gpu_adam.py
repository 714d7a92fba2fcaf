"""GPU Adam step vs the oracle's (Sec. 6.1)."""
import numpy as np
import pytest

from paper_2604_21984_gb300 import inputs as gen
from tests.gpu_util import dev, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    return require_gpu()


def test_adam_matches_oracle(capi, oracle):
    torch = pytest.importorskip("torch")
    H, W = 300, 200
    p = gen.sites_random_spd(H, W, 5000, seed=91)
    p[2] = np.random.default_rng(0).uniform(1.0, 21.0, 5000)   # some beyond the clamp
    p[3] = np.abs(p[3]) + 0.5
    p = gen.deactivate_random(p, 0.1, seed=92)
    rng = np.random.default_rng(93)
    pt = dev(p)
    m = torch.zeros_like(pt)
    v = torch.zeros_like(pt)
    # the same learning rates on both sides (large enough that every clamp
    # is reached): the test is of the arithmetic, not of the defaults
    lr = (1e-3, 1e-3, 1e-2, 1e-3, 5e-3, 5e-3, 5e-3, 1e-2, 1e-2, 1e-2, 1e-3)
    hp = capi.adam_hparams(lr=lr)
    lr_named = dict(zip(oracle.PLANE_NAMES, lr))
    pr, mr, vr = p.astype(np.float64), np.zeros((11, 5000)), np.zeros((11, 5000))
    for t in range(1, 4):
        g = (rng.standard_normal((11, 5000)) * 10.0 ** rng.uniform(-6, -1, (11, 1))).astype(np.float32)
        capi.sad_adam_step(pt, dev(g), m, v, H, W, t, hp)
        pr, mr, vr = oracle.adam_step(pr, g, mr, vr, t, H, W, lr=lr_named)
    got = pt.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(got, pr, rtol=2e-5, atol=2e-5)
