"""GPU gradient-weighted initialisation (Sec. 4.4) vs the oracle: bit-exact."""
import numpy as np
import pytest

from paper_2604_21984_gb300 import inputs as gen
from tests.gpu_util import dev, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    return require_gpu()


@pytest.mark.parametrize("H,W,n,cap,lam", [(64, 64, 256, 256, 0.3), (512, 768, 32768, 65536, 0.3),
                                          (37, 91, 500, 520, 0.0), (8, 8, 64, 64, 1.0),
                                          (1, 5, 3, 4, 0.5)])
def test_init_sites_bit_exact(capi, oracle, H, W, n, cap, lam):
    img = gen.image_noise_polygons_lines(H, W, seed=H + W, n_polygons=8, n_lines=4)
    got = capi.sad_init_sites(dev(img), n, cap, lam, 1234, 6.25).cpu().numpy()
    ref = oracle.init_sites(img, n, cap, lam, 1234, 6.25)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))


def test_init_flat_image_and_ties(capi, oracle):
    """A flat image with lambda = 0 has all weights 0: every key is +inf and
    the n smallest-index pixels are chosen (ties by index)."""
    img = np.full((16, 20, 3), 0.4, np.float32)
    got = capi.sad_init_sites(dev(img), 30, 30, 0.0, 9, 5.0).cpu().numpy()
    ref = oracle.init_sites(img, 30, 30, 0.0, 9, 5.0)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))
    assert np.array_equal(np.floor(got[1]) * 20 + np.floor(got[0]), np.arange(30))
