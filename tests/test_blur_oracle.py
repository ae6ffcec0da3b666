"""The adaptive-blur oracle against its pins: constants stay constant, sub-half-pixel
sigma is the identity, and away from the borders a uniform sigma equals scipy's
separable Gaussian filter (truncate = 3)."""
import numpy as np
import pytest

from oracle import blur


def test_constant_image_is_invariant():
    rng = np.random.default_rng(0)
    lv = rng.uniform(3, 6, (20, 24))
    out = blur.adaptive_blur(np.full((20, 24), 2.5), lv, 1.0 / 256)
    assert np.abs(out - 2.5).max() < 1e-12


def test_fine_mesh_is_identity():
    rng = np.random.default_rng(1)
    img = rng.uniform(0, 1, (16, 16))
    assert (blur.adaptive_blur(img, np.full((16, 16), 9.0), 1.0 / 256) == img).all()   # sigma = 0.25 px


def test_uniform_sigma_matches_scipy_interior():
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(2)
    img = rng.uniform(0, 1, (40, 44))
    pixel = 1.0 / 256
    level = np.full(img.shape, 5.0)             # sigma = 2^-5 / (2 / 256) = 4 px, radius 12
    ref = ndimage.gaussian_filter1d(ndimage.gaussian_filter1d(img, 4.0, axis=1, truncate=3.0), 4.0, axis=0,
                                    truncate=3.0)
    out = blur.adaptive_blur(img, level, pixel)
    assert np.abs(out[12:-12, 12:-12] - ref[12:-12, 12:-12]).max() < 1e-12


def test_varying_sigma_follows_the_level():
    img = np.zeros((1, 64))
    img[0, 32] = 1.0
    lv = np.full((1, 64), 4.0)                  # sigma 8 px on the left half
    lv[0, 40:] = 9.0                            # 0.25 px on the right: copied
    out = blur.adaptive_blur(img, lv, 1.0 / 256)
    assert out[0, 32] < 0.2 and out[0, 30] > 0
    assert (out[0, 40:] == 0).all()
