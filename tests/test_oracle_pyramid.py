"""Pins of the oracle's image pyramid and Sobel gradients (the RLOF pyramid the paper
names in Section 2 but does not define; reading: 2x2 box decimation, Sobel/8, clamped
border). CPU only."""
import numpy as np
import pytest
from scipy import ndimage

import oracle


@pytest.mark.parametrize("shape", [(128, 256), (37, 91), (375, 1242)])
def test_levels_are_block_means(shape):
    rng = np.random.default_rng(shape[0])
    img = rng.integers(0, 256, size=shape).astype(np.uint8)
    L = 5
    pyr = oracle.pyramid(img, L)
    for l, (I, _, _) in enumerate(pyr):
        Hl, Wl = I.shape
        assert (Wl, Hl) == oracle.level_sizes(shape[1], shape[0], L)[l]
        s = 2 ** l
        block = img[: Hl * s, : Wl * s].astype(np.float64).reshape(Hl, s, Wl, s).mean(axis=(1, 3))
        assert np.array_equal(I, block)
        # values are multiples of 4^-l (exact dyadics)
        assert np.array_equal(I * 4 ** l, np.rint(I * 4 ** l))


@pytest.mark.parametrize("shape", [(64, 96), (23, 77)])
def test_gradients_match_library_sobel(shape):
    rng = np.random.default_rng(5)
    img = rng.integers(0, 256, size=shape).astype(np.uint8)
    for I, Ix, Iy in oracle.pyramid(img, 3):
        assert np.array_equal(Ix, ndimage.sobel(I, axis=1, mode="nearest") / 8.0)
        assert np.array_equal(Iy, ndimage.sobel(I, axis=0, mode="nearest") / 8.0)


def test_ramp_gradient_is_slope():
    a, b = 1.5, -0.75
    y, x = np.mgrid[0:40, 0:60].astype(np.float64)
    img = a * x + b * y + 100.0
    (I, Ix, Iy), = oracle.pyramid(img, 1)
    assert np.allclose(Ix[1:-1, 1:-1], a, atol=1e-12)
    assert np.allclose(Iy[1:-1, 1:-1], b, atol=1e-12)
    # clamped border halves the one-sided difference
    assert np.allclose(Ix[5, 0], a / 2) and np.allclose(Iy[0, 5], b / 2)
