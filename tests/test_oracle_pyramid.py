"""Pins of the oracle's pyramid (Sec. IV-C "Image pyramids").

The pyramid is integer and has a plain definition, so it is pinned against a
library convolution (scipy.ndimage, clamp-to-edge = mode 'nearest') and
closed-form impulse cases stored in tests/golden/pyramid_impulse.txt."""
import os

import numpy as np
import pytest

scipy_ndimage = pytest.importorskip("scipy.ndimage")

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "pyramid_impulse.txt")
K1 = np.array([1, 4, 6, 4, 1], dtype=np.int64)


def scipy_down(img):
    k2 = np.outer(K1, K1)
    s = scipy_ndimage.correlate(img.astype(np.int64), k2, mode="nearest")
    H, W = img.shape
    s = s[0:2 * (H // 2):2, 0:2 * (W // 2):2]
    return ((s + 128) // 256).astype(np.uint8)


@pytest.mark.parametrize("shape", [(2, 2), (3, 7), (5, 5), (6, 9), (17, 31), (48, 64), (61, 83)])
def test_pyr_down_matches_library_convolution(orc, shape):
    rng = np.random.default_rng(shape[0] * 1000 + shape[1])
    img = rng.integers(0, 256, size=shape, dtype=np.uint8)
    np.testing.assert_array_equal(orc.pyr_down(img), scipy_down(img))


def test_pyramid_levels_chain_and_dims(orc):
    rng = np.random.default_rng(5)
    img = rng.integers(0, 256, size=(123, 301), dtype=np.uint8)
    lv = orc.pyramid(img, 5)
    assert [l.shape for l in lv] == [(123, 301), (61, 150), (30, 75), (15, 37), (7, 18)]
    np.testing.assert_array_equal(lv[0], img)
    cur = img
    for l in range(1, 5):
        cur = scipy_down(cur)
        np.testing.assert_array_equal(lv[l], cur)


def test_constant_image_stays_constant(orc):
    for c in (0, 1, 127, 128, 255):
        img = np.full((40, 52), c, np.uint8)
        for lv in orc.pyramid(img, 4):
            assert (lv == c).all()


def test_golden_impulses(orc):
    n = 0
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        name, W, H, x, y, v, x1, y1, exp = line.split()
        img = np.zeros((int(H), int(W)), np.uint8)
        img[int(y), int(x)] = int(v)
        got = orc.pyr_down(img)[int(y1), int(x1)]
        assert int(got) == int(exp), name
        n += 1
    assert n >= 7


def test_border_clamp(orc):
    # a bright first column: clamp-to-edge replicates it into taps x = -1, -2
    img = np.zeros((8, 8), np.uint8)
    img[:, 0] = 200
    out = orc.pyr_down(img)
    # level-1 x=0 sees level-0 x in {-2,-1,0,1,2} -> {0,0,0,1,2}: weights 1+4+6 = 11
    assert out[2, 0] == (11 * 16 * 200 + 128) >> 8
    assert out[2, 1] == (1 * 16 * 200 + 128) >> 8  # x1=1 sees x=0 with weight 1
