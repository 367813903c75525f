"""GPU pyramid == FP64 oracle pyramid, byte for byte (integer work)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def glt():
    import paper_2607_16897_gb300 as g
    return g


SIZES = [(320, 240, 3), (640, 480, 4), (641, 479, 4), (752, 480, 4), (1280, 720, 5),
         (16, 16, 1), (37, 23, 2), (200, 130, 4), (129, 67, 3)]


@pytest.mark.parametrize("W,H,L", SIZES)
@pytest.mark.parametrize("device_input", [False, True])
def test_pyramid_bit_exact(glt, orc, W, H, L, device_input):
    import torch
    rng = np.random.default_rng(W * 7 + H)
    img = rng.integers(0, 256, size=(H, W), dtype=np.uint8)
    trk = glt.Tracker(W, H, (W, W, W / 2, H / 2), levels=L, max_points=16)
    ref = orc.pyramid(img, L)
    for slot in (glt.GLT_REF, glt.GLT_CUR):
        src = torch.from_numpy(img).cuda() if device_input else img
        trk.build_pyramid(slot, src)
        for l in range(L):
            np.testing.assert_array_equal(trk.get_pyramid(slot, l), ref[l], err_msg=f"level {l}")
    trk.close()


def test_pyramid_rendered_and_pitched_input(glt, orc, syn):
    import ctypes
    import torch
    p = syn.pair_c1(0)
    W, H = p.cam.W, p.cam.H
    padded = np.zeros((H, W + 37), np.uint8)
    padded[:, :W] = p.cur
    trk = glt.Tracker(W, H, p.cam.K, levels=3, max_points=16)
    dev = torch.from_numpy(padded).cuda()
    rc = glt.glt_build_pyramid(trk.handle, glt.GLT_CUR, dev.data_ptr(), W + 37, 1,
                               torch.cuda.current_stream().cuda_stream)
    assert rc == glt.GLT_OK
    ref = orc.pyramid(p.cur, 3)
    for l in range(3):
        np.testing.assert_array_equal(trk.get_pyramid(glt.GLT_CUR, l), ref[l])
    # a source pointer that is not 4-byte aligned (one byte into the rows)
    padded[:, 1:W + 1] = p.ref
    dev = torch.from_numpy(padded).cuda()
    rc = glt.glt_build_pyramid(trk.handle, glt.GLT_CUR, dev.data_ptr() + 1, W + 37, 1,
                               torch.cuda.current_stream().cuda_stream)
    assert rc == glt.GLT_OK
    for l, lv in enumerate(orc.pyramid(p.ref, 3)):
        np.testing.assert_array_equal(trk.get_pyramid(glt.GLT_CUR, l), lv)
    assert glt.glt_build_pyramid(trk.handle, 5, dev.data_ptr(), W, 1, None) == glt.GLT_ERR_INVALID_ARG
    assert glt.glt_build_pyramid(trk.handle, 0, dev.data_ptr(), W - 1, 1, None) == glt.GLT_ERR_INVALID_ARG
    trk.close()


def test_constant_and_extreme_images(glt, orc):
    for c in (0, 255):
        img = np.full((97, 131), c, np.uint8)
        trk = glt.Tracker(131, 97, (100, 100, 65, 48), levels=4, max_points=16)
        trk.build_pyramid(glt.GLT_CUR, img)
        for l, ref in enumerate(orc.pyramid(img, 4)):
            np.testing.assert_array_equal(trk.get_pyramid(glt.GLT_CUR, l), ref)
        trk.close()


@pytest.mark.parametrize("W,H", [(640, 480), (752, 480), (1280, 720), (336, 200), (1920, 1080)])
def test_large_frames_match_the_oracle(glt, orc, W, H):
    """The frame sizes of the benchmark workloads and larger ones, five levels,
    with saturated and black borders (the clamp reads them): every level is
    byte for byte the oracle's."""
    rng = np.random.default_rng(W + H)
    img = rng.integers(0, 256, (H, W), dtype=np.uint8)
    img[:, :3] = 255
    img[-2:, :] = 0
    trk = glt.Tracker(W, H, (W, W, W / 2, H / 2), levels=5, max_points=16)
    trk.build_pyramid(glt.GLT_CUR, img)
    for l, ref in enumerate(orc.pyramid(img, 5)):
        np.testing.assert_array_equal(trk.get_pyramid(glt.GLT_CUR, l), ref, err_msg=f"level {l}")
    trk.close()
