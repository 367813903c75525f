"""glt_track_image_async: the CUR pyramid and the solve issued as one chain of
programmatic dependent launches (each kernel starts while its predecessor
runs and waits on the device for its data).  The pyramid it leaves must equal
the FP64 oracle's byte for byte, and the result must equal the unchained path
(glt_build_pyramid + glt_track_frame_async) bit for bit, for every image size
class (odd sizes, widths that allow 16-, 4- and 1-byte loads, one level), every
cluster shape and the Jacobian / pattern / precision variants."""
import ctypes

import numpy as np
import pytest

from helpers import I34, ROT_TOL, TRANS_TOL, both_sides, pose_diff

pytestmark = pytest.mark.gpu

SIZES = [(320, 240, 3), (640, 480, 4), (641, 479, 4), (752, 480, 4), (1280, 720, 5),
         (16, 16, 1), (37, 23, 2), (200, 130, 4), (129, 67, 3), (644, 481, 6)]
SHAPES = [(1, 128), (2, 256), (8, 128), (3, 512), (16, 128), (8, 256)]


@pytest.fixture(scope="module")
def glt():
    import paper_2607_16897_gb300 as g
    return g


def random_points(rng, W, H, n):
    u = rng.uniform(2.0, W - 3.0, n)
    v = rng.uniform(2.0, H - 3.0, n)
    d = rng.uniform(1.0, 5.0, n)
    return np.stack([u, v, d], 1).astype(np.float32)


def chained_vs_separate(glt, trk, frame_dev, init_dev, pitch=None):
    import torch
    out1 = torch.zeros(glt.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    out2 = torch.zeros(glt.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    trk.track_image_async(frame_dev, init_dev, out1, pitch=pitch)
    torch.cuda.synchronize()
    pyr = [trk.get_pyramid(glt.GLT_CUR, l) for l in range(trk.L)]
    # overwrite the levels, then the separate calls
    trk.build_pyramid(glt.GLT_CUR, np.zeros((trk.H, trk.W), np.uint8))
    if pitch is None:
        trk.build_pyramid(glt.GLT_CUR, frame_dev)
    else:
        import ctypes
        rc = glt.glt_build_pyramid(trk.handle, glt.GLT_CUR, ctypes.c_void_p(frame_dev), pitch, 1,
                                   torch.cuda.current_stream().cuda_stream)
        assert rc == glt.GLT_OK
    trk.track_frame_async(init_dev, out2)
    torch.cuda.synchronize()
    return pyr, glt.parse_results(out1)[0], glt.parse_results(out2)[0]


@pytest.mark.parametrize("W,H,L", SIZES)
@pytest.mark.parametrize("cluster,threads", SHAPES)
def test_chained_pyramid_bit_exact(glt, orc, W, H, L, cluster, threads):
    import torch
    rng = np.random.default_rng(W * 31 + H + cluster)
    img = rng.integers(0, 256, size=(H, W), dtype=np.uint8)
    ref = rng.integers(0, 256, size=(H, W), dtype=np.uint8)
    trk = glt.Tracker(W, H, (W, W, W / 2, H / 2), levels=L, max_points=64, cluster=cluster,
                      threads=threads)
    trk.build_pyramid(glt.GLT_REF, ref)
    trk.set_map_points(random_points(rng, W, H, 64))
    init = torch.tensor(np.concatenate([I34.ravel(), [0.0, 0.0]]), dtype=torch.float64).cuda()
    pyr, r1, r2 = chained_vs_separate(glt, trk, torch.from_numpy(img).cuda(), init)
    for l, lv in enumerate(orc.pyramid(img, L)):
        np.testing.assert_array_equal(pyr[l], lv, err_msg=f"level {l}")
    assert np.array_equal(r1["T"], r2["T"]) and r1["passes"] == r2["passes"]
    assert r1["status"] == r2["status"] and r1["n_valid"] == r2["n_valid"]
    trk.close()


def test_pitched_and_unaligned_frames(glt, orc):
    """Frame rows with a pitch, and a frame one byte off 4-byte alignment."""
    import torch
    W, H, L = 640, 480, 4
    rng = np.random.default_rng(5)
    img = rng.integers(0, 256, size=(H, W), dtype=np.uint8)
    trk = glt.Tracker(W, H, (500.0, 500.0, 320.0, 240.0), levels=L, max_points=64)
    trk.build_pyramid(glt.GLT_REF, img)
    trk.set_map_points(random_points(rng, W, H, 64))
    init = torch.tensor(np.concatenate([I34.ravel(), [0.0, 0.0]]), dtype=torch.float64).cuda()
    want = orc.pyramid(img, L)
    # (byte offset, row stride): 16-byte loads, 4-byte loads, byte loads
    for off, stride in ((0, W + 16), (0, W + 4), (1, W + 37)):
        buf = np.zeros((H, stride), np.uint8)
        buf[:, off:off + W] = img
        dev = torch.from_numpy(buf).cuda()
        pyr, r1, r2 = chained_vs_separate(glt, trk, dev.data_ptr() + off, init, pitch=stride)
        for l in range(L):
            np.testing.assert_array_equal(pyr[l], want[l], err_msg=f"offset {off} level {l}")
        assert np.array_equal(r1["T"], r2["T"])
    trk.close()


@pytest.mark.parametrize("kw", [dict(jacobian="ic"), dict(pattern=7, jacobian="ic", levels=4),
                                dict(precision="mixed"), dict()])
def test_chained_track_matches_oracle(glt, orc, syn, kw):
    """Rendered frames: the chained track agrees with the oracle (GLT_MIXED
    adds the FP16 packing kernel to the chain)."""
    import torch
    p = syn.pair_c1(3, sigma=2.0)
    kw = dict(kw)
    levels = kw.pop("levels", 3)
    trk, o = both_sides(glt, orc, p.cam.W, p.cam.H, p.cam.K, p.ref, p.cur, p.uvd, levels=levels, **kw)
    init = torch.tensor(np.concatenate([I34.ravel(), [0.0, 0.0]]), dtype=torch.float64).cuda()
    out = torch.zeros(glt.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    trk.track_image_async(torch.from_numpy(p.cur).cuda(), init, out)
    g = glt.parse_results(out)[0]
    r = o.track_frame(I34)
    ang, dt = pose_diff(g["T"], r["T"])
    assert ang <= ROT_TOL and dt <= TRANS_TOL, (kw, ang, dt)
    for l, lv in enumerate(orc.pyramid(p.cur, levels)):
        np.testing.assert_array_equal(trk.get_pyramid(glt.GLT_CUR, l), lv)
    trk.close()


def test_arguments(glt, orc, syn):
    import torch
    p = syn.pair_c1(0)
    trk = glt.Tracker(p.cam.W, p.cam.H, p.cam.K, levels=3, max_points=len(p.uvd))
    init = torch.zeros(14, dtype=torch.float64, device="cuda")
    out = torch.zeros(glt.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    cur = torch.from_numpy(p.cur).cuda()
    with pytest.raises(glt.GltError, match=r"\(-3\)"):          # no map points yet
        trk.track_image_async(cur, init, out)
    trk.build_pyramid(glt.GLT_REF, p.ref)
    trk.set_map_points(p.uvd)
    with pytest.raises(glt.GltError, match=r"\(-1\)"):
        trk.track_image_async(cur, init, out, pitch=p.cam.W - 1)
    trk.close()


def test_one_call_per_frame(glt, orc, syn):
    """glt_track_image (host or device frame, explicit or state-driven start)
    returns what the asynchronous chain returns, and advances the state."""
    import torch
    p = syn.pair_c1(4, sigma=2.0)
    trk, o = both_sides(glt, orc, p.cam.W, p.cam.H, p.cam.K, p.ref, p.cur, p.uvd, levels=3)
    init = torch.tensor(np.concatenate([I34.ravel(), [0.0, 0.0]]), dtype=torch.float64).cuda()
    out = torch.zeros(glt.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    trk.track_image_async(torch.from_numpy(p.cur).cuda(), init, out)
    want = glt.parse_results(out)[0]
    host = trk.track_image(p.cur, I34, (0.0, 0.0))
    dev = trk.track_image(torch.from_numpy(p.cur).cuda(), I34, (0.0, 0.0))
    for g in (host, dev):
        assert np.array_equal(g["T"], want["T"]) and g["passes"] == want["passes"]
    st = trk.get_state()
    assert st.frames == 2 and np.array_equal(np.array(st.T_cr[:]).reshape(3, 4), dev["T"])
    # pitched host frame, state-driven start (the motion is identity after two equal frames)
    padded = np.zeros((p.cam.H, p.cam.W + 24), np.uint8)
    padded[:, :p.cam.W] = p.cur
    g = trk.track_image(padded[:, :p.cam.W])
    r = o.track_frame(want["T"])
    ang, dt = pose_diff(g["T"], r["T"])
    assert ang <= ROT_TOL and dt <= TRANS_TOL
    assert trk.get_state().frames == 3
    with pytest.raises(ValueError):
        trk.track_image(p.cur[:, :10])              # narrower than the tracker
    r = glt.glt_result()
    rc = glt.glt_track_image(trk.handle, p.cur.ctypes.data, p.cam.W - 1, 0, None, None,
                             ctypes.byref(r), None)
    assert rc == glt.GLT_ERR_INVALID_ARG             # pitch below the width
    trk.close()
