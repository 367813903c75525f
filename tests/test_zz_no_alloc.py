"""glt_linearize_noalloc: the allocation-free linearisation entry point.

It is meant for callers that cannot allocate device memory where they call
it (inside stream capture, in real-time loops with a fixed memory budget, in
plugins of frameworks that own all device memory).  This test drives it
through the C ABI on caller-owned device buffers and checks it against the
tracker's glt_debug_linearize on the same inputs, twice in a row (the
scratch array it shares between calls must be left ready for the next one).
Collected last on purpose: a failure here leaves every other test run."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_matches_debug_linearize_twice():
    import torch

    import oracle
    import paper_2607_16897_gb300 as glt
    import synth

    p = synth.pair_c1(4, sigma=2.0, N=500)
    W, H, K = p.cam.W, p.cam.H, p.cam.K
    trk = glt.Tracker(W, H, K, levels=3, max_points=500)
    trk.build_pyramid(glt.GLT_REF, p.ref)
    trk.set_map_points(p.uvd)
    trk.build_pyramid(glt.GLT_CUR, p.cur)
    ref_lv = oracle.pyramid(p.ref, 3)
    cur_lv = oracle.pyramid(p.cur, 3)
    uvd_dev = torch.from_numpy(np.ascontiguousarray(p.uvd, np.float32)).cuda()
    out_dev = torch.zeros(46, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    T = orc_pose = oracle.se3_exp([0.01, -0.02, 0.015, 0.01, -0.02, 0.005])
    a, b = 0.03, 2.0
    Tc = np.ascontiguousarray(T, np.float64).reshape(12)
    for level in (0, 2):
        ref_dev = torch.from_numpy(np.ascontiguousarray(ref_lv[level])).cuda()
        cur_dev = torch.from_numpy(np.ascontiguousarray(cur_lv[level])).cuda()
        want = trk.debug_linearize(level, orc_pose, a, b, want_res=False)
        for call in range(2):
            out_dev.fill_(float("nan"))
            rc = glt.glt_linearize_noalloc(
                ref_dev.data_ptr(), ref_lv[level].shape[1], cur_dev.data_ptr(),
                cur_lv[level].shape[1], W, H, level, K[0], K[1], K[2], K[3], uvd_dev.data_ptr(),
                len(p.uvd), Tc.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), a, b, 9.0, 1e-3,
                out_dev.data_ptr(), stream)
            assert rc == glt.GLT_OK, glt.glt_last_error()
            torch.cuda.synchronize()
            out = out_dev.cpu().numpy()
            Hm = np.zeros((8, 8))
            idx = 0
            for i in range(8):
                for j in range(i, 8):
                    Hm[i, j] = Hm[j, i] = out[idx]
                    idx += 1
            g, E, n = out[36:44], out[44], int(out[45])
            assert n == want["n"] > 0, (level, call)
            # the tolerances of the parity tests: H 1e-5 relative (Frobenius),
            # E 1e-5 relative, g within 1e-5 of sum |w J r| <= sqrt(2 E H_ii)
            assert np.linalg.norm(Hm - want["H"]) <= 1e-5 * np.linalg.norm(want["H"])
            assert abs(E - want["E"]) <= 1e-5 * want["E"]
            bound = np.sqrt(2.0 * want["E"] * np.diag(want["H"]))
            assert (np.abs(g - want["g"]) <= 1e-5 * bound).all(), (level, call)
    # sizes beyond the static scratch are refused without touching the GPU
    rc = glt.glt_linearize_noalloc(ref_dev.data_ptr(), 80, cur_dev.data_ptr(), 80, W, H, 2,
                                   K[0], K[1], K[2], K[3], uvd_dev.data_ptr(), 65537,
                                   Tc.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), a, b, 9.0,
                                   1e-3, out_dev.data_ptr(), stream)
    assert rc == glt.GLT_ERR_CAPACITY and b"65536" in glt.glt_last_error()
    trk.close()
