"""glt_linearize_noalloc: the allocation-free linearisation entry point.

It is meant for callers that cannot allocate device memory where they call
it: real-time loops with a memory budget fixed at start-up, and plugins of
frameworks that own every device allocation.  These tests drive it through
the C ABI on caller-owned device buffers and check it against the tracker's
glt_debug_linearize on the same inputs, two calls in a row (the scratch array
it shares between calls must be left ready for the next one), against the
FP64 oracle directly, at the capacity of its static scratch (65536 points,
all 512 block partials) and with no points at all.  Collected last on
purpose: a failure here leaves every other test run."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

MAX_POINTS = 65536


def _unpack(out):
    Hm = np.zeros((8, 8))
    idx = 0
    for i in range(8):
        for j in range(i, 8):
            Hm[i, j] = Hm[j, i] = out[idx]
            idx += 1
    return Hm, out[36:44], out[44], int(out[45])


class _Case:
    """A C1 frame pair with its level images and points on the device."""

    def __init__(self, torch, oracle, synth, N=500):
        self.p = synth.pair_c1(4, sigma=2.0, N=N)
        self.ref_lv = oracle.pyramid(self.p.ref, 3)
        self.cur_lv = oracle.pyramid(self.p.cur, 3)
        self.ref_dev = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in self.ref_lv]
        self.cur_dev = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in self.cur_lv]
        self.out_dev = torch.zeros(46, dtype=torch.float64, device="cuda")
        self.T = oracle.se3_exp([0.01, -0.02, 0.015, 0.01, -0.02, 0.005])
        self.a, self.b = 0.03, 2.0

    def call(self, glt, torch, level, uvd_dev, n):
        W, H, K = self.p.cam.W, self.p.cam.H, self.p.cam.K
        Tc = np.ascontiguousarray(self.T, np.float64).reshape(12)
        self.out_dev.fill_(float("nan"))
        rc = glt.glt_linearize_noalloc(
            self.ref_dev[level].data_ptr(), self.ref_lv[level].shape[1],
            self.cur_dev[level].data_ptr(), self.cur_lv[level].shape[1], W, H, level, K[0], K[1],
            K[2], K[3], uvd_dev.data_ptr() if uvd_dev is not None else 0, n,
            Tc.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), self.a, self.b, 9.0, 1e-3,
            self.out_dev.data_ptr(), torch.cuda.current_stream().cuda_stream)
        assert rc == glt.GLT_OK, glt.glt_last_error()
        torch.cuda.synchronize()
        return self.out_dev.cpu().numpy()


def _close(out, want, where):
    """The parity tolerances of the tests: H 1e-5 relative (Frobenius), E 1e-5
    relative, n exact, g within 1e-5 of sum |w J r| <= sqrt(2 E H_ii)."""
    Hm, g, E, n = _unpack(out)
    assert n == want["n"] > 0, where
    assert np.linalg.norm(Hm - want["H"]) <= 1e-5 * np.linalg.norm(want["H"]), where
    assert abs(E - want["E"]) <= 1e-5 * want["E"], where
    bound = np.sqrt(2.0 * want["E"] * np.diag(want["H"]))
    assert (np.abs(g - want["g"]) <= 1e-5 * bound).all(), where


def test_noalloc_matches_debug_linearize_twice():
    import torch

    import oracle
    import paper_2607_16897_gb300 as glt
    import synth

    c = _Case(torch, oracle, synth)
    p = c.p
    trk = glt.Tracker(p.cam.W, p.cam.H, p.cam.K, levels=3, max_points=500)
    trk.build_pyramid(glt.GLT_REF, p.ref)
    trk.set_map_points(p.uvd)
    trk.build_pyramid(glt.GLT_CUR, p.cur)
    uvd_dev = torch.from_numpy(np.ascontiguousarray(p.uvd, np.float32)).cuda()
    for level in (0, 2):
        want = trk.debug_linearize(level, c.T, c.a, c.b, want_res=False)
        for call in range(2):
            _close(c.call(glt, torch, level, uvd_dev, len(p.uvd)), want, (level, call))
    # sizes beyond the static scratch are refused without touching the GPU
    Tc = np.ascontiguousarray(c.T, np.float64).reshape(12)
    rc = glt.glt_linearize_noalloc(c.ref_dev[2].data_ptr(), 80, c.cur_dev[2].data_ptr(), 80,
                                   p.cam.W, p.cam.H, 2, *p.cam.K, uvd_dev.data_ptr(),
                                   MAX_POINTS + 1,
                                   Tc.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), c.a, c.b,
                                   9.0, 1e-3, c.out_dev.data_ptr(),
                                   torch.cuda.current_stream().cuda_stream)
    assert rc == glt.GLT_ERR_CAPACITY and b"65536" in glt.glt_last_error()
    trk.close()


def test_noalloc_matches_the_oracle():
    """The same quantities from the FP64 oracle's linearisation directly."""
    import torch

    import oracle
    import paper_2607_16897_gb300 as glt
    import synth

    c = _Case(torch, oracle, synth)
    p = c.p
    o = oracle.OracleTracker(p.cam.W, p.cam.H, p.cam.K, levels=3)
    o.build_pyramid(0, p.ref)
    o.set_map_points(p.uvd)
    o.build_pyramid(1, p.cur)
    uvd_dev = torch.from_numpy(np.ascontiguousarray(p.uvd, np.float32)).cuda()
    for level in (0, 1):
        want = o.debug_linearize(level, c.T, c.a, c.b, per_sample=False)
        for call in range(2):
            _close(c.call(glt, torch, level, uvd_dev, len(p.uvd)), want, (level, call))


def test_noalloc_at_capacity_and_empty():
    """65536 points (the 500 points of a pair repeated) fill all 512 block
    partials of the static scratch; n = 0 writes zeros without a kernel; a
    normal call after both still matches."""
    import torch

    import oracle
    import paper_2607_16897_gb300 as glt
    import synth

    c = _Case(torch, oracle, synth)
    p = c.p
    reps = -(-MAX_POINTS // len(p.uvd))
    big = np.ascontiguousarray(np.tile(p.uvd, (reps, 1))[:MAX_POINTS], np.float32)
    trk = glt.Tracker(p.cam.W, p.cam.H, p.cam.K, levels=3, max_points=MAX_POINTS)
    trk.build_pyramid(glt.GLT_REF, p.ref)
    trk.set_map_points(big)
    trk.build_pyramid(glt.GLT_CUR, p.cur)
    big_dev = torch.from_numpy(big).cuda()
    want = trk.debug_linearize(0, c.T, c.a, c.b, want_res=False)
    for call in range(2):
        _close(c.call(glt, torch, 0, big_dev, MAX_POINTS), want, ("capacity", call))
    out = c.call(glt, torch, 0, None, 0)
    assert np.array_equal(out, np.zeros(46)), out
    small = torch.from_numpy(np.ascontiguousarray(p.uvd, np.float32)).cuda()
    trk.set_map_points(p.uvd)
    want = trk.debug_linearize(0, c.T, c.a, c.b, want_res=False)
    _close(c.call(glt, torch, 0, small, len(p.uvd)), want, "after empty")
    trk.close()
