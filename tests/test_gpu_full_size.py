"""Final-pose parity at the full sizes of the benchmark workloads, through the
C ABI: the 1280x720 stream (f 1050, 8000 map points, 5 levels, 1 m/s and
60 deg/s) in FP32 and in mixed precision, and a 640x480 stream of the learned
proposal's workload (2000 points, 5 levels, motion up to 2 m/s, 90 deg/s).
Each frame starts from the constant-velocity state of the frames before it
(affine pair carried over), and the GPU and the FP64 oracle solve from that
same start: pose within 1e-5 rad and 1e-5 m, a within 1e-5, b within 1e-3."""
import numpy as np
import pytest

from helpers import (A_TOL, B_TOL, I34, ROT_TOL, TRANS_TOL, both_sides, compare_linearization,
                     pose_diff)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def glt():
    import paper_2607_16897_gb300 as g
    return g


def _run_sequence(glt, orc, syn, seq, N, L, frames, precision, truth_tol):
    ref, uvd = syn.reference_points(seq, 0, N, 0.5, 8.0)
    cam = seq.cam
    trk, o = both_sides(glt, orc, cam.W, cam.H, cam.K, ref, seq.frame(1)[0], uvd, levels=L,
                        precision=precision, max_points=N)
    T_prev, T_prev2, ab = I34, I34, (0.0, 0.0)
    worst = (0.0, 0.0)
    for k in range(1, frames + 1):
        cur, _ = seq.frame(k)
        trk.build_pyramid(glt.GLT_CUR, cur)
        o.build_pyramid(1, cur)
        M = syn.pose_mul(T_prev, syn.pose_inv(T_prev2))
        T_init = syn.pose_mul(M, T_prev)
        if k == 1:
            # the linearisation itself at the start state, finest and coarsest level
            for level in (0, L - 1):
                compare_linearization(trk.debug_linearize(level, T_init, *ab),
                                      o.debug_linearize(level, T_init, *ab),
                                      f"{precision} level {level}")
        g = trk.track_frame(T_init, ab)
        r = o.track_frame(T_init, ab)
        ang, dt = pose_diff(g["T"], r["T"])
        assert ang <= ROT_TOL and dt <= TRANS_TOL, f"frame {k}: {ang:.2e} rad {dt:.2e} m"
        assert abs(g["a"] - r["a"]) <= A_TOL and abs(g["b"] - r["b"]) <= B_TOL, k
        assert g["status"] == r["status"] == 0, k
        worst = (max(worst[0], ang), max(worst[1], dt))
        ta, tt = pose_diff(g["T"], syn.relative(seq.T_wc[0], seq.T_wc[k]))
        assert ta < truth_tol[0] and tt < truth_tol[1], (k, ta, tt)
        T_prev2, T_prev, ab = T_prev, g["T"], (g["a"], g["b"])
    trk.close()
    return worst


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_full_size_1280x720_8000_points(glt, orc, syn, precision):
    cam = syn.camera_for(1280, 720, 1050.0)
    seq = syn.sequence(2000, 300, cam, syn.ROOM_LARGE, 1.0, 60.0)
    _run_sequence(glt, orc, syn, seq, 8000, 5, 8, precision, (np.deg2rad(0.1), 5e-3))


def test_full_size_640x480_fast_motion(glt, orc, syn):
    from synth.jobs import stream_motion
    speed, ang = stream_motion(5000)
    cam = syn.camera_for(640, 480, 525.0)
    seq = syn.sequence(5000, 24, cam, syn.ROOM_LARGE, speed, ang)
    _run_sequence(glt, orc, syn, seq, 2000, 5, 8, "fp32", (np.deg2rad(0.2), 1e-2))
