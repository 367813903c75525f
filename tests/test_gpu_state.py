"""The tracker's state on the GPU path (checkpoint / resume and the
constant-velocity start of Sec. IV-A): glt_track_frame without an initial
state starts from glt_state_predict of the tracker's state and advances it;
every such frame matches the FP64 oracle run from the same start, and a
tracker restored from a checkpoint continues the sequence bit for bit."""
import ctypes

import numpy as np
import pytest

from helpers import A_TOL, B_TOL, I34, ROT_TOL, TRANS_TOL, both_sides, pose_diff

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def glt():
    import paper_2607_16897_gb300 as g
    return g


def predicted(glt, st):
    T = (ctypes.c_double * 12)()
    ab = (ctypes.c_double * 2)()
    assert glt.glt_state_predict(ctypes.byref(st), T, ab) == 0
    return np.array(T[:]).reshape(3, 4), tuple(ab[:])


@pytest.fixture(scope="module")
def sequence(syn):
    cam = syn.camera_for(640, 480, 525.0)
    seq = syn.sequence(3, 12, cam, syn.ROOM_LARGE, 0.5, 30.0)
    ref, uvd = syn.reference_points(seq, 0, 2000, 0.5, 8.0)
    return cam, seq, ref, uvd


def test_state_driven_frames_match_oracle(glt, orc, syn, sequence):
    cam, seq, ref, uvd = sequence
    trk, o = both_sides(glt, orc, 640, 480, cam.K, ref, seq.frame(1)[0], uvd, levels=4)
    st = trk.get_state()
    assert st.frames == 0 and st.reference == 1
    assert np.array_equal(np.array(st.T_cr[:]).reshape(3, 4), I34)
    T_prev, T_prev2 = I34, I34
    for k in range(1, 7):
        cur, _ = seq.frame(k)
        trk.build_pyramid(glt.GLT_CUR, cur)
        o.build_pyramid(1, cur)
        T0, ab0 = predicted(glt, trk.get_state())
        # the prediction is the constant-velocity model T_k = M T_{k-1}
        M = syn.pose_mul(T_prev, syn.pose_inv(T_prev2))
        assert np.abs(T0 - syn.pose_mul(M, T_prev)).max() < 1e-12
        g = trk.track_frame()
        r = o.track_frame(T0, ab0)
        ang, dt = pose_diff(g["T"], r["T"])
        assert ang <= ROT_TOL and dt <= TRANS_TOL, (k, ang, dt)
        assert abs(g["a"] - r["a"]) <= A_TOL and abs(g["b"] - r["b"]) <= B_TOL
        st = trk.get_state()
        assert st.frames == k and np.array_equal(np.array(st.T_cr[:]).reshape(3, 4), g["T"])
        assert (st.a, st.b) == (g["a"], g["b"])
        T_prev2, T_prev = T_prev, g["T"]
        ang, dt = pose_diff(g["T"], syn.relative(seq.T_wc[0], seq.T_wc[k]))
        assert ang < np.deg2rad(0.1) and dt < 5e-3, (k, ang, dt)
    # a new reference restarts the pose and keeps the motion
    motion = np.array(st.motion[:])
    trk.set_map_points(uvd[:1000])
    st = trk.get_state()
    assert st.reference == 2 and st.frames == 0 and (st.a, st.b) == (0.0, 0.0)
    assert np.array_equal(np.array(st.T_cr[:]).reshape(3, 4), I34)
    assert np.array_equal(np.array(st.motion[:]), motion)
    trk.close()


def test_resume_from_a_checkpoint(glt, orc, syn, sequence):
    cam, seq, ref, uvd = sequence
    frames = [seq.frame(k)[0] for k in range(1, 9)]
    a, _ = both_sides(glt, orc, 640, 480, cam.K, ref, frames[0], uvd, levels=4)
    res, ck = [], None
    for k, cur in enumerate(frames):
        if k == 4:
            ck = a.get_state()
        a.build_pyramid(glt.GLT_CUR, cur)
        res.append(a.track_frame())
    # a second tracker with the same reference, restored from the checkpoint
    b, _ = both_sides(glt, orc, 640, 480, cam.K, ref, frames[0], uvd, levels=4)
    b.set_map_points(uvd)                       # another map-point version than a's
    b.set_state(ck)
    assert b.get_state().reference == 2 and b.get_state().frames == 4
    for k in range(4, 8):
        b.build_pyramid(glt.GLT_CUR, frames[k])
        g = b.track_frame()
        assert np.array_equal(g["T"], res[k]["T"]) and g["passes"] == res[k]["passes"], k
        assert (g["a"], g["b"]) == (res[k]["a"], res[k]["b"])
    bad = b.get_state()
    bad.frames = -1
    with pytest.raises(glt.GltError):
        b.set_state(bad)
    bad.frames = 0
    bad.motion[3] = float("inf")
    with pytest.raises(glt.GltError):
        b.set_state(bad)
    a.close()
    b.close()
