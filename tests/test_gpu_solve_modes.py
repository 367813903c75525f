"""The two forms of the tracker's 8x8 solve and SE(3) step
(glt_config.solve): GLT_SOLVE_FP64 (the default: the FP64 L D L^T
factorisation and exponential) and GLT_SOLVE_FP32 (FP32 factors and
exponential increment, FP64 state and composition).  Both match the FP64
oracle within the tolerances, return rotations to FP64 rounding, and take
the FP64 "not positive definite" decision."""
import numpy as np
import pytest

from helpers import A_TOL, B_TOL, I34, ROT_TOL, TRANS_TOL, both_sides, pose_diff

pytestmark = pytest.mark.gpu
MODES = ["fp64", "fp32"]


@pytest.fixture(scope="module")
def glt():
    import paper_2607_16897_gb300 as g
    return g


def check_same(g, o, where=""):
    ang, dt = pose_diff(g["T"], o["T"])
    assert ang <= ROT_TOL and dt <= TRANS_TOL, f"{where}: pose diff {ang:.2e} rad {dt:.2e} m"
    assert abs(g["a"] - o["a"]) <= A_TOL and abs(g["b"] - o["b"]) <= B_TOL, where
    assert g["status"] == o["status"], where


@pytest.mark.parametrize("solve", MODES)
@pytest.mark.parametrize("seed", range(6))
def test_modes_match_oracle_c1(glt, orc, syn, solve, seed):
    p = syn.pair_c1(seed, sigma=2.0)
    trk, o = both_sides(glt, orc, p.cam.W, p.cam.H, p.cam.K, p.ref, p.cur, p.uvd, levels=3, solve=solve)
    g = trk.track_frame(I34)
    check_same(g, o.track_frame(I34), f"{solve} seed {seed}")
    # the final pose is a rotation to FP64 rounding in every mode
    R = g["T"][:, :3]
    assert np.abs(R.T @ R - np.eye(3)).max() < 1e-12, solve
    trk.close()


@pytest.mark.parametrize("solve", MODES)
def test_modes_c2_sequence(glt, orc, syn, solve):
    """640x480, 2000 points, 4 levels, constant-velocity starts along a
    sequence."""
    cam = syn.camera_for(640, 480, 525.0)
    seq = syn.sequence(1, 24, cam, syn.ROOM_LARGE, 0.5, 30.0)
    ref, uvd = syn.reference_points(seq, 0, 2000, 0.5, 8.0)
    trk, o = both_sides(glt, orc, 640, 480, cam.K, ref, seq.frame(1)[0], uvd, levels=4, solve=solve)
    T_prev, T_prev2 = I34, I34
    for k in range(1, 9):
        cur, _ = seq.frame(k)
        trk.build_pyramid(glt.GLT_CUR, cur)
        o.build_pyramid(1, cur)
        M = syn.pose_mul(T_prev, syn.pose_inv(T_prev2))
        T_init = syn.pose_mul(M, T_prev)
        g = trk.track_frame(T_init, (0.0, 0.0))
        check_same(g, o.track_frame(T_init, (0.0, 0.0)), f"{solve} frame {k}")
        T_prev2, T_prev = T_prev, g["T"]
    trk.close()


@pytest.mark.parametrize("solve", MODES)
def test_modes_decide_definiteness_as_fp64(glt, orc, syn, solve):
    p = syn.pair_c1(0, sigma=2.0)
    W, H, K = p.cam.W, p.cam.H, p.cam.K
    flat = np.full_like(p.cur, 100)
    trk, o = both_sides(glt, orc, W, H, K, p.ref, flat, p.uvd, levels=3, solve=solve)
    g = trk.track_frame(I34)
    assert g["status"] & glt.GLT_TRACK_NOT_PD, solve
    check_same(g, o.track_frame(I34), f"{solve} flat")
    trk.close()
    trk, o = both_sides(glt, orc, W, H, K, p.ref, p.cur, p.uvd[:1], levels=3, solve=solve)
    check_same(trk.track_frame(I34), o.track_frame(I34), f"{solve} one point")
    trk.close()


def test_solve_mode_is_checked(glt):
    with pytest.raises(glt.GltError):
        glt.Tracker(320, 240, (256.0, 256.0, 160.0, 120.0), solve=2)
