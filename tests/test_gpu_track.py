"""Full coarse-to-fine track on the GPU vs the FP64 oracle on the same inputs:
final pose within 1e-5 rad and 1e-5 m, a within 1e-5, b within 1e-3 gray."""
import numpy as np
import pytest

from helpers import (A_TOL, B_TOL, I34, ROT_TOL, TRANS_TOL, both_sides, pose_diff)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def glt():
    import paper_2607_16897_gb300 as g
    return g


def check_same(g, o, where=""):
    ang, dt = pose_diff(g["T"], o["T"])
    assert ang <= ROT_TOL and dt <= TRANS_TOL, f"{where}: pose diff {ang:.2e} rad {dt:.2e} m"
    assert abs(g["a"] - o["a"]) <= A_TOL, f"{where}: a {g['a']} vs {o['a']}"
    assert abs(g["b"] - o["b"]) <= B_TOL, f"{where}: b {g['b']} vs {o['b']}"
    assert g["status"] == o["status"], where
    return ang, dt


@pytest.mark.parametrize("seed", range(20))
def test_track_c1_matches_oracle(glt, orc, syn, seed):
    p = syn.pair_c1(seed, sigma=2.0)
    trk, o = both_sides(glt, orc, p.cam.W, p.cam.H, p.cam.K, p.ref, p.cur, p.uvd, levels=3)
    g = trk.track_frame(I34)
    r = o.track_frame(I34)
    check_same(g, r, f"seed {seed}")
    # both recover the true motion (2 deg, 3 cm) to the oracle's accuracy
    ang, dt = pose_diff(g["T"], p.T_cr)
    assert ang < np.deg2rad(0.05) and dt < 2e-3
    # the GPU's pass trace follows the same level schedule
    tr = trk.get_trace()
    assert len(tr) == g["passes"]
    assert [e["level"] for e in tr if not e["candidate"]] == [2, 1, 0]
    trk.close()


@pytest.mark.parametrize("cluster,threads", [(1, 128), (1, 256), (2, 128), (3, 256), (4, 256),
                                             (8, 128), (16, 128), (2, 512)])
def test_track_any_cluster_shape(glt, orc, syn, cluster, threads):
    p = syn.pair_c1(7, sigma=2.0)
    trk, o = both_sides(glt, orc, p.cam.W, p.cam.H, p.cam.K, p.ref, p.cur, p.uvd, levels=3,
                        cluster=cluster, threads=threads)
    check_same(trk.track_frame(I34), o.track_frame(I34), f"shape {cluster}x{threads}")
    trk.close()


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_track_c2_sequence_frames(glt, orc, syn, precision):
    """Config-2 geometry: 640x480, 2000 points, 4 levels, constant-velocity
    init along a sequence; every frame checked against the oracle with the
    same initial state."""
    cam = syn.camera_for(640, 480, 525.0)
    seq = syn.sequence(1, 24, cam, syn.ROOM_LARGE, 0.5, 30.0)
    ref, uvd = syn.reference_points(seq, 0, 2000, 0.5, 8.0)
    trk, o = both_sides(glt, orc, 640, 480, cam.K, ref, seq.frame(1)[0], uvd, levels=4,
                        precision=precision)
    T_prev, T_prev2 = I34, I34
    for k in range(1, 9):
        cur, _ = seq.frame(k)
        trk.build_pyramid(glt.GLT_CUR, cur)
        o.build_pyramid(1, cur)
        # constant velocity: T_k = M T_{k-1}, M = T_{k-1} T_{k-2}^-1
        M = syn.pose_mul(T_prev, syn.pose_inv(T_prev2))
        T_init = syn.pose_mul(M, T_prev)
        g = trk.track_frame(T_init, (0.0, 0.0))
        r = o.track_frame(T_init, (0.0, 0.0))
        check_same(g, r, f"frame {k}")
        T_prev2, T_prev = T_prev, g["T"]
        ang, dt = pose_diff(g["T"], syn.relative(seq.T_wc[0], seq.T_wc[k]))
        assert ang < np.deg2rad(0.1) and dt < 5e-3, (k, ang, dt)
    trk.close()


def test_track_degenerate_cases(glt, orc, syn):
    p = syn.pair_c1(0, sigma=2.0)
    W, H, K = p.cam.W, p.cam.H, p.cam.K
    # no map points at all
    trk, o = both_sides(glt, orc, W, H, K, p.ref, p.cur, p.uvd[:0], levels=3, max_points=8)
    g = trk.track_frame(I34)
    assert g["status"] & glt.GLT_TRACK_TOO_FEW_POINTS and np.array_equal(g["T"], I34)
    check_same(g, o.track_frame(I34))
    trk.close()
    # one point: fewer samples than min_valid on every level
    trk, o = both_sides(glt, orc, W, H, K, p.ref, p.cur, p.uvd[:1], levels=3)
    check_same(trk.track_frame(I34), o.track_frame(I34), "one point")
    trk.close()
    # textureless current frame: H singular -> not positive definite
    flat = np.full_like(p.cur, 100)
    trk, o = both_sides(glt, orc, W, H, K, p.ref, flat, p.uvd, levels=3)
    g = trk.track_frame(I34)
    assert g["status"] & glt.GLT_TRACK_NOT_PD
    check_same(g, o.track_frame(I34), "flat")
    trk.close()
    # no iterations: state unchanged, no passes
    trk, o = both_sides(glt, orc, W, H, K, p.ref, p.cur, p.uvd, levels=3, max_iters=[0] * 8)
    T0 = orc.se3_exp([0.01, 0.0, 0.0, 0.0, 0.02, 0.0])
    g = trk.track_frame(T0, (0.1, 2.0))
    assert np.array_equal(g["T"], T0) and g["passes"] == 0 and np.isnan(g["cost"])
    trk.close()
    # only the finest level iterates
    trk, o = both_sides(glt, orc, W, H, K, p.ref, p.cur, p.uvd, levels=3, max_iters=[10, 0, 0])
    check_same(trk.track_frame(I34), o.track_frame(I34), "level 0 only")
    # non-finite initial state is rejected on the host
    bad = I34.copy()
    bad[0, 0] = np.nan
    with pytest.raises(glt.GltError):
        trk.track_frame(bad)
    trk.close()


def test_track_capacity_and_reuse(glt, orc, syn):
    p = syn.pair_c1(11, sigma=2.0, N=500)
    trk, o = both_sides(glt, orc, p.cam.W, p.cam.H, p.cam.K, p.ref, p.cur, p.uvd, levels=3,
                        max_points=500)
    with pytest.raises(glt.GltError):
        trk.set_map_points(np.zeros((501, 3), np.float32))
    g1 = trk.track_frame(I34)
    g2 = trk.track_frame(I34)
    assert np.array_equal(g1["T"], g2["T"]) and g1["passes"] == g2["passes"]  # deterministic
    # fewer points on the same tracker
    trk.set_map_points(p.uvd[:200])
    o.set_map_points(p.uvd[:200])
    check_same(trk.track_frame(I34), o.track_frame(I34), "200 points")
    trk.close()


def test_track_async_device_io(glt, orc, syn):
    import torch
    p = syn.pair_c1(12, sigma=2.0)
    trk, o = both_sides(glt, orc, p.cam.W, p.cam.H, p.cam.K, p.ref, p.cur, p.uvd, levels=3,
                        device_inputs=True)
    init = torch.tensor(np.concatenate([I34.ravel(), [0.0, 0.0]]), dtype=torch.float64).cuda()
    out = torch.zeros(glt.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    trk.track_frame_async(init, out)
    torch.cuda.synchronize()
    g = glt.parse_results(out)[0]
    check_same(g, o.track_frame(I34), "async")
    trk.close()


def test_pass_floor_is_below_a_real_pass(glt, orc, syn):
    """The latency floor of a pass (no points) is positive and below the mean
    pass time of a real solve on the same shape; the cached-Hessian tail
    (a matrix-vector product) is cheaper than the factorisation."""
    import torch
    p = syn.pair_c1(1, sigma=2.0)
    trk, _ = both_sides(glt, orc, p.cam.W, p.cam.H, p.cam.K, p.ref, p.cur, p.uvd, levels=3,
                        cluster=4, threads=256)
    trk.track_frame(I34)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    g = trk.track_frame(I34)
    e1.record()
    torch.cuda.synchronize()
    per_pass = 1000.0 * e0.elapsed_time(e1) / g["passes"]
    floor = glt.pass_floor(4, 256)
    assert 0.5 < floor < per_pass, (floor, per_pass)
    assert glt.pass_floor(4, 512, cached=True) < glt.pass_floor(4, 512)
    # the FP32 solve's tail is shorter than the FP64 one
    assert glt.pass_floor(4, 256, solve="fp32") < floor
    with pytest.raises(glt.GltError):
        glt.pass_floor(4, 256, cached=True)       # the cached-Hessian kernel runs 512 threads
    with pytest.raises(glt.GltError):
        glt.pass_floor(4, 256, solve=2)
    trk.close()
