"""Checks of the seeded input generator (not of the method)."""
import numpy as np


def test_render_is_deterministic_and_seeded(syn):
    cam = syn.camera_for(160, 120, 128)
    T = syn.pose(np.eye(3), np.zeros(3))
    a1, d1 = syn.render(syn.ROOM_SMALL, T, cam, 0.05, 3.0, 2.0, noise_seed=5)
    a2, d2 = syn.render(syn.ROOM_SMALL, T, cam, 0.05, 3.0, 2.0, noise_seed=5)
    a3, _ = syn.render(syn.ROOM_SMALL, T, cam, 0.05, 3.0, 2.0, noise_seed=6)
    np.testing.assert_array_equal(a1, a2)
    np.testing.assert_array_equal(d1, d2)
    assert (a1 != a3).mean() > 0.3
    # noise statistics: sigma = 2 around the noise-free radiance
    _, _, rad = syn.render(syn.ROOM_SMALL, T, cam, 0.05, 3.0, 0.0, want_rad=True)
    diff = a1.astype(np.float64) - rad
    assert abs(diff.mean()) < 0.1 and 1.8 < diff.std() < 2.3


def test_depth_is_camera_z_and_consistent_across_views(syn):
    p = syn.pair_c1(0, sigma=0.0, N=50)
    fx, fy, cx, cy = p.cam.K
    u, v, d = p.uvd[:, 0].astype(float), p.uvd[:, 1].astype(float), p.uvd[:, 2].astype(float)
    x_r = np.stack([d * (u - cx) / fx, d * (v - cy) / fy, d], 1)
    xc = x_r @ p.T_cr[:, :3].T + p.T_cr[:, 3]
    T_wc_cur = syn.pose_mul(syn.pose(np.eye(3), np.zeros(3)), syn.pose_inv(p.T_cr))
    for i in range(10):
        uc = fx * xc[i, 0] / xc[i, 2] + cx
        vc = fy * xc[i, 1] / xc[i, 2] + cy
        assert abs(syn.depth_at(syn.ROOM_SMALL, T_wc_cur, p.cam, uc, vc) - xc[i, 2]) < 1e-5


def test_point_selection(syn):
    p = syn.pair_c1(1, sigma=2.0, N=500)
    assert p.uvd.shape == (500, 3)
    assert (p.uvd[:, 2] >= 1.0).all() and (p.uvd[:, 2] <= 5.0).all()
    assert len({(round(u), round(v)) for u, v in p.uvd[:, :2]}) == 500


def test_sequence_speeds(syn):
    cam = syn.camera_for(160, 120, 131.25)
    seq = syn.sequence(1, 120, cam, syn.ROOM_LARGE, 0.5, 30.0)
    pos = seq.T_wc[:, :, 3]
    speed = np.linalg.norm(np.diff(pos, axis=0), axis=1).mean() * 30
    assert 0.3 < speed <= 0.5 + 1e-9
    lo, hi = np.array(syn.ROOM_LARGE.lo), np.array(syn.ROOM_LARGE.hi)
    assert (pos > lo + 0.99).all() and (pos < hi - 0.99).all()
    assert (np.abs(seq.a) <= 0.1 + 1e-12).all() and (np.abs(seq.b) <= 10 + 1e-9).all()
