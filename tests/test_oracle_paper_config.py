"""Pins of the oracle's paper-configuration options: the p x p patches of
Sec. IV-A / Sec. V (7 x 7 and 11 x 11) instead of the 8-pixel pattern, and a
solve that keeps the affine pair fixed (the paper estimates no affine
brightness), run as plain Gauss-Newton with a fixed number of iterations per
level (no damping, no Huber weights, no early stop).

Independent checks: exact patch values on affine ramps (bilinear
interpolation is exact there), Jacobians against central finite differences
of the residual with the pose perturbed through scipy's expm, known-pose
recovery on rendered pairs, the exact fixed affine pair, the iteration counts
of the fixed schedule, and the pattern layout written out by hand."""
import numpy as np
import pytest

expm = pytest.importorskip("scipy.linalg").expm
I34 = np.hstack([np.eye(3), np.zeros((3, 1))])
GN_FIXED = dict(lambda0=0.0, accept_step=1e30, eps_step=0.0, eps_step_coarse=0.0, huber_k=1e30)


def twist(xi):
    v, w = xi[:3], xi[3:]
    M = np.zeros((4, 4))
    M[:3, :3] = [[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]]
    M[:3, 3] = v
    return expm(M)


def test_pattern_layout(orc):
    dx, dy = orc.pattern_offsets(0)
    assert list(zip(dx, dy)) == [(0, 0), (-2, 0), (2, 0), (0, -2), (0, 2), (-1, -1), (1, -1), (-1, 1)]
    dx, dy = orc.pattern_offsets(7)
    assert len(dx) == 49
    assert list(zip(dx[:8], dy[:8])) == [(-3, -3), (-2, -3), (-1, -3), (0, -3), (1, -3), (2, -3), (3, -3), (-3, -2)]
    assert (dx[24], dy[24]) == (0, 0)
    assert len(orc.pattern_offsets(11)[0]) == 121
    for bad in (1, 4, 13):
        with pytest.raises(ValueError):
            orc.pattern_offsets(bad)


@pytest.mark.parametrize("p", [7, 11])
def test_square_patch_exact_on_ramp(orc, p):
    W, H = 160, 120
    y, x = np.mgrid[0:H, 0:W]
    img = 0.7 * x - 1.3 * y + 100.0
    rng = np.random.default_rng(p)
    uvd = np.stack([rng.uniform(0, W, 40), rng.uniform(0, H, 40), rng.uniform(1, 3, 40)], 1).astype(np.float32)
    I0, valid = orc.ref_patch(img, 0, uvd, pattern=p)
    I8, valid8 = orc.ref_patch(img, 0, uvd, pattern=0)
    dx, dy = orc.pattern_offsets(p)
    h = (p - 1) // 2
    for i in range(40):
        u, v = float(uvd[i, 0]), float(uvd[i, 1])
        inside = u - h >= 1 and u + h < W - 2 and v - h >= 1 and v + h < H - 2
        assert bool(valid[i]) == inside
        if inside:
            np.testing.assert_allclose(I0[i], 0.7 * (u + dx) - 1.3 * (v + dy) + 100.0, atol=1e-9)
    assert not np.any(valid & ~valid8)        # a bigger patch is never valid where the 8-pixel one is not


def test_square_patch_jacobians_on_a_ramp(orc):
    """On affine-ramp images (interpolated central differences are the exact
    derivative there): the forward rows of a 7 x 7 patch equal central
    differences of the residual (pose perturbed through scipy's expm), and the
    IC rows equal the forward rows evaluated on the reference at the identity."""
    K0 = (300.0, 310.0, 160.5, 119.25)
    W, H = 320, 240
    y, x = np.mgrid[0:H, 0:W]
    ref = 0.7 * x - 1.3 * y + 100.0
    cur = 0.6 * x - 1.1 * y + 90.0
    rng = np.random.default_rng(7)
    N = 30
    uvd = np.stack([rng.uniform(30, 290, N), rng.uniform(30, 210, N), rng.uniform(1, 4, N)], 1).astype(np.float32)
    x_r = orc.backproject(K0, uvd)
    I0, valid = orc.ref_patch(ref, 0, uvd, pattern=7)
    T = orc.se3_exp([0.004, -0.003, 0.002, 0.002, -0.001, 0.0015])
    o = orc.linearize(cur, K0, 0, x_r, I0, valid, T, 0.0, 0.0, per_sample=True, pattern=7)
    ok = o["point_valid"]
    assert ok.sum() > 20 and o["J"].shape[1] == 49
    M = np.eye(4)
    M[:3] = T
    eps = 1e-6
    for c in range(6):
        d = np.zeros(6)
        d[c] = eps
        rp = orc.linearize(cur, K0, 0, x_r, I0, valid, (M @ twist(d))[:3], 0.0, 0.0, pattern=7)["res"]
        rm = orc.linearize(cur, K0, 0, x_r, I0, valid, (M @ twist(-d))[:3], 0.0, 0.0, pattern=7)["res"]
        fd = (rp - rm) / (2 * eps)
        np.testing.assert_allclose(o["J"][ok][:, :, c], fd[ok], rtol=1e-5, atol=1e-4)
    Jic = orc.ic_jacobian(ref, K0, 0, x_r, uvd, valid, pattern=7)
    at_ref = orc.linearize(ref, K0, 0, x_r, I0, valid, I34, 0.0, 0.0, per_sample=True, pattern=7)
    np.testing.assert_allclose(Jic[ok], at_ref["J"][ok][:, :, :6], rtol=1e-12, atol=1e-9)


@pytest.mark.parametrize("jacobian", ["forward", "ic"])
@pytest.mark.parametrize("p", [7, 11])
def test_paper_configuration_recovers_pose(orc, syn, jacobian, p):
    """p x p patches, no affine, no Huber, plain GN with 10 iterations on each
    of 3 levels: a noise-free pair without exposure change is recovered, every
    level runs exactly its iteration count, and (a, b) stay at their start."""
    pair = syn.pair_c1(3, sigma=0.0, a=0.0, b=0.0)
    tr = orc.OracleTracker(pair.cam.W, pair.cam.H, pair.cam.K, levels=3, pattern=p,
                           jacobian=jacobian, affine=False, **GN_FIXED)
    tr.build_pyramid(0, pair.ref)
    tr.set_map_points(pair.uvd)
    tr.build_pyramid(1, pair.cur)
    res = tr.track_frame(I34, (0.0, 0.0))
    assert res["iters"] == [10, 10, 10]
    assert res["a"] == 0.0 and res["b"] == 0.0
    rot = np.rad2deg(syn.rotation_angle(res["T"][:, :3].T @ pair.T_cr[:, :3]))
    trans = 1000 * np.linalg.norm(res["T"][:, 3] - pair.T_cr[:, 3])
    assert rot < 0.02 and trans < 1.0, (rot, trans)


def test_fixed_affine_keeps_the_initial_pair(orc, syn):
    pair = syn.pair_c1(5, sigma=2.0)
    tr = orc.OracleTracker(pair.cam.W, pair.cam.H, pair.cam.K, levels=3, affine=False)
    tr.build_pyramid(0, pair.ref)
    tr.set_map_points(pair.uvd)
    tr.build_pyramid(1, pair.cur)
    res = tr.track_frame(I34, (0.05, 3.0))    # the pair's true exposure change, held fixed
    assert res["a"] == 0.05 and res["b"] == 3.0
    full = orc.OracleTracker(pair.cam.W, pair.cam.H, pair.cam.K, levels=3)
    full.build_pyramid(0, pair.ref)
    full.set_map_points(pair.uvd)
    full.build_pyramid(1, pair.cur)
    r2 = full.track_frame(I34)
    assert np.linalg.norm(res["T"][:, 3] - r2["T"][:, 3]) < 1e-3
