"""Pins of the oracle's inverse-compositional mode (Sec. IV-B: the Jacobian
J_ik = grad I0(u_i^0 + du_k) dpi/dx dx/ddelta evaluated on the reference side
with x = T0 P_i, cached per reference; T <- T exp(delta) after each solve).

Independent checks:
  * on an affine-ramp reference image the cached rows are the exact
    derivative of the interpolated template under a reference-side motion
    exp(delta) x_r, by central finite differences through scipy's expm;
  * with the current frame equal to the reference and T = I the cached rows
    equal the forward rows (same image, same point), which the forward pins
    fix independently;
  * known-pose recovery on rendered pairs, agreement with the forward solve
    at convergence, and a planted sign error in the cache that must fail.
"""
import numpy as np
import pytest

expm = pytest.importorskip("scipy.linalg").expm

PAT = np.array([[0, 0], [-2, 0], [2, 0], [0, -2], [0, 2], [-1, -1], [1, -1], [-1, 1]])
I34 = np.hstack([np.eye(3), np.zeros((3, 1))])


def twist(xi):
    v, w = xi[:3], xi[3:]
    M = np.zeros((4, 4))
    M[:3, :3] = [[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]]
    M[:3, 3] = v
    return expm(M)


@pytest.mark.parametrize("level", [0, 1, 2])
def test_ic_rows_are_the_template_derivative_on_a_ramp(orc, level):
    """On I0 = al x + be y + ga (bilinear interpolation and central
    differences exact), d/d delta I0(pi_l(exp(delta) x_r) + du_k) at 0
    equals the cached row, by central differences of the closed form."""
    K0 = (300.0, 310.0, 160.5, 119.25)
    W, H = 320 >> level, 240 >> level
    al, be, ga = 0.7, -1.3, 100.0
    y, x = np.mgrid[0:H, 0:W]
    img = al * x + be * y + ga
    rng = np.random.default_rng(level)
    N = 12
    uvd = np.stack([rng.uniform(20, 300, N), rng.uniform(20, 220, N), rng.uniform(1, 4, N)], 1)
    uvd = uvd.astype(np.float32)
    x_r = orc.backproject(K0, uvd)
    valid = np.ones(N, np.uint8)
    J = orc.ic_jacobian(img, K0, level, x_r, uvd, valid)
    s = 2.0 ** -level
    fx, fy, cx, cy = (k * s for k in K0)

    def template(X, k):
        u = fx * X[0] / X[2] + cx + PAT[k, 0]
        v = fy * X[1] / X[2] + cy + PAT[k, 1]
        return al * u + be * v + ga

    eps = 1e-6
    for i in range(N):
        Xh = np.append(x_r[i], 1.0)
        for c in range(6):
            d = np.zeros(6)
            d[c] = eps
            Xp = (twist(d) @ Xh)[:3]
            Xm = (twist(-d) @ Xh)[:3]
            for k in range(8):
                fd = (template(Xp, k) - template(Xm, k)) / (2 * eps)
                assert abs(fd - J[i, k, c]) <= 1e-5 * max(1.0, abs(fd)), (i, k, c, fd, J[i, k, c])


def test_ic_rows_equal_forward_rows_on_the_reference_at_identity(orc, syn):
    p = syn.pair_c1(4, sigma=2.0)
    tr = orc.OracleTracker(p.cam.W, p.cam.H, p.cam.K, levels=3, jacobian="ic")
    tr.build_pyramid(0, p.ref)
    tr.set_map_points(p.uvd)
    tr.build_pyramid(1, p.ref)          # current frame = reference
    for level in range(3):
        fwd = orc.linearize(tr.pyr[1][level], p.cam.K, level, tr.x_r, tr.I0[level],
                            tr.valid[level], I34, 0.0, 0.0, per_sample=True)
        ic = tr.debug_linearize(level, I34, 0.0, 0.0)
        ok = fwd["point_valid"]
        assert ok.sum() > 100
        np.testing.assert_allclose(ic["J"][ok][:, :, :6], fwd["J"][ok][:, :, :6], rtol=1e-10, atol=1e-9)
        np.testing.assert_allclose(tr.Jic[level][ok], fwd["J"][ok][:, :, :6], rtol=1e-10, atol=1e-9)
        # at a = 0.2 the pose columns scale with e^a, the affine ones are unchanged
        ic2 = tr.debug_linearize(level, I34, 0.2, 1.0)
        np.testing.assert_allclose(ic2["J"][ok][:, :, :6], np.exp(0.2) * ic["J"][ok][:, :, :6],
                                   rtol=1e-12, atol=1e-12)


def pose_err(syn, T, Tt):
    return (np.rad2deg(syn.rotation_angle(T[:, :3].T @ Tt[:, :3])),
            1000.0 * np.linalg.norm(T[:, 3] - Tt[:, 3]))


def ic_tracker(orc, p, **cfg):
    tr = orc.OracleTracker(p.cam.W, p.cam.H, p.cam.K, levels=3, jacobian="ic", **cfg)
    tr.build_pyramid(0, p.ref)
    tr.set_map_points(p.uvd)
    tr.build_pyramid(1, p.cur)
    return tr


@pytest.mark.parametrize("seed", range(4))
def test_ic_recovers_known_pose_noise_free(orc, syn, seed):
    p = syn.pair_c1(seed, sigma=0.0)
    res = ic_tracker(orc, p).track_frame(I34)
    rot, trans = pose_err(syn, res["T"], p.T_cr)
    assert res["status"] == 0
    assert rot < 0.01 and trans < 0.5, (rot, trans)


def test_ic_agrees_with_forward_at_convergence(orc, syn):
    """Both solves estimate the same pose; with noise their fixed points
    (J_ic^T W r = 0 and J_fwd^T W r = 0) differ by far less than the error
    against the truth."""
    for seed in range(3):
        p = syn.pair_c1(20 + seed, sigma=2.0)
        ic = ic_tracker(orc, p).track_frame(I34)
        fw = orc.OracleTracker(p.cam.W, p.cam.H, p.cam.K, levels=3)
        fw.build_pyramid(0, p.ref)
        fw.set_map_points(p.uvd)
        fw.build_pyramid(1, p.cur)
        f = fw.track_frame(I34)
        rot, trans = pose_err(syn, ic["T"], f["T"])
        assert rot < 0.01 and trans < 0.3, (seed, rot, trans)
        rot_t, trans_t = pose_err(syn, ic["T"], p.T_cr)
        assert rot_t < 0.05 and trans_t < 2.0


def test_ic_with_a_flipped_cache_fails(orc, syn):
    """A sign error in the cached rows (the reference-side increment composed
    the wrong way round) walks away from the solution."""
    p = syn.pair_c1(1, sigma=2.0)
    tr = ic_tracker(orc, p)
    good = tr.track_frame(I34)
    tr.Jic = -tr.Jic
    bad = tr.track_frame(I34)
    _, trans_good = pose_err(syn, good["T"], p.T_cr)
    _, trans_bad = pose_err(syn, bad["T"], p.T_cr)
    assert trans_good < 2.0 and trans_bad > 10.0, (trans_good, trans_bad)
