"""Pins of the oracle's reference patches and linearisation (Sec. IV-A Eqs. 1-5
with the affine brightness and Huber weights this library adds).

Independent checks used here:
  * affine-ramp images, on which bilinear interpolation and central
    differences are exact, so residuals and Jacobians have closed forms;
  * central finite differences of the residual / energy, with the pose
    perturbed through scipy's matrix exponential (not the oracle's);
  * a dense stacked Jacobian multiplied out with numpy (J^T W J, J^T W r);
  * identical frames, which must give zero residuals and zero gradient.
"""
import numpy as np
import pytest

expm = pytest.importorskip("scipy.linalg").expm

PAT = np.array([[0, 0], [-2, 0], [2, 0], [0, -2], [0, 2], [-1, -1], [1, -1], [-1, 1]])


def ramp(W, H, al, be, ga):
    y, x = np.mgrid[0:H, 0:W]
    return al * x + be * y + ga


def twist_matrix(xi):
    v, w = xi[:3], xi[3:]
    M = np.zeros((4, 4))
    M[:3, :3] = [[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]]
    M[:3, 3] = v
    return M


def perturb(T, xi):
    """T exp(xi) via scipy's matrix exponential."""
    M = np.eye(4)
    M[:3, :] = T
    return (M @ expm(twist_matrix(xi)))[:3, :]


def random_points(rng, N, W, H, K, dmin=1.0, dmax=4.0, border=12):
    u = rng.uniform(border, W - border, N)
    v = rng.uniform(border, H - border, N)
    d = rng.uniform(dmin, dmax, N)
    return np.stack([u, v, d], 1).astype(np.float32)


def small_pose(rng, rot=0.01, trans=0.02):
    return perturb(np.hstack([np.eye(3), np.zeros((3, 1))]),
                   np.concatenate([rng.normal(size=3) * trans, rng.normal(size=3) * rot]))


K0 = (300.0, 310.0, 160.5, 119.25)
W0, H0 = 320, 240


@pytest.mark.parametrize("level", [0, 1, 2])
def test_ref_patch_is_exact_on_ramp(orc, level):
    rng = np.random.default_rng(level)
    W, H = W0 >> level, H0 >> level
    img = ramp(W, H, 0.7, -1.3, 100.0)
    uvd = random_points(rng, 200, W0, H0, K0)
    I0, valid = orc.ref_patch(img, level, uvd)
    s = 2.0 ** -level
    for i in range(len(uvd)):
        u, v = uvd[i, 0] * s, uvd[i, 1] * s
        inside = all(1 <= u + dx < W - 2 and 1 <= v + dy < H - 2 for dx, dy in PAT)
        assert bool(valid[i]) == inside
        if inside:
            exp = 0.7 * (u + PAT[:, 0]) - 1.3 * (v + PAT[:, 1]) + 100.0
            np.testing.assert_allclose(I0[i], exp, atol=1e-10)


def test_backproject_reprojects(orc):
    rng = np.random.default_rng(1)
    uvd = random_points(rng, 50, W0, H0, K0)
    x = orc.backproject(K0, uvd)
    fx, fy, cx, cy = K0
    np.testing.assert_allclose(fx * x[:, 0] / x[:, 2] + cx, uvd[:, 0], atol=1e-9)
    np.testing.assert_allclose(fy * x[:, 1] / x[:, 2] + cy, uvd[:, 1], atol=1e-9)
    np.testing.assert_allclose(x[:, 2], uvd[:, 2])


def _lin_setup(rng, level, N=60, al=1.1, be=-0.6):
    W, H = W0 >> level, H0 >> level
    cur = ramp(W, H, al, be, 90.0)
    uvd = random_points(rng, N, W0, H0, K0, border=40)
    I0 = rng.uniform(40, 160, size=(N, 8))
    valid = np.ones(N, np.uint8)
    return W, H, cur, uvd, I0, valid


@pytest.mark.parametrize("level", [0, 1, 2])
def test_jacobian_matches_finite_differences_on_ramp(orc, level):
    rng = np.random.default_rng(10 + level)
    W, H, cur, uvd, I0, valid = _lin_setup(rng, level)
    x_r = orc.backproject(K0, uvd)
    T = small_pose(rng)
    a, b = 0.04, -2.0
    base = orc.linearize(cur, K0, level, x_r, I0, valid, T, a, b, 9.0)
    pv = base["point_valid"]
    assert pv.sum() >= 30
    J = base["J"][pv]
    eps = 1e-6
    for i in range(8):
        xi = np.zeros(8)
        xi[i] = eps
        Tp, Tm = perturb(T, xi[:6]), perturb(T, -xi[:6])
        rp = orc.linearize(cur, K0, level, x_r, I0, valid, Tp, a + xi[6], b + xi[7], 9.0)
        rm = orc.linearize(cur, K0, level, x_r, I0, valid, Tm, a - xi[6], b - xi[7], 9.0)
        assert (rp["point_valid"] == pv).all() and (rm["point_valid"] == pv).all()
        fd = (rp["res"][pv] - rm["res"][pv]) / (2 * eps)
        scale = np.abs(J[:, :, i]).max() + 1e-12
        np.testing.assert_allclose(J[:, :, i], fd, atol=2e-6 * scale, rtol=0)


def test_affine_columns_and_residual_closed_form(orc):
    rng = np.random.default_rng(3)
    level = 1
    W, H, cur, uvd, I0, valid = _lin_setup(rng, level)
    x_r = orc.backproject(K0, uvd)
    T = small_pose(rng)
    a, b = -0.07, 5.0
    out = orc.linearize(cur, K0, level, x_r, I0, valid, T, a, b, 9.0)
    pv = out["point_valid"]
    s = 0.5
    R, t = T[:, :3], T[:, 3]
    xc = x_r @ R.T + t
    u = K0[0] * s * xc[:, 0] / xc[:, 2] + K0[2] * s
    v = K0[1] * s * xc[:, 1] / xc[:, 2] + K0[3] * s
    Iq = 1.1 * (u[:, None] + PAT[None, :, 0]) - 0.6 * (v[:, None] + PAT[None, :, 1]) + 90.0
    r = Iq - np.exp(a) * I0 - b
    np.testing.assert_allclose(out["res"][pv], r[pv], atol=1e-9)
    np.testing.assert_allclose(out["J"][pv][:, :, 6], -np.exp(a) * I0[pv], atol=1e-9)
    np.testing.assert_allclose(out["J"][pv][:, :, 7], -1.0)
    # Huber weights and energy
    k = 9.0
    ar = np.abs(r[pv])
    np.testing.assert_allclose(out["w"][pv], np.where(ar <= k, 1.0, k / ar), atol=1e-12)
    rho = np.where(ar <= k, 0.5 * r[pv] ** 2, k * ar - 0.5 * k * k)
    np.testing.assert_allclose(out["E"], rho.sum(), rtol=1e-12)
    assert out["n"] == 8 * pv.sum()
    assert (ar > k).any() and (ar <= k).any()


def test_gradient_is_derivative_of_huber_energy(orc):
    """g = J^T W r must equal dE/d(delta) (Huber is C1), checked by central
    differences of the energy on a ramp image."""
    rng = np.random.default_rng(21)
    level = 0
    W, H, cur, uvd, I0, valid = _lin_setup(rng, level, N=80)
    x_r = orc.backproject(K0, uvd)
    T = small_pose(rng)
    a, b = 0.02, 1.0
    base = orc.linearize(cur, K0, level, x_r, I0, valid, T, a, b, 9.0, per_sample=False)
    eps = 1e-6
    for i in range(8):
        xi = np.zeros(8)
        xi[i] = eps
        Ep = orc.linearize(cur, K0, level, x_r, I0, valid, perturb(T, xi[:6]), a + xi[6],
                           b + xi[7], 9.0, per_sample=False)["E"]
        Em = orc.linearize(cur, K0, level, x_r, I0, valid, perturb(T, -xi[:6]), a - xi[6],
                           b - xi[7], 9.0, per_sample=False)["E"]
        fd = (Ep - Em) / (2 * eps)
        assert abs(fd - base["g"][i]) <= 1e-5 * (abs(base["g"][i]) + 1.0)


def test_normal_equations_match_dense_stack(orc, syn):
    p = syn.pair_c1(3, sigma=2.0, N=120)
    tr = orc.OracleTracker(p.cam.W, p.cam.H, p.cam.K, levels=3)
    tr.build_pyramid(0, p.ref)
    tr.set_map_points(p.uvd)
    tr.build_pyramid(1, p.cur)
    rng = np.random.default_rng(0)
    for level in range(3):
        T = small_pose(rng, 0.02, 0.03)
        out = tr.debug_linearize(level, T, 0.03, 2.0)
        pv = out["point_valid"]
        J = out["J"][pv].reshape(-1, 8)
        w = out["w"][pv].reshape(-1)
        r = out["res"][pv].reshape(-1)
        Hb = J.T @ (w[:, None] * J)
        gb = J.T @ (w * r)
        np.testing.assert_allclose(out["H"], Hb, rtol=1e-12, atol=1e-9 * np.abs(Hb).max())
        np.testing.assert_allclose(out["g"], gb, rtol=1e-12, atol=1e-9 * np.abs(gb).max())
        Hm = out["H"]
        np.testing.assert_allclose(Hm, Hm.T, rtol=1e-14, atol=1e-14 * np.abs(Hm).max())
        ev = np.linalg.eigvalsh(Hm)
        assert ev.min() >= -1e-12 * np.abs(ev).max()
        assert out["n"] == 8 * pv.sum()


def test_identical_frames_give_zero_residual(orc, syn):
    p = syn.pair_c1(5, sigma=2.0)
    tr = orc.OracleTracker(p.cam.W, p.cam.H, p.cam.K, levels=3)
    tr.build_pyramid(0, p.ref)
    tr.set_map_points(p.uvd)
    tr.build_pyramid(1, p.ref)
    I = np.hstack([np.eye(3), np.zeros((3, 1))])
    for level in range(3):
        out = tr.debug_linearize(level, I, 0.0, 0.0)
        pv = out["point_valid"]
        assert pv.sum() > 0.8 * len(pv)
        assert np.abs(out["res"][pv]).max() <= 1e-9
        assert np.abs(out["g"]).max() <= 1e-7 * np.abs(out["H"]).max() ** 0.5
    res = tr.track_frame(I)
    np.testing.assert_allclose(res["T"], I, atol=1e-9)
    assert abs(res["a"]) < 1e-9 and abs(res["b"]) < 1e-7


def test_validity_bounds_and_depth(orc):
    # unit intrinsics make u = x/z exact, so samples land exactly on the bounds
    K = (1.0, 1.0, 0.0, 0.0)
    W, H = 40, 30
    img = ramp(W, H, 1.0, 2.0, 10.0)
    # min x sample is u0-2; max x sample u0+2; valid iff 1 <= q < W-2
    us = [3.0, 2.999, W - 4 - 1e-3, W - 4.0]
    uvd = np.array([[u, 15.0, 1.0] for u in us], np.float32)
    x_r = orc.backproject(K, uvd)
    I0 = np.zeros((len(us), 8))
    valid = np.ones(len(us), np.uint8)
    I = np.hstack([np.eye(3), np.zeros((3, 1))])
    out = orc.linearize(img, K, 0, x_r, I0, valid, I, 0.0, 0.0)
    expect = [1 <= np.float32(u) - 2 and np.float32(u) + 2 < W - 2 for u in us]
    assert list(out["point_valid"]) == expect == [True, False, True, False]
    # reference validity mask is honoured
    out2 = orc.linearize(img, K, 0, x_r, I0, np.array([0, 1, 1, 1], np.uint8), I, 0.0, 0.0)
    assert not out2["point_valid"][0]
    # depth below zmin drops the point
    T = I.copy()
    T[2, 3] = -1.0 + 0.5e-3
    out3 = orc.linearize(img, K, 0, x_r, I0, valid, T, 0.0, 0.0, zmin=1e-3)
    assert out3["n"] == 0 and np.isnan(out3["res"]).all()


def test_gradient_sampling_on_quadratic_image(orc):
    """On I = al x^2 + be y^2 + ga x y + c the central differences equal the
    analytic gradient and its bilinear interpolation is exact, so the pose
    columns of J equal grad I(q) times the projection Jacobian, which is taken
    here by finite differences of the pinhole projection through scipy's expm."""
    rng = np.random.default_rng(31)
    level = 1
    W, H = W0 >> level, H0 >> level
    al, be, ga = 0.011, -0.007, 0.004
    y, x = np.mgrid[0:H, 0:W]
    cur = al * x * x + be * y * y + ga * x * y + 50.0
    uvd = random_points(rng, 40, W0, H0, K0, border=40)
    x_r = orc.backproject(K0, uvd)
    I0 = rng.uniform(40, 160, size=(40, 8))
    T = small_pose(rng)
    out = orc.linearize(cur, K0, level, x_r, I0, np.ones(40, np.uint8), T, 0.0, 0.0, 9.0)
    pv = out["point_valid"]
    s = 2.0 ** -level
    fx, fy, cx, cy = (k * s for k in K0)

    def proj(Tm):
        xc = x_r @ Tm[:, :3].T + Tm[:, 3]
        return np.stack([fx * xc[:, 0] / xc[:, 2] + cx, fy * xc[:, 1] / xc[:, 2] + cy], 1)

    uv = proj(T)
    eps = 1e-6
    Jg = np.zeros((len(x_r), 2, 6))
    for i in range(6):
        d = np.zeros(6)
        d[i] = eps
        Jg[:, :, i] = (proj(perturb(T, d)) - proj(perturb(T, -d))) / (2 * eps)
    for k, (dx, dy) in enumerate(PAT):
        qx, qy = uv[:, 0] + dx, uv[:, 1] + dy
        gx = 2 * al * qx + ga * qy
        gy = 2 * be * qy + ga * qx
        exp = gx[:, None] * Jg[:, 0, :] + gy[:, None] * Jg[:, 1, :]
        got = out["J"][:, k, :6]
        np.testing.assert_allclose(got[pv], exp[pv], rtol=1e-6, atol=1e-6 * np.abs(exp).max())
