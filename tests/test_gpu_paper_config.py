"""The paper's configuration on the GPU against the oracle: p x p patches (7 x 7
and 11 x 11, Sec. IV-A / V) in the forward and inverse-compositional forms, the
affine pair held fixed, plain Gauss-Newton with a fixed number of iterations
per level, 6 levels.  Same tolerances as the 8-pixel form."""
import numpy as np
import pytest

from helpers import I34, ROT_TOL, TRANS_TOL, both_sides, compare_linearization, pose_diff

pytestmark = pytest.mark.gpu

GN_FIXED = dict(lambda0=0.0, accept_step=1e30, eps_step=0.0, eps_step_coarse=0.0, huber_k=1e30)


@pytest.fixture(scope="module")
def glt():
    import paper_2607_16897_gb300 as g
    return g


@pytest.mark.parametrize("jacobian", ["forward", "ic"])
@pytest.mark.parametrize("pattern", [7, 11])
def test_square_patch_linearize_matches_oracle(glt, orc, syn, pattern, jacobian):
    p = syn.pair_c1(6, sigma=2.0)
    trk, ref = both_sides(glt, orc, p.cam.W, p.cam.H, p.cam.K, p.ref, p.cur, p.uvd, levels=3,
                          pattern=pattern, jacobian=jacobian)
    rng = np.random.default_rng(pattern)
    states = [(I34, 0.0, 0.0)]
    for _ in range(2):
        xi = np.concatenate([rng.normal(size=3) * 0.02, rng.normal(size=3) * 0.01])
        states.append((orc.se3_exp(xi), float(rng.normal() * 0.05), float(rng.normal() * 3)))
    for T, a, b in states:
        for level in range(3):
            g = trk.debug_linearize(level, T, a, b)
            assert g["res"].shape[1] == pattern * pattern
            compare_linearization(g, ref.debug_linearize(level, T, a, b),
                                  f"p {pattern} {jacobian} level {level}")
    trk.close()


@pytest.mark.parametrize("jacobian", ["ic", "forward"])
@pytest.mark.parametrize("W,H,f,pattern", [(640, 480, 525.0, 7), (752, 480, 458.0, 11)])
def test_paper_configuration_track_matches_oracle(glt, orc, syn, W, H, f, pattern, jacobian):
    cam = syn.camera_for(W, H, f)
    seq = syn.sequence(31, 10, cam, syn.ROOM_LARGE, 0.5, 30.0, a_range=(0.0, 0.0), b_range=(0.0, 0.0))
    ref, uvd = syn.reference_points(seq, 0, 2000, 0.5, 8.0)
    for k in (1, 4):
        cur, _ = seq.frame(k)
        trk, o = both_sides(glt, orc, W, H, cam.K, ref, cur, uvd, levels=6, pattern=pattern,
                            jacobian=jacobian, affine=False, **GN_FIXED)
        T0 = syn.relative(seq.T_wc[0], seq.T_wc[k - 1])
        g = trk.track_frame(T0, (0.0, 0.0))
        r = o.track_frame(T0, (0.0, 0.0))
        ang, dt = pose_diff(g["T"], r["T"])
        assert ang <= ROT_TOL and dt <= TRANS_TOL, (k, ang, dt)
        assert g["a"] == 0.0 and g["b"] == 0.0
        assert g["iters"][:6] == r["iters"] == [10] * 6
        ang_t, dt_t = pose_diff(g["T"], syn.relative(seq.T_wc[0], seq.T_wc[k]))
        assert dt_t < 3e-3, dt_t
        trk.close()


def test_fixed_affine_with_the_8_pixel_pattern(glt, orc, syn):
    p = syn.pair_c1(2, sigma=2.0)
    trk, o = both_sides(glt, orc, p.cam.W, p.cam.H, p.cam.K, p.ref, p.cur, p.uvd, levels=3,
                        affine=False)
    g = trk.track_frame(I34, (0.05, 3.0))
    r = o.track_frame(I34, (0.05, 3.0))
    assert g["a"] == 0.05 and g["b"] == 3.0
    ang, dt = pose_diff(g["T"], r["T"])
    assert ang <= ROT_TOL and dt <= TRANS_TOL
    trk.close()


def test_pattern_arguments_are_checked(glt):
    K = (256.0, 256.0, 160.0, 120.0)
    for kw in (dict(pattern=4), dict(pattern=13), dict(pattern=1), dict(pattern=7, precision="mixed"),
               dict(affine=2)):
        with pytest.raises(glt.GltError):
            glt.Tracker(320, 240, K, **kw)
