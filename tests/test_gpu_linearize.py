"""One linearisation at the same state on both sides: per-sample residuals
within 1e-3 gray, H within 1e-5 relative (Frobenius), g within 1e-5 of
sum |w J r|, identical valid-sample counts (Eqs. 3-5)."""
import numpy as np
import pytest

from helpers import I34, both_sides, compare_linearization

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def glt():
    import paper_2607_16897_gb300 as g
    return g


def states(orc, rng, n=4):
    out = [(I34, 0.0, 0.0)]
    for _ in range(n):
        xi = np.concatenate([rng.normal(size=3) * 0.02, rng.normal(size=3) * 0.01])
        out.append((orc.se3_exp(xi), float(rng.normal() * 0.05), float(rng.normal() * 3)))
    return out


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_linearize_c1(glt, orc, syn, seed, precision):
    p = syn.pair_c1(seed, sigma=2.0)
    trk, ref = both_sides(glt, orc, p.cam.W, p.cam.H, p.cam.K, p.ref, p.cur, p.uvd, levels=3,
                          precision=precision)
    rng = np.random.default_rng(seed)
    for T, a, b in states(orc, rng):
        for level in range(3):
            g = trk.debug_linearize(level, T, a, b)
            o = ref.debug_linearize(level, T, a, b)
            compare_linearization(g, o, f"seed {seed} level {level}")
    trk.close()


@pytest.mark.parametrize("N", [1, 31, 127, 128, 129, 1000, 2000, 4000])
def test_linearize_c2_sizes_and_ragged_tails(glt, orc, syn, N):
    cam = syn.camera_for(640, 480, 525.0)
    seq = syn.sequence(1, 12, cam, syn.ROOM_LARGE, 0.5, 30.0)
    ref, uvd = syn.reference_points(seq, 0, N, 0.5, 8.0)
    cur, _ = seq.frame(6)
    trk, o = both_sides(glt, orc, 640, 480, cam.K, ref, cur, uvd, levels=4)
    T = syn.relative(seq.T_wc[0], seq.T_wc[6])
    a, b = seq.rel_affine(0, 6)
    for level in range(4):
        compare_linearization(trk.debug_linearize(level, T, a, b), o.debug_linearize(level, T, a, b),
                              f"N {N} level {level}")
    trk.close()


def test_linearize_1280_mixed(glt, orc, syn):
    cam = syn.camera_for(1280, 720, 1050.0)
    seq = syn.sequence(2000, 4, cam, syn.ROOM_LARGE, 1.0, 60.0)
    ref, uvd = syn.reference_points(seq, 0, 8000, 0.5, 8.0)
    cur, _ = seq.frame(2)
    T = syn.relative(seq.T_wc[0], seq.T_wc[2])
    a, b = seq.rel_affine(0, 2)
    for prec in ("fp32", "mixed"):
        trk, o = both_sides(glt, orc, 1280, 720, cam.K, ref, cur, uvd, levels=5, precision=prec)
        for level in (0, 2, 4):
            compare_linearization(trk.debug_linearize(level, T, a, b),
                                  o.debug_linearize(level, T, a, b), f"{prec} level {level}")
        trk.close()


def test_linearize_edge_cases(glt, orc, syn):
    p = syn.pair_c1(3, sigma=2.0)
    # every point out of view: n = 0, H = 0
    trk, o = both_sides(glt, orc, p.cam.W, p.cam.H, p.cam.K, p.ref, p.cur, p.uvd, levels=3)
    T = I34.copy()
    T[0, 3] = 50.0
    g = trk.debug_linearize(0, T, 0.0, 0.0)
    assert g["n"] == 0 and not np.any(g["H"]) and np.isnan(g["res"]).all()
    # a point behind the camera and one with non-positive depth
    uvd = p.uvd[:40].copy()
    uvd[0, 2] = -1.0
    uvd[1, 2] = 0.0
    trk2, o2 = both_sides(glt, orc, p.cam.W, p.cam.H, p.cam.K, p.ref, p.cur, uvd, levels=3)
    Tb = I34.copy()
    Tb[2, 3] = -2.5   # pushes the nearest points behind zmin
    for TT in (I34, Tb):
        compare_linearization(trk2.debug_linearize(0, TT, 0.0, 0.0), o2.debug_linearize(0, TT, 0.0, 0.0))
    trk.close()
    trk2.close()
