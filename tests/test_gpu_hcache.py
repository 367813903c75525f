"""The paper's cached Hessian on the GPU against the oracle (Sec. IV-B: H
precomputed once per reference update; Sec. IV-C: per-point H_i reduced into
one H per level at the reference, the track stage reducing only b per pass):
the per-reference H of every level and the pass's g, E, n and residuals at
the same states, whole solves in the paper's configuration (p x p patches,
6 levels, fixed-count Gauss-Newton) and with the 8-pixel pattern, batches of
such streams, and the not-positive-definite outcome.  Same tolerances as the
other forms."""
import numpy as np
import pytest

from helpers import I34, ROT_TOL, TRANS_TOL, both_sides, compare_linearization, pose_diff

pytestmark = pytest.mark.gpu

GN_FIXED = dict(lambda0=0.0, accept_step=1e30, eps_step=0.0, eps_step_coarse=0.0, huber_k=1e30)
CACHED = dict(GN_FIXED, jacobian="ic", hessian="cached", affine=False)


@pytest.fixture(scope="module")
def glt():
    import paper_2607_16897_gb300 as g
    return g


@pytest.mark.parametrize("pattern", [0, 7, 11, 5])
def test_cached_linearize_matches_oracle(glt, orc, syn, pattern):
    p = syn.pair_c1(6, sigma=2.0)
    cfg = dict(CACHED, pattern=pattern)
    if pattern == 5:
        cfg["huber_k"] = 9.0      # the weights enter g only (H is the reference's)
    trk, ref = both_sides(glt, orc, p.cam.W, p.cam.H, p.cam.K, p.ref, p.cur, p.uvd, levels=3, **cfg)
    rng = np.random.default_rng(pattern)
    states = [(I34, 0.0, 0.0)]
    for _ in range(2):
        xi = np.concatenate([rng.normal(size=3) * 0.02, rng.normal(size=3) * 0.01])
        states.append((orc.se3_exp(xi), float(rng.normal() * 0.05), float(rng.normal() * 3)))
    for T, a, b in states:
        for level in range(3):
            g = trk.debug_linearize(level, T, a, b)
            o = ref.debug_linearize(level, T, a, b)
            assert np.all(g["H"][6:] == 0) and np.all(g["H"][:, 6:] == 0) and np.all(g["g"][6:] == 0)
            compare_linearization(g, o, f"p {pattern} level {level}")
    trk.close()


@pytest.mark.parametrize("W,H,f,pattern", [(640, 480, 525.0, 7), (752, 480, 458.0, 11)])
def test_paper_configuration_cached_track_matches_oracle(glt, orc, syn, W, H, f, pattern):
    cam = syn.camera_for(W, H, f)
    seq = syn.sequence(31, 10, cam, syn.ROOM_LARGE, 0.5, 30.0, a_range=(0.0, 0.0), b_range=(0.0, 0.0))
    ref, uvd = syn.reference_points(seq, 0, 2000, 0.5, 8.0)
    trk, o = both_sides(glt, orc, W, H, cam.K, ref, seq.frame(1)[0], uvd, levels=6, pattern=pattern,
                        **CACHED)
    for k in (1, 4, 7):
        cur, _ = seq.frame(k)
        trk.build_pyramid(glt.GLT_CUR, cur)
        o.build_pyramid(1, cur)
        T0 = syn.relative(seq.T_wc[0], seq.T_wc[k - 1])
        g = trk.track_frame(T0, (0.0, 0.0))
        r = o.track_frame(T0, (0.0, 0.0))
        ang, dt = pose_diff(g["T"], r["T"])
        assert ang <= ROT_TOL and dt <= TRANS_TOL, (k, ang, dt)
        assert g["a"] == 0.0 and g["b"] == 0.0 and g["status"] == r["status"] == 0
        assert g["iters"][:6] == r["iters"] == [10] * 6
        ang_t, dt_t = pose_diff(g["T"], syn.relative(seq.T_wc[0], seq.T_wc[k]))
        assert dt_t < 3e-3, dt_t
    trk.close()


@pytest.mark.parametrize("seed", range(6))
def test_cached_track_8_pixel_pattern(glt, orc, syn, seed):
    """The cached Hessian with the library's 8-pixel pattern and an exposure
    change held at its true value."""
    p = syn.pair_c1(seed, sigma=2.0)
    trk, o = both_sides(glt, orc, p.cam.W, p.cam.H, p.cam.K, p.ref, p.cur, p.uvd, levels=3,
                        **CACHED)
    g = trk.track_frame(I34, (0.05, 3.0))
    r = o.track_frame(I34, (0.05, 3.0))
    ang, dt = pose_diff(g["T"], r["T"])
    assert ang <= ROT_TOL and dt <= TRANS_TOL, (seed, ang, dt)
    assert g["status"] == r["status"] and g["passes"] == r["passes"]
    trk.close()


def test_cached_batch_matches_oracle(glt, orc, syn):
    import torch
    pairs = [syn.pair_c1(s, sigma=2.0, N=n) for s, n in ((1, 500), (2, 37), (3, 300))]
    trks, orcs = [], []
    for p in pairs:
        t, o = both_sides(glt, orc, p.cam.W, p.cam.H, p.cam.K, p.ref, p.cur, p.uvd, levels=3,
                          pattern=7, **CACHED)
        trks.append(t)
        orcs.append(o)
    batch = glt.Batch(trks)
    frames = [torch.from_numpy(p.cur).cuda() for p in pairs]
    ptrs = torch.tensor([f.data_ptr() for f in frames], dtype=torch.int64, device="cuda")
    init = torch.from_numpy(np.stack([np.concatenate([I34.ravel(), [0.0, 0.0]])] * 3)).cuda()
    out = torch.zeros(3 * glt.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    batch.build_pyramid(ptrs)
    batch.track(init, out)
    torch.cuda.synchronize()
    for i, r in enumerate(glt.parse_results(out)):
        o = orcs[i].track_frame(I34, (0.0, 0.0))
        ang, dt = pose_diff(r["T"], o["T"])
        assert ang <= ROT_TOL and dt <= TRANS_TOL, (i, ang, dt)
        assert r["status"] == o["status"] and r["passes"] == o["passes"]
    batch.close()
    # a batch may not mix the cached and the per-pass form
    p = pairs[0]
    other = glt.Tracker(p.cam.W, p.cam.H, p.cam.K, levels=3, max_points=500)
    with pytest.raises(glt.GltError):
        glt.Batch([trks[0], other])
    other.close()
    for t in trks:
        t.close()


def test_cached_hessian_not_positive_definite(glt, orc, syn):
    """A reference without texture gives a singular H: every level ends at once
    with NOT_PD, on both sides."""
    p = syn.pair_c1(0, sigma=2.0)
    flat = np.full_like(p.ref, 100)
    trk, o = both_sides(glt, orc, p.cam.W, p.cam.H, p.cam.K, flat, p.cur, p.uvd, levels=3,
                        **CACHED)
    g = trk.track_frame(I34, (0.0, 0.0))
    r = o.track_frame(I34, (0.0, 0.0))
    assert g["status"] & glt.GLT_TRACK_NOT_PD and r["status"] & orc.NOT_PD
    assert np.array_equal(g["T"], I34) and g["iters_total"] == r["iters_total"] == 0
    trk.close()


def test_cached_hessian_arguments_are_checked(glt):
    K = (256.0, 256.0, 160.0, 120.0)
    ok = dict(CACHED, max_points=10)
    glt.Tracker(320, 240, K, **ok).close()
    for bad in (dict(jacobian="forward"), dict(affine=True), dict(lambda0=1e-4),
                dict(precision="mixed"), dict(threads=256), dict(hessian=2)):
        with pytest.raises(glt.GltError):
            glt.Tracker(320, 240, K, **dict(ok, **bad))
