"""Pins of the oracle's coarse-to-fine LM tracker (Sec. IV-A: coarse level
initialises the finer one; Sec. IV-C "Track": Cholesky solve, T <- T exp(delta)).

The tracker is an iteration, so it is pinned by what the solution must satisfy:
  * pure brightness change with unchanged geometry -> exact (a, b), identity pose;
  * known-pose recovery on rendered frame pairs (noise-free and sigma = 2);
  * the converged state is a minimum of the cost on a brute-force grid;
  * the schedule's degenerate cases (no iterations, too few points, singular H).
"""
import numpy as np
import pytest

I34 = np.hstack([np.eye(3), np.zeros((3, 1))])


def tracker_for(orc, p, L=3, **cfg):
    tr = orc.OracleTracker(p.cam.W, p.cam.H, p.cam.K, levels=L, **cfg)
    tr.build_pyramid(0, p.ref)
    tr.set_map_points(p.uvd)
    tr.build_pyramid(1, p.cur)
    return tr


def pose_err(syn, T, Tt):
    return (np.rad2deg(syn.rotation_angle(T[:, :3].T @ Tt[:, :3])),
            1000.0 * np.linalg.norm(T[:, 3] - Tt[:, 3]))


def test_pure_affine_change_is_recovered_exactly(orc, syn):
    # every level run to eps_step: the stop rule looks at the pose part of the
    # step only, so a coarse-level stop can leave b some 1e-7 gray short
    p = syn.pair_c1(1, sigma=2.0)
    tr = tracker_for(orc, p, eps_step_coarse=1e-6)
    a, b = 0.05, 3.0
    cur = [np.exp(a) * lv.astype(np.float64) + b for lv in tr.pyr[0]]
    res = orc.track(cur, p.cam.K, tr.x_r, tr.I0, tr.valid, tr.cfg, I34, 0.0, 0.0)
    assert abs(res["a"] - a) < 1e-9
    assert abs(res["b"] - b) < 1e-7
    np.testing.assert_allclose(res["T"], I34, atol=1e-9)
    assert res["status"] == 0


@pytest.mark.parametrize("seed", range(5))
def test_known_pose_recovery_noise_free(orc, syn, seed):
    p = syn.pair_c1(seed, sigma=0.0)
    res = tracker_for(orc, p).track_frame(I34)
    rot, trans = pose_err(syn, res["T"], p.T_cr)
    assert rot <= 0.01 and trans <= 0.5, (rot, trans)
    assert abs(res["a"] - p.a) < 2e-3 and abs(res["b"] - p.b) < 0.3
    assert res["status"] == 0


def test_known_pose_recovery_with_noise(orc, syn):
    errs = []
    for seed in range(20):
        p = syn.pair_c1(seed, sigma=2.0)
        res = tracker_for(orc, p).track_frame(I34)
        errs.append(pose_err(syn, res["T"], p.T_cr))
    errs = np.array(errs)
    assert errs[:, 0].max() <= 0.05 and errs[:, 1].max() <= 2.0, errs
    # the initial error is 2 degrees / 30 mm: every seed must improve on it 100x
    assert (errs[:, 0] < 0.02).mean() >= 0.9


@pytest.mark.parametrize("seed", [0, 2, 6])
def test_converged_state_is_a_grid_minimum(orc, syn, seed):
    """The Jacobian uses bilinearly sampled central-difference gradients, not
    the exact derivative of the bilinear interpolant, so the LM fixed point
    sits within ~1e-4 of the cost minimum; a +-1e-3 grid must not beat it."""
    p = syn.pair_c1(seed, sigma=2.0, N=60)
    tr = tracker_for(orc, p)
    res = tr.track_frame(I34)
    base = tr.debug_linearize(0, res["T"], res["a"], res["b"], per_sample=False)
    c0 = base["E"] / base["n"]
    # the reported cost is that of the last evaluated state (the final step,
    # below eps_step, is taken without a pass of its own): the trace's last
    # accepted finest-level evaluation, within 1e-6 of the cost at the pose
    last = [e["cost"] for e in res["trace"] if e["level"] == 0 and (e["accepted"] or not e["candidate"])][-1]
    assert res["cost"] == last
    assert abs(c0 - res["cost"]) <= 1e-6 * c0
    steps = [1e-3] * 6 + [1e-3, 1e-1]
    for i in range(8):
        for sgn in (-1, 1):
            d = np.zeros(8)
            d[i] = sgn * steps[i]
            T = orc.se3_mul(res["T"], orc.se3_exp(d[:6]))
            o = tr.debug_linearize(0, T, res["a"] + d[6], res["b"] + d[7], per_sample=False)
            assert o["E"] / o["n"] >= c0 - 1e-12 * c0, (i, sgn)


def test_weak_first_order_optimality(orc, syn):
    """Bilinear interpolation makes the cost only piecewise smooth, so the
    gradient at the minimum is bounded by the kinks, not zero."""
    for seed in range(3):
        p = syn.pair_c1(seed, sigma=2.0)
        tr = tracker_for(orc, p)
        res = tr.track_frame(I34)
        lin = tr.debug_linearize(0, res["T"], res["a"], res["b"])
        pv = lin["point_valid"]
        absg = np.abs(lin["J"][pv] * (lin["w"][pv] * lin["res"][pv])[:, :, None]).sum((0, 1))
        assert (np.abs(lin["g"]) <= 5e-3 * absg).all()


def test_initial_state_far_is_worse_than_converged(orc, syn):
    p = syn.pair_c1(4, sigma=2.0)
    tr = tracker_for(orc, p)
    res = tr.track_frame(I34)
    start = tr.debug_linearize(0, I34, 0.0, 0.0, per_sample=False)
    assert res["cost"] < 0.2 * start["E"] / start["n"]
    assert sum(res["iters"]) == res["iters_total"]
    # one start pass per level and one pass per candidate, except the last
    # step of a coarse level that ends on its step threshold (taken unevaluated)
    evaluated = [sum(1 for e in res["trace"] if e["candidate"] and e["level"] == l) for l in range(3)]
    unevaluated = [res["iters"][l] - evaluated[l] for l in range(3)]
    assert all(u in (0, 1) for u in unevaluated) and sum(unevaluated) >= 1
    assert res["passes"] == len(res["trace"]) == res["iters_total"] + 3 - sum(unevaluated)


def test_zero_iterations_leave_state(orc, syn):
    p = syn.pair_c1(0, sigma=2.0)
    tr = tracker_for(orc, p, max_iters=[0] * 8)
    T0 = orc.se3_exp([0.01, 0, 0, 0, 0.02, 0])
    res = tr.track_frame(T0, (0.1, 2.0))
    np.testing.assert_array_equal(res["T"], T0)
    assert res["a"] == 0.1 and res["b"] == 2.0 and res["passes"] == 0
    assert np.isnan(res["cost"])


def test_too_few_points(orc, syn):
    p = syn.pair_c1(0, sigma=2.0)
    p.uvd = p.uvd[:1]
    tr = tracker_for(orc, p)
    res = tr.track_frame(I34)
    assert res["status"] & orc.TOO_FEW_POINTS
    np.testing.assert_array_equal(res["T"], I34)
    assert res["iters_total"] == 0 and res["passes"] == 3


def test_non_finite_start_and_sums_diverge(orc, syn):
    """Failure detection: a start that is not finite is returned unsolved; a
    gain e^a beyond the FP64 range makes every level start's sums NaN, so no
    level runs; both set DIVERGED and nothing else."""
    p = syn.pair_c1(0, sigma=2.0)
    tr = tracker_for(orc, p)
    T0 = I34.copy()
    T0[1, 3] = np.nan
    res = tr.track_frame(T0)
    assert res["status"] == orc.DIVERGED and res["passes"] == 0
    res = tr.track_frame(np.zeros((3, 4)))          # rotation with no direction
    assert res["status"] == orc.DIVERGED and res["passes"] == 0
    res = tr.track_frame(I34, (1000.0, 0.0))
    assert res["status"] == orc.DIVERGED and res["passes"] == 3
    np.testing.assert_array_equal(res["T"], I34)
    assert res["a"] == 1000.0 and res["iters_total"] == 0
    # an ordinary start after them is untouched by the rule
    assert tr.track_frame(I34)["status"] == 0


def test_singular_hessian_is_not_pd(orc, syn):
    p = syn.pair_c1(0, sigma=2.0)
    p.cur = np.full_like(p.cur, 100)   # no texture: the pose block of H is zero
    tr = tracker_for(orc, p)
    res = tr.track_frame(I34)
    assert res["status"] & orc.NOT_PD
    np.testing.assert_array_equal(res["T"], I34)


def test_trace_follows_the_accept_rule(orc, syn):
    """Every accepted candidate lowers the cost or is a small (Gauss-Newton)
    step below accept_step; every rejected one does neither."""
    for seed in range(4):
        p = syn.pair_c1(seed, sigma=2.0)
        tracker = tracker_for(orc, p)
        res = tracker.track_frame(I34)
        tr = res["trace"]
        acc_step = tracker.cfg["accept_step"]
        assert len(tr) == res["passes"]
        cur = None
        n_small = 0
        for e in tr:
            if not e["candidate"]:
                cur = e["cost"]
                continue
            small = e["step"] < acc_step
            if e["accepted"]:
                assert e["cost"] < cur or small
                n_small += (not e["cost"] < cur)
                cur = e["cost"]
            else:
                assert not e["cost"] < cur and not small
        assert res["cost"] == cur
        # the final step of the finest level is below eps_step or hit a stop rule
        assert [e["level"] for e in tr if not e["candidate"]] == [2, 1, 0]


def test_final_state_is_path_independent(orc, syn):
    """Gauss-Newton near convergence has one fixed point per level: starting
    level 0 from states 1e-4 apart ends within eps_step (1e-6) of each other."""
    p = syn.pair_c1(15, sigma=2.0)
    tracker = tracker_for(orc, p)
    base = tracker.track_frame(I34)
    rng = np.random.default_rng(0)
    ends = []
    for _ in range(4):
        T0 = orc.se3_mul(base["T"], orc.se3_exp(rng.normal(size=6) * 1e-4))
        r = orc.track(tracker.pyr[1], p.cam.K, tracker.x_r, tracker.I0, tracker.valid,
                      dict(tracker.cfg, max_iters=[10, 0, 0] + [0] * 5), T0, base["a"], base["b"])
        ends.append(r["T"])
    for T in ends:
        assert np.linalg.norm(T[:, 3] - ends[0][:, 3]) < 1e-6
        assert np.abs(T[:, :3] - ends[0][:, :3]).max() < 1e-6


def test_initial_rotation_is_reorthonormalised(orc, syn):
    """A slightly non-orthonormal initial rotation is projected onto SO(3)
    (Gram-Schmidt on the rows) before the solve: the result is orthonormal
    and equals the result from the projected initial pose."""
    p = syn.pair_c1(2, sigma=2.0)
    tr = tracker_for(orc, p)
    T0 = orc.se3_exp([0.005, -0.01, 0.002, 0.01, -0.02, 0.005])
    bad = T0.copy()
    bad[:, :3] += 1e-3 * np.array([[0.3, -0.2, 0.5], [0.1, 0.4, -0.3], [-0.2, 0.6, 0.1]])
    r = tr.track_frame(bad)
    R = r["T"][:, :3]
    assert np.abs(R @ R.T - np.eye(3)).max() < 1e-13
    # Gram-Schmidt of `bad` written out with numpy
    q0 = bad[0, :3] / np.linalg.norm(bad[0, :3])
    q1 = bad[1, :3] - (bad[1, :3] @ q0) * q0
    q1 /= np.linalg.norm(q1)
    G = bad.copy()
    G[:, :3] = np.stack([q0, q1, np.cross(q0, q1)])
    r2 = tr.track_frame(G)
    np.testing.assert_allclose(r["T"], r2["T"], atol=1e-12)


@pytest.mark.parametrize("seed", [3, 8])
def test_coarse_level_stop_rule_keeps_the_fixed_point(orc, syn, seed):
    """Levels above the finest stop once a candidate step is below
    eps_step_coarse; that step is taken without a pass of its own (it would be
    accepted whatever its cost), so every evaluated candidate of such a level
    is at or above the threshold and the level counts one step more than it
    evaluated.  The final state equals the one of a schedule that runs every
    level to eps_step: the coarse levels only have to bring the state into the
    finest level's basin, where Gauss-Newton has one fixed point."""
    p = syn.pair_c1(seed, sigma=2.0)
    tracker = tracker_for(orc, p)
    res = tracker.track_frame(I34)
    eps_c = tracker.cfg["eps_step_coarse"]
    assert eps_c > tracker.cfg["eps_step"]
    tr = res["trace"]
    for lvl in (2, 1):
        steps = [e["step"] for e in tr if e["candidate"] and e["level"] == lvl]
        assert all(s >= eps_c for s in steps)
        assert res["iters"][lvl] == len(steps) + 1 or len(steps) == tracker.cfg["max_iters"][lvl]
    # the levels' start passes follow one another with no coarse pass between
    # the unevaluated step and the next level's start
    starts = [k for k, e in enumerate(tr) if not e["candidate"]]
    assert [tr[k]["level"] for k in starts] == [2, 1, 0]
    fine = orc.OracleTracker(p.cam.W, p.cam.H, p.cam.K, levels=3, eps_step_coarse=1e-6)
    fine.build_pyramid(0, p.ref)
    fine.set_map_points(p.uvd)
    fine.build_pyramid(1, p.cur)
    ref = fine.track_frame(I34)
    assert res["passes"] < ref["passes"]
    assert np.linalg.norm(res["T"][:, 3] - ref["T"][:, 3]) < 1e-6
    assert np.abs(res["T"][:, :3] - ref["T"][:, :3]).max() < 1e-6
