"""The vectorized sequence driver of the batched end-to-end loop (bench.py
BatchDriver) against one SequenceDriver per stream, on synthetic
trajectories and tracker results (no GPU): the same initial states, motion
features, acceptance decisions and reference schedule."""
import math
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    sys.path.insert(0, ROOT)
    import bench as b
    return b


def rot(axis, th):
    axis = np.asarray(axis, float) / np.linalg.norm(axis)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + math.sin(th) * K + (1 - math.cos(th)) * K @ K


class FakeWorkload:
    """The attributes the drivers read: true world->camera poses, solver
    settings, point count and the acceptance threshold."""

    def __init__(self, rng, frames, pattern=0):
        self.N = int(rng.integers(300, 4000))
        self.max_cost = 2.5
        self.solver = {"pattern": pattern} if pattern else {}
        self.poses = []
        for k in range(frames):
            T = np.zeros((3, 4))
            T[:, :3] = rot(rng.normal(size=3), 0.02 * k + rng.normal() * 0.01)
            T[:, 3] = rng.normal(size=3) * 0.05 + 0.02 * k
            self.poses.append(T)

    def T_ref_world(self, r):
        return self.poses[r]


def fake_result(bench, rng, wl, drv_r, k, bad_kind):
    # the relative pose the tracker would return: truth plus a small error
    Trel = bench.pose_mul(wl.poses[k], bench.pose_inv(wl.poses[drv_r]))
    E = np.zeros((3, 4))
    E[:, :3] = rot(rng.normal(size=3), 1e-4)
    E[:, 3] = rng.normal(size=3) * 1e-4
    T = bench.pose_mul(E, Trel)
    K = 8 if not wl.solver else wl.solver["pattern"] ** 2
    res = {"T": T, "a": float(rng.normal() * 0.01), "b": float(rng.normal()),
           "status": 0, "n_valid": int(0.9 * K * wl.N), "cost": float(rng.uniform(0.5, 2.0))}
    if bad_kind == 1:
        res["status"] = 2
    elif bad_kind == 2:
        res["cost"] = 9.0
    elif bad_kind == 3:
        res["n_valid"] = int(0.4 * K * wl.N)
    return res


@pytest.mark.parametrize("seed", range(4))
def test_batch_driver_follows_the_per_stream_driver(bench, seed):
    rng = np.random.default_rng(seed)
    S, F = 7, 24
    wls = [FakeWorkload(rng, F, pattern=7 if s == 3 else 0) for s in range(S)]
    drvs = [bench.SequenceDriver(w) for w in wls]
    bd = bench.BatchDriver(wls)
    for d in drvs:
        d.refresh(0)
    assert list(bd.refresh(0)) == list(range(S))
    for k in range(1, F):
        # initial states and the inter-frame motions (the proposal stage's input)
        init = bd.init_for()
        mot = bd.motion()
        for s, d in enumerate(drvs):
            np.testing.assert_allclose(init[s], d.init_for(k), atol=1e-12, rtol=0)
            np.testing.assert_allclose(mot[s], d.motion(k), atol=1e-12, rtol=0)
            assert tuple(bd.ab[s]) == d.ab_init()
        # one tracked frame per stream, some of them failing the acceptance test
        res = [fake_result(bench, rng, wls[s], drvs[s].r, k,
                           int(rng.integers(4)) if rng.random() < 0.15 else 0) for s in range(S)]
        for s, d in enumerate(drvs):
            d.record(k, res[s])
        bd.record(k, np.stack([r["T"] for r in res]), np.array([r["a"] for r in res]),
                  np.array([r["b"] for r in res]), np.array([r["status"] for r in res]),
                  np.array([r["n_valid"] for r in res]), np.array([r["cost"] for r in res]))
        assert list(bd.rejected) == [d.rejected for d in drvs]
        # the reference schedule
        want = [s for s, d in enumerate(drvs) if d.refresh(k)]
        assert list(bd.refresh(k)) == want
        assert list(bd.r) == [d.r for d in drvs]
    assert bd.rejected.sum() > 0 and bd.accepted.sum() > 0


def test_batched_pose_helpers(bench):
    rng = np.random.default_rng(9)
    T = np.stack([np.hstack([rot(rng.normal(size=3), rng.uniform(-2, 2)), rng.normal(size=(3, 1))])
                  for _ in range(6)])
    U = np.stack([np.hstack([rot(rng.normal(size=3), rng.uniform(-2, 2)), rng.normal(size=(3, 1))])
                  for _ in range(6)])
    for i in range(6):
        np.testing.assert_allclose(bench.poses_mul(T, U)[i], bench.pose_mul(T[i], U[i]), atol=1e-14)
        np.testing.assert_allclose(bench.poses_inv(T)[i], bench.pose_inv(T[i]), atol=1e-14)
    skew = T.copy()
    skew[:, 0, 1] += 1e-3
    Q = bench.poses_orthonormalised(skew)
    for i in range(6):
        np.testing.assert_allclose(Q[i], bench.orthonormalised(skew[i]), atol=1e-14)
