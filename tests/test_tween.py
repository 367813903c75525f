"""The tween-frame switch policy (Sec. III, Sec. IV-D): which direct-tracking
results are kept, when control returns to the indirect pipeline, and the
acceptance rate (the quantity of the paper's Table III).  Host logic only."""
import importlib.util
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def tween():
    # host-only module: loaded without the package's compiled part
    spec = importlib.util.spec_from_file_location(
        "tween_host_only", os.path.join(ROOT, "paper_2607_16897_gb300", "tween.py"))
    mod = importlib.util.module_from_spec(spec)
    sys.modules["tween_host_only"] = mod
    spec.loader.exec_module(mod)
    return mod


def res(status=0, n_valid=16000, cost=1.0):
    return {"status": status, "n_valid": n_valid, "cost": cost}


def test_acceptance_conditions(tween):
    sw = tween.TweenSwitch(max_direct=8, max_cost=2.5, min_valid_frac=0.5)
    N = 2000                                   # 8 N = 16000 samples
    assert sw.direct_ok(res(), N)
    assert not sw.direct_ok(res(status=1), N)          # too few points on a level
    assert not sw.direct_ok(res(status=2), N)          # not positive definite
    assert not sw.direct_ok(res(n_valid=7999), N)      # under half of the samples usable
    assert sw.direct_ok(res(n_valid=8000), N)
    assert not sw.direct_ok(res(cost=2.5000001), N)    # robust error above the threshold
    assert sw.direct_ok(res(cost=2.5), N)
    assert not sw.direct_ok(res(cost=float("nan")), N)
    assert not sw.direct_ok(res(cost=float("inf")), N)
    p7 = tween.TweenSwitch(samples_per_point=49)
    assert not p7.direct_ok(res(n_valid=16000), N)     # 49 N samples for 7 x 7 patches


def test_switch_back_after_the_direct_budget_or_a_rejection(tween):
    sw = tween.TweenSwitch(max_direct=3)
    N = 100
    sw.after_indirect()                                # reference 0
    assert not sw.after_direct(res(n_valid=800), N)
    assert not sw.after_direct(res(n_valid=800), N)
    assert sw.after_direct(res(n_valid=800), N)        # third direct frame: budget used up
    sw.after_indirect()
    assert sw.after_direct(res(cost=9.0, n_valid=800), N)   # rejected: back to indirect at once
    sw.after_indirect()
    assert sw.history == ["indirect", "direct", "direct", "direct", "indirect", "rejected", "indirect"]
    assert sw.direct_accepted == 3 and sw.direct_rejected == 1 and sw.indirect_frames == 3
    assert sw.frames == 7
    assert sw.acceptance_rate == pytest.approx(3 / 7)


def test_steady_state_rate_follows_the_budget(tween):
    """With every direct frame accepted the direct share is max_direct /
    (max_direct + 1): one indirect keyframe per max_direct tween frames."""
    for m in (1, 4, 8, 12):
        sw = tween.TweenSwitch(max_direct=m)
        for _ in range(20):
            sw.after_indirect()
            while not sw.after_direct(res(n_valid=8 * 50), 50):
                pass
        assert sw.acceptance_rate == pytest.approx(m / (m + 1))
