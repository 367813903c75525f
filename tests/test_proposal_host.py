"""Host-side logic of the learned proposal (no GPU): the SE(3) log behind the
motion input and the training targets, checked against the oracle's SE(3)
exp/log and against closed cases."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def prop():
    import importlib.util
    import os
    import sys
    # the module's top level needs no library; load it without the package's
    # compiled part so this runs on any host
    here = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                        "paper_2607_16897_gb300", "proposal.py")
    spec = importlib.util.spec_from_file_location("proposal_host_only", here)
    mod = importlib.util.module_from_spec(spec)
    sys.modules["proposal_host_only"] = mod
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("scale", [0.0, 1e-7, 1e-4, 2e-3, 0.05, 0.7, 2.5])
def test_se3_log_inverts_oracle_exp(prop, orc, scale):
    rng = np.random.default_rng(int(scale * 1e7) + 3)
    for _ in range(5):
        xi = rng.normal(size=6)
        xi[3:] *= scale / max(np.linalg.norm(xi[3:]), 1e-300)
        xi[:3] *= 0.3
        T = orc.se3_exp(xi)
        assert np.allclose(prop.se3_log(T), xi, atol=1e-12, rtol=1e-9), (scale, xi)
        assert np.allclose(prop.se3_log(T), orc.se3_log(T), atol=1e-12)


def test_target_and_motion_feature(prop, orc):
    rng = np.random.default_rng(5)
    T0 = orc.se3_exp(rng.normal(size=6) * 0.3)
    d = np.array([0.003, -0.002, 0.004, 0.001, -0.0015, 0.0005, 0.02, -0.7])
    Tc = orc.se3_mul(T0, orc.se3_exp(d[:6]))
    t = prop.target(T0, (0.1, 2.0), Tc, (0.1 + d[6], 2.0 + d[7]))
    assert np.allclose(t * prop.OUT_SCALE, d, atol=1e-7)
    # motion: x_{k-1} = M x_{k-2} with world->camera poses
    M = orc.se3_exp(np.array([0.01, 0.0, 0.02, 0.0, 0.01, 0.0]))
    Tpp = orc.se3_exp(rng.normal(size=6) * 0.2)
    Tp = orc.se3_mul(M, Tpp)
    m = prop.motion_feature(Tp, Tpp)
    assert np.allclose(m * prop.MOTION_SCALE, orc.se3_log(M), atol=1e-7)
    assert not np.any(prop.motion_feature(Tp, None))


def test_init_params_layout(prop):
    w = prop.init_params(0)
    assert w.dtype == np.float32 and w.size == 189064
    assert not np.any(w[144:160])                      # conv1 bias zero
    assert np.abs(w[188032:189056]).max() < 0.1 * np.sqrt(6 / 128) + 1e-6   # scaled last layer


def test_stream_motion_range(prop):
    for s in range(10000, 10050):
        v, w = prop.stream_motion(s)
        assert 0.5 <= v <= 2.0 and 30.0 <= w <= 90.0
