"""The tracking state of the C ABI (checkpoint / resume, constant-velocity
start, Sec. IV-A): glt_state_update and glt_state_predict are host code and run
here without a GPU.  Pinned against closed forms: poses that advance by one
fixed rigid motion E (T_k = E^k T_0) are predicted exactly by the constant-
velocity model, whatever E is."""
import ctypes
import math

import numpy as np
import pytest


@pytest.fixture(scope="module")
def glt():
    import paper_2607_16897_gb300 as g
    return g


def rigid(rng, rot=0.3, trans=0.5):
    """A random rigid transform from Rodrigues' formula (rotation about a
    random axis by a random angle), written out here."""
    axis = rng.normal(size=3)
    axis /= np.linalg.norm(axis)
    th = rng.uniform(-rot, rot)
    Kx = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    R = np.eye(3) + math.sin(th) * Kx + (1 - math.cos(th)) * Kx @ Kx
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = rng.normal(size=3) * trans
    return T


def result(glt, T4, a=0.0, b=0.0):
    r = glt.glt_result()
    for i, v in enumerate(T4[:3].reshape(12)):
        r.T[i] = v
    r.a, r.b = a, b
    return r


def predict(glt, st):
    T = (ctypes.c_double * 12)()
    ab = (ctypes.c_double * 2)()
    rc = glt.glt_state_predict(ctypes.byref(st), T, ab)
    return rc, np.vstack([np.array(T[:]).reshape(3, 4), [0, 0, 0, 1]]), tuple(ab[:])


def fresh_state(glt):
    st = glt.glt_state()
    for i in (0, 5, 10):
        st.T_cr[i] = 1.0
        st.motion[i] = 1.0
    return st


def test_layout(glt):
    assert ctypes.sizeof(glt.glt_state) == 216
    assert glt.glt_state.reference.offset == 26 * 8


@pytest.mark.parametrize("seed", range(5))
def test_constant_motion_is_predicted_exactly(glt, seed):
    rng = np.random.default_rng(seed)
    E, T = rigid(rng), rigid(rng, 1.0, 2.0)
    st = fresh_state(glt)
    assert glt.glt_state_update(ctypes.byref(st), ctypes.byref(result(glt, T, 0.1, -2.0))) == 0
    for k in range(1, 6):
        T = E @ T
        assert glt.glt_state_update(ctypes.byref(st), ctypes.byref(result(glt, T, 0.1 * k, 3.0))) == 0
        rc, P, ab = predict(glt, st)
        assert rc == 0
        assert np.abs(P - E @ T).max() < 1e-12, k          # the next pose of the constant motion
        assert ab == (0.1 * k, 3.0)                          # the last affine pair
        assert np.abs(np.array(st.motion[:]).reshape(3, 4) - E[:3]).max() < 1e-12
    assert st.frames == 6


def test_first_frame_predicts_the_last_pose(glt):
    """Identity motion (a new tracker): the prediction is the pose itself."""
    rng = np.random.default_rng(7)
    T = rigid(rng)
    st = fresh_state(glt)
    for i, v in enumerate(T[:3].reshape(12)):
        st.T_cr[i] = v
    rc, P, _ = predict(glt, st)
    assert rc == 0 and np.abs(P - T).max() < 1e-14


def test_prediction_is_orthonormalised(glt):
    st = fresh_state(glt)
    st.T_cr[1] = 1e-3          # a slightly sheared rotation
    st.T_cr[4] = 2e-3
    rc, P, _ = predict(glt, st)
    R = P[:3, :3]
    assert rc == 0
    assert np.abs(R @ R.T - np.eye(3)).max() < 1e-15 and abs(np.linalg.det(R) - 1) < 1e-15
    assert abs(R[0, 0] - 1 / math.hypot(1, 1e-3)) < 1e-15   # the first row is only normalised


def test_non_finite_result_leaves_the_state(glt):
    st = fresh_state(glt)
    before = bytes(st)
    bad = result(glt, np.eye(4))
    bad.T[3] = float("nan")
    assert glt.glt_state_update(ctypes.byref(st), ctypes.byref(bad)) == glt.GLT_ERR_INVALID_ARG
    bad = result(glt, np.eye(4), b=float("inf"))
    assert glt.glt_state_update(ctypes.byref(st), ctypes.byref(bad)) == glt.GLT_ERR_INVALID_ARG
    assert bytes(st) == before
    st.motion[0] = float("nan")
    assert predict(glt, st)[0] == glt.GLT_ERR_INVALID_ARG


def test_null_arguments(glt):
    st = fresh_state(glt)
    assert glt.glt_get_state(None, ctypes.byref(st)) == glt.GLT_ERR_INVALID_ARG
    assert glt.glt_set_state(None, ctypes.byref(st)) == glt.GLT_ERR_INVALID_ARG
    assert glt.glt_state_update(None, None) == glt.GLT_ERR_INVALID_ARG
    assert glt.glt_state_predict(ctypes.byref(st), None, None) == glt.GLT_ERR_INVALID_ARG
    assert glt.glt_nn_save(None, b"x") == glt.GLT_ERR_INVALID_ARG
    assert glt.glt_nn_load(None, b"x") == glt.GLT_ERR_INVALID_ARG
    assert glt.glt_status_string(glt.GLT_ERR_IO) == b"file error"
