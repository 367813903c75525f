"""Pins of the oracle's SE(3) exponential/logarithm (Sec. IV-A: 6-D twist,
T <- T exp(delta)).  The exponential is checked against scipy's matrix
exponential of the 4x4 twist matrix, which is the definition of exp on se(3)."""
import numpy as np
import pytest

expm = pytest.importorskip("scipy.linalg").expm
logm = pytest.importorskip("scipy.linalg").logm


def twist_matrix(xi):
    v, w = xi[:3], xi[3:]
    M = np.zeros((4, 4))
    M[:3, :3] = [[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]]
    M[:3, 3] = v
    return M


def to4(T):
    M = np.eye(4)
    M[:3, :] = T
    return M


ANGLES = [0.0, 1e-9, 3e-6, 9.99e-5, 1.001e-4, 1e-3, 0.0999, 0.1001, 0.3, 1.5, 2.9]


@pytest.mark.parametrize("theta", ANGLES)
def test_exp_matches_matrix_exponential(orc, theta):
    rng = np.random.default_rng(int(theta * 1e6) + 3)
    ax = rng.normal(size=3)
    ax /= np.linalg.norm(ax)
    xi = np.concatenate([rng.normal(size=3) * 0.3, theta * ax])
    T = orc.se3_exp(xi)
    ref = expm(twist_matrix(xi))[:3, :]
    np.testing.assert_allclose(T, ref, atol=1e-13, rtol=0)
    R = T[:, :3]
    np.testing.assert_allclose(R.T @ R, np.eye(3), atol=1e-14)
    assert np.linalg.det(R) > 0


@pytest.mark.parametrize("theta", ANGLES[:-1])
def test_log_inverts_exp(orc, theta):
    rng = np.random.default_rng(int(theta * 1e6) + 11)
    ax = rng.normal(size=3)
    ax /= np.linalg.norm(ax)
    xi = np.concatenate([rng.normal(size=3) * 0.2, theta * ax])
    np.testing.assert_allclose(orc.se3_log(orc.se3_exp(xi)), xi, atol=1e-12, rtol=1e-10)


def test_log_matches_matrix_logarithm(orc):
    rng = np.random.default_rng(2)
    for _ in range(10):
        xi = rng.normal(size=6) * 0.4
        T = orc.se3_exp(xi)
        L = np.real(logm(to4(T)))
        ref = np.array([L[0, 3], L[1, 3], L[2, 3], L[2, 1], L[0, 2], L[1, 0]])
        np.testing.assert_allclose(orc.se3_log(T), ref, atol=1e-10)


def test_exp_of_negative_is_inverse(orc):
    rng = np.random.default_rng(4)
    for _ in range(20):
        xi = rng.normal(size=6) * rng.choice([1e-7, 1e-3, 0.5])
        P = to4(orc.se3_mul(orc.se3_exp(xi), orc.se3_exp(-xi)))
        np.testing.assert_allclose(P, np.eye(4), atol=1e-14)


@pytest.mark.parametrize("th0", [1e-4, 0.1])
def test_series_branches_are_continuous(orc, th0):
    ax = np.array([0.3, -0.5, 0.8])
    ax /= np.linalg.norm(ax)
    v = np.array([0.1, 0.2, -0.3])
    lo = np.concatenate([v, (th0 * (1 - 1e-9)) * ax])
    hi = np.concatenate([v, (th0 * (1 + 1e-9)) * ax])
    Tlo, Thi = orc.se3_exp(lo), orc.se3_exp(hi)
    np.testing.assert_allclose(Tlo, Thi, atol=1e-15 + 2e-9 * th0)
    np.testing.assert_allclose(orc.se3_log(Tlo), lo, atol=1e-15)
    np.testing.assert_allclose(orc.se3_log(Thi), hi, atol=1e-15)


def test_compose_matches_homogeneous_product(orc):
    rng = np.random.default_rng(8)
    A = orc.se3_exp(rng.normal(size=6))
    B = orc.se3_exp(rng.normal(size=6))
    np.testing.assert_allclose(to4(orc.se3_mul(A, B)), to4(A) @ to4(B), atol=1e-14)
