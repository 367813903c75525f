"""Pins of the FP64 oracle of the proposal network: library correlation for the
convolution, an explicit-loop forward pass, central finite differences for
every gradient, the closed form of the first Adam step, and torch's bfloat16
rounding."""
import numpy as np
import pytest

signal = pytest.importorskip("scipy.signal")


@pytest.fixture(scope="module")
def nn():
    from oracle import nn as m
    return m


def test_conv_matches_library_correlation(nn):
    rng = np.random.default_rng(0)
    for (H, W) in [(30, 40), (15, 20), (8, 10)]:
        x = rng.normal(size=(2, 3, H, W))
        w = rng.normal(size=(4, 3, 3, 3))
        b = rng.normal(size=4)
        out = nn.conv2d_s2(x, w, b)
        for bi in range(2):
            for o in range(4):
                ref = np.full(((H + 1) // 2, (W + 1) // 2), b[o])
                for c in range(3):
                    xp = np.pad(x[bi, c], 1)
                    ref += signal.correlate2d(xp, w[o, c], mode="valid")[::2, ::2][:ref.shape[0], :ref.shape[1]]
                np.testing.assert_allclose(out[bi, o], ref, atol=1e-12)


def test_forward_matches_explicit_loops(nn):
    rng = np.random.default_rng(1)
    p = nn.init_params(3)
    for k in p:
        p[k] = p[k] + 0.05 * rng.normal(size=p[k].shape)
    x = rng.normal(size=(1, 1, 30, 40))
    m = rng.normal(size=(1, 6))
    y, _ = nn.forward(p, x, m)

    def conv(a, w, bias):
        C, H, W = a.shape
        Ho, Wo = (H + 1) // 2, (W + 1) // 2
        out = np.zeros((w.shape[0], Ho, Wo))
        for o in range(w.shape[0]):
            for i in range(Ho):
                for j in range(Wo):
                    s = bias[o]
                    for c in range(C):
                        for di in range(3):
                            for dj in range(3):
                                r, q = 2 * i + di - 1, 2 * j + dj - 1
                                if 0 <= r < H and 0 <= q < W:
                                    s += w[o, c, di, dj] * a[c, r, q]
                    out[o, i, j] = max(s, 0.0)
        return out

    a = conv(x[0], p["conv1.w"], p["conv1.b"])
    a = conv(a, p["conv2.w"], p["conv2.b"])
    a = conv(a, p["conv3.w"], p["conv3.b"])
    f = list(a.ravel()) + list(m[0])
    h = [max(p["fc1.b"][o] + sum(p["fc1.w"][o, i] * f[i] for i in range(1286)), 0.0) for o in range(128)]
    yy = [p["fc2.b"][o] + sum(p["fc2.w"][o, i] * h[i] for i in range(128)) for o in range(8)]
    np.testing.assert_allclose(y[0], yy, rtol=1e-10, atol=1e-12)


def test_gradients_match_finite_differences(nn):
    rng = np.random.default_rng(2)
    p = nn.init_params(5)
    for k in p:
        p[k] = p[k] + 0.05 * rng.normal(size=p[k].shape)
    x = rng.normal(size=(3, 1, 30, 40))
    m = rng.normal(size=(3, 6))
    t = rng.normal(size=(3, 8))
    y, cache = nn.forward(p, x, m)
    g, dx, dm = nn.backward(p, cache, y, t)
    flat = nn.flatten(p)
    gflat = nn.flatten(g)
    eps = 1e-6
    # every bias, plus 400 random weights spread over all layers
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in nn.SHAPES])
    idx = []
    for (name, shape), o0, o1 in zip(nn.SHAPES, offs[:-1], offs[1:]):
        idx += list(range(o0, o1)) if name.endswith(".b") else list(rng.integers(o0, o1, 40))
    idx += list(rng.integers(0, nn.N_PARAMS, 200))
    for i in idx:
        fp = flat.copy(); fp[i] += eps
        fm = flat.copy(); fm[i] -= eps
        Lp = nn.loss(nn.forward(nn.unflatten(fp), x, m)[0], t)
        Lm = nn.loss(nn.forward(nn.unflatten(fm), x, m)[0], t)
        fd = (Lp - Lm) / (2 * eps)
        assert abs(fd - gflat[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, gflat[i])
    for _ in range(30):
        b, r, c = rng.integers(3), rng.integers(30), rng.integers(40)
        xp = x.copy(); xp[b, 0, r, c] += eps
        xm = x.copy(); xm[b, 0, r, c] -= eps
        fd = (nn.loss(nn.forward(p, xp, m)[0], t) - nn.loss(nn.forward(p, xm, m)[0], t)) / (2 * eps)
        assert abs(fd - dx[b, 0, r, c]) <= 1e-6 * max(1.0, abs(fd))
    for b in range(3):
        for k in range(6):
            mp = m.copy(); mp[b, k] += eps
            mm = m.copy(); mm[b, k] -= eps
            fd = (nn.loss(nn.forward(p, x, mp)[0], t) - nn.loss(nn.forward(p, x, mm)[0], t)) / (2 * eps)
            assert abs(fd - dm[b, k]) <= 1e-6 * max(1.0, abs(fd))


def test_first_adam_step_closed_form(nn):
    rng = np.random.default_rng(3)
    p = nn.init_params(1)
    g = {k: rng.normal(size=v.shape) for k, v in p.items()}
    before = {k: v.copy() for k, v in p.items()}
    nn.adam_step(p, g, {}, lr=1e-3)
    for k in p:
        # t = 1: m_hat = g, v_hat = g^2, step = lr * g / (|g| + eps)
        np.testing.assert_allclose(p[k], before[k] - 1e-3 * g[k] / (np.abs(g[k]) + 1e-8), rtol=1e-12)


def test_bf16_rounding_matches_torch(nn):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    a = (rng.normal(size=5000) * 10.0 ** rng.integers(-6, 6, 5000)).astype(np.float32)
    ref = torch.from_numpy(a).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(nn.to_bf16(a), ref)


def test_parameter_count(nn):
    assert nn.N_PARAMS == 189064
    p = nn.init_params(0)
    np.testing.assert_array_equal(nn.flatten(nn.unflatten(nn.flatten(p))), nn.flatten(p))
