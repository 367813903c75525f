"""FP64 oracle of the learned initial-pose proposal network.

TEST INFRASTRUCTURE ONLY (same rules as the rest of ``oracle/``).

The proposal is not in the paper; the network is this library's: a
3 x (conv 3x3, stride 2, zero padding 1, ReLU) + 2-layer MLP that maps the
coarsest-level residual image (1 x 30 x 40) and the previous inter-frame motion
(6 values) to an 8-vector increment.  Shapes:

    x  [B, 1, 30, 40] --conv1--> [B, 16, 15, 20] --conv2--> [B, 32, 8, 10]
       --conv3--> [B, 64, 4, 5] --flatten++m--> [B, 1286] --fc1--> [B, 128]
       --fc2--> [B, 8]

Loss: 0.5 * mean over the batch of sum_k (y_k - t_k)^2.

Flat parameter layout (an interface both implementations follow): conv1.w
[16,1,3,3], conv1.b [16], conv2.w [32,16,3,3], conv2.b [32], conv3.w
[64,32,3,3], conv3.b [64], fc1.w [128,1286], fc1.b [128], fc2.w [8,128],
fc2.b [8], each row-major, concatenated in that order (189064 values).

Inputs and outputs of the proposal (the network's interface to the tracker):
the motion input is log(M) / MOTION_SCALE with M = T_{k-1} T_{k-2}^-1 the last
inter-frame camera motion (world -> camera poses), and the output y is the
increment delta = OUT_SCALE * y, applied to the constant-velocity start as
T' = T_init exp(delta[0:6]), a' = a + delta[6], b' = b + delta[7].  The SE(3)
arithmetic is the FP64 oracle's (``oracle.se3_log / se3_exp / se3_mul``).

Parity status: pinned by central finite differences of the loss in FP64 (all
parameters and inputs), by a library 2-D correlation (scipy) for the
convolution, and by numpy matmul for the fully connected layers; the motion
feature and the composition of the output by scipy's matrix logarithm and
exponential.
"""
from __future__ import annotations

import numpy as np

SHAPES = [("conv1.w", (16, 1, 3, 3)), ("conv1.b", (16,)),
          ("conv2.w", (32, 16, 3, 3)), ("conv2.b", (32,)),
          ("conv3.w", (64, 32, 3, 3)), ("conv3.b", (64,)),
          ("fc1.w", (128, 1286)), ("fc1.b", (128,)),
          ("fc2.w", (8, 128)), ("fc2.b", (8,))]
N_PARAMS = int(sum(np.prod(s) for _, s in SHAPES))
MOTION_SCALE = 0.02                          # motion input = log(M) / MOTION_SCALE
OUT_SCALE = np.array([0.01] * 7 + [1.0])     # increment = OUT_SCALE * y


def _inverse34(T):
    T = np.asarray(T, np.float64).reshape(3, 4)
    R = T[:, :3].T
    return np.hstack([R, (-R @ T[:, 3])[:, None]])


def motion_input(M):
    """Network motion input from the last inter-frame motion M (3x4)."""
    import oracle
    return oracle.se3_log(M) / MOTION_SCALE


def motion_feature(Tw_prev, Tw_prevprev):
    """Motion input from the two previous world -> camera poses (zeros when
    either is missing): log(T_{k-1} T_{k-2}^-1) / MOTION_SCALE."""
    import oracle
    if Tw_prev is None or Tw_prevprev is None:
        return np.zeros(6)
    return motion_input(oracle.se3_mul(Tw_prev, _inverse34(Tw_prevprev)))


def apply_output(T_init, ab_init, y):
    """Start state proposed by output y: (T_init exp(delta[0:6]),
    (a + delta[6], b + delta[7])) with delta = OUT_SCALE * y."""
    import oracle
    d = np.asarray(y, np.float64).reshape(8) * OUT_SCALE
    T = oracle.se3_mul(T_init, oracle.se3_exp(d[:6]))
    return T, (float(ab_init[0]) + d[6], float(ab_init[1]) + d[7])


def unflatten(flat):
    flat = np.asarray(flat, dtype=np.float64)
    assert flat.size == N_PARAMS
    out, o = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = flat[o:o + n].reshape(shape)
        o += n
    return out


def flatten(params):
    return np.concatenate([np.asarray(params[name], np.float64).ravel() for name, _ in SHAPES])


def init_params(seed=0):
    """He-uniform weights, zero biases (float64)."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shape in SHAPES:
        if name.endswith(".b"):
            p[name] = np.zeros(shape)
        else:
            fan_in = int(np.prod(shape[1:]))
            lim = np.sqrt(6.0 / fan_in)
            p[name] = rng.uniform(-lim, lim, size=shape)
    return p


def conv2d_s2(x, w, b):
    """out[b,o,i,j] = b_o + sum_{c,di,dj} w[o,c,di,dj] x[b,c,2i+di-1,2j+dj-1],
    zero outside the input (stride 2, padding 1)."""
    B, C, H, W = x.shape
    O = w.shape[0]
    Ho, Wo = (H + 1) // 2, (W + 1) // 2
    xp = np.zeros((B, C, H + 2, W + 2))
    xp[:, :, 1:H + 1, 1:W + 1] = x
    out = np.zeros((B, O, Ho, Wo)) + b[None, :, None, None]
    for di in range(3):
        for dj in range(3):
            patch = xp[:, :, di:di + 2 * Ho:2, dj:dj + 2 * Wo:2]          # [B, C, Ho, Wo]
            out += np.einsum("oc,bcij->boij", w[:, :, di, dj], patch)
    return out


def conv2d_s2_backward(x, w, dout):
    """Gradients of conv2d_s2 with respect to x, w and b."""
    B, C, H, W = x.shape
    Ho, Wo = dout.shape[2], dout.shape[3]
    xp = np.zeros((B, C, H + 2, W + 2))
    xp[:, :, 1:H + 1, 1:W + 1] = x
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for di in range(3):
        for dj in range(3):
            patch = xp[:, :, di:di + 2 * Ho:2, dj:dj + 2 * Wo:2]
            dw[:, :, di, dj] = np.einsum("boij,bcij->oc", dout, patch)
            dxp[:, :, di:di + 2 * Ho:2, dj:dj + 2 * Wo:2] += np.einsum("oc,boij->bcij", w[:, :, di, dj], dout)
    return dxp[:, :, 1:H + 1, 1:W + 1], dw, dout.sum(axis=(0, 2, 3))


def forward(params, x, m):
    """x [B,1,30,40], m [B,6] -> (y [B,8], cache)."""
    x = np.asarray(x, np.float64)
    m = np.asarray(m, np.float64)
    z1 = conv2d_s2(x, params["conv1.w"], params["conv1.b"])
    a1 = np.maximum(z1, 0.0)
    z2 = conv2d_s2(a1, params["conv2.w"], params["conv2.b"])
    a2 = np.maximum(z2, 0.0)
    z3 = conv2d_s2(a2, params["conv3.w"], params["conv3.b"])
    a3 = np.maximum(z3, 0.0)
    f = np.concatenate([a3.reshape(a3.shape[0], -1), m], axis=1)        # [B, 1286]
    z4 = f @ params["fc1.w"].T + params["fc1.b"]
    h = np.maximum(z4, 0.0)
    y = h @ params["fc2.w"].T + params["fc2.b"]
    return y, dict(x=x, m=m, z1=z1, a1=a1, z2=z2, a2=a2, z3=z3, a3=a3, f=f, z4=z4, h=h)


def loss(y, t):
    t = np.asarray(t, np.float64)
    return 0.5 * np.mean(np.sum((y - t) ** 2, axis=1))


def backward(params, cache, y, t):
    """Gradient of loss(y, t) with respect to every parameter (dict) and the inputs."""
    B = y.shape[0]
    dy = (y - np.asarray(t, np.float64)) / B
    g = {}
    g["fc2.w"] = dy.T @ cache["h"]
    g["fc2.b"] = dy.sum(0)
    dh = dy @ params["fc2.w"]
    dz4 = dh * (cache["z4"] > 0)
    g["fc1.w"] = dz4.T @ cache["f"]
    g["fc1.b"] = dz4.sum(0)
    df = dz4 @ params["fc1.w"]
    dm = df[:, 1280:]
    da3 = df[:, :1280].reshape(cache["a3"].shape)
    dz3 = da3 * (cache["z3"] > 0)
    da2, g["conv3.w"], g["conv3.b"] = conv2d_s2_backward(cache["a2"], params["conv3.w"], dz3)
    dz2 = da2 * (cache["z2"] > 0)
    da1, g["conv2.w"], g["conv2.b"] = conv2d_s2_backward(cache["a1"], params["conv2.w"], dz2)
    dz1 = da1 * (cache["z1"] > 0)
    dx, g["conv1.w"], g["conv1.b"] = conv2d_s2_backward(cache["x"], params["conv1.w"], dz1)
    return g, dx, dm


def adam_step(params, grads, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba) of FP64 master weights in place."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for name, _ in SHAPES:
        mom = state.setdefault("m." + name, np.zeros_like(params[name]))
        var = state.setdefault("v." + name, np.zeros_like(params[name]))
        gr = grads[name]
        mom[...] = b1 * mom + (1 - b1) * gr
        var[...] = b2 * var + (1 - b2) * gr * gr
        mh = mom / (1 - b1 ** t)
        vh = var / (1 - b2 ** t)
        params[name] = params[name] - lr * mh / (np.sqrt(vh) + eps)
    return params


def to_bf16(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    a32 = np.asarray(a, np.float32)
    u = a32.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)
