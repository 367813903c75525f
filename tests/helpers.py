"""Test-side helpers: run the CUDA library and the FP64 oracle on the same
seeded inputs and compare them with the parity tolerances."""
import numpy as np

I34 = np.hstack([np.eye(3), np.zeros((3, 1))])

# parity tolerances (gray levels, relative, radians, metres)
RES_TOL = 1e-3
RES_FP32 = 1e-4      # FP32 rounding of one residual sample (projection + interpolation)
H_TOL = 1e-5
G_TOL = 1e-5
ROT_TOL = 1e-5
TRANS_TOL = 1e-5
A_TOL = 1e-5
B_TOL = 1e-3


def both_sides(glt, oracle, W, H, K, ref, cur, uvd, device_inputs=False, **cfg):
    """A GPU Tracker and an OracleTracker set up on the same inputs."""
    import torch
    L = cfg.get("levels", 4)
    gcfg = dict(cfg)
    gcfg.setdefault("max_points", max(len(uvd), 1))
    trk = glt.Tracker(W, H, K, **gcfg)
    ocfg = {k: v for k, v in cfg.items() if k in oracle.DEFAULT_CONFIG}
    orc = oracle.OracleTracker(W, H, K, **ocfg)
    if device_inputs:
        trk.build_pyramid(glt.GLT_REF, torch.from_numpy(np.ascontiguousarray(ref)).cuda())
        trk.set_map_points(torch.from_numpy(np.ascontiguousarray(uvd, np.float32)).cuda())
        trk.build_pyramid(glt.GLT_CUR, torch.from_numpy(np.ascontiguousarray(cur)).cuda())
        torch.cuda.synchronize()
    else:
        trk.build_pyramid(glt.GLT_REF, ref)
        trk.set_map_points(uvd)
        trk.build_pyramid(glt.GLT_CUR, cur)
    orc.build_pyramid(0, ref)
    orc.set_map_points(uvd)
    orc.build_pyramid(1, cur)
    assert orc.L == L
    return trk, orc


def pose_diff(Ta, Tb):
    dR = Ta[:, :3].T @ Tb[:, :3]
    s = 0.5 * np.linalg.norm([dR[2, 1] - dR[1, 2], dR[0, 2] - dR[2, 0], dR[1, 0] - dR[0, 1]])
    ang = float(np.arctan2(s, 0.5 * (np.trace(dR) - 1.0)))
    return ang, float(np.linalg.norm(Ta[:, 3] - Tb[:, 3]))


def compare_linearization(g, o, where=""):
    """g: GPU debug_linearize dict (with res), o: oracle linearize dict (per sample)."""
    gres = g["res"].astype(np.float64)
    ores = o["res"]
    gv = ~np.isnan(gres[:, 0])
    ov = o["point_valid"]
    assert (gv == ov).all(), f"{where}: point validity differs at {np.where(gv != ov)[0][:10]}"
    assert g["n"] == o["n"], where
    if o["n"] == 0:
        return {}
    d = np.abs(gres[ov] - ores[ov]).max()
    assert d <= RES_TOL, f"{where}: residual diff {d}"
    dH = np.linalg.norm(g["H"] - o["H"]) / np.linalg.norm(o["H"])
    assert dH <= H_TOL, f"{where}: H rel diff {dH}"
    # g = J^T W r: 1e-5 of sum |w J r| (the scale of its terms; g itself -> 0 at
    # the optimum), plus the FP32 residual rounding RES_FP32 per sample, which
    # adds in quadrature over the samples (it only matters for a handful of points)
    wJ = o["J"][ov] * o["w"][ov][:, :, None]
    absg = np.abs(wJ * o["res"][ov][:, :, None]).sum((0, 1))
    quad = np.sqrt((wJ ** 2).sum((0, 1)))
    tol = G_TOL * np.linalg.norm(absg) + 3 * RES_FP32 * np.linalg.norm(quad)
    dg = np.linalg.norm(g["g"] - o["g"]) / np.linalg.norm(absg)
    assert np.linalg.norm(g["g"] - o["g"]) <= tol, f"{where}: g diff {dg} (res diff {d})"
    # E = sum rho(r): same reading as g, d rho = w r dr adds in quadrature
    wr = (o["w"][ov] * o["res"][ov]).ravel()
    dE = abs(g["E"] - o["E"]) / max(o["E"], 1e-30)
    assert abs(g["E"] - o["E"]) <= 1e-5 * o["E"] + 3 * RES_FP32 * np.sqrt((wr ** 2).sum()), \
        f"{where}: E diff {dE}"
    return {"res": d, "H": dH, "g": dg, "E": dE}


def ambiguous_points(oracle, orc, level, T, tol_px=1e-3):
    """Points whose FP64 projection puts a pattern sample within tol_px of a
    validity bound (the two precisions may legitimately decide differently)."""
    K = orc.K
    s = 2.0 ** -level
    W, H = orc.W >> level, orc.H >> level
    xc = orc.x_r @ T[:, :3].T + T[:, 3]
    u = K[0] * s * xc[:, 0] / xc[:, 2] + K[2] * s
    v = K[1] * s * xc[:, 1] / xc[:, 2] + K[3] * s
    amb = np.zeros(len(u), bool)
    for lo, hi, q in ((3, W - 4, u), (3, H - 4, v)):
        # sample-0 coordinate must satisfy lo <= q < hi (pattern +-2, taps, gradients)
        amb |= (np.abs(q - lo) < tol_px) | (np.abs(q - hi) < tol_px)
    return amb
