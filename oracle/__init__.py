"""FP64 CPU oracle of pose-only direct photometric tracking (GLidE-SLAM, Sec. IV).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg may import this package; the product
path (``paper_2607_16897_gb300``) never does and shares no code with it.

The arithmetic lives in ``oracle.c`` (plain C, FP64, compiled here with gcc);
this module only marshals numpy arrays into it and mirrors the library's API
(`build_pyramid`, `set_map_points`, `track_frame`, `debug_linearize`) so tests
can run both sides on the same inputs.  ``nn.py`` holds the FP64 oracle of the
learned initial-pose proposal.

Parity status of each function (what pins it is listed in the tests):
  pyramid           pinned: brute-force 2-D convolution, closed-form cases
  se3_exp / log     pinned: scipy matrix exponential / logarithm, round trips
  ref_patch         pinned: exact bilinear values on affine-ramp images
  linearize         pinned: dense-J brute force, finite differences on a ramp
                    image, zero residual on identical frames, PSD/symmetry
  track             pinned: pure-affine recovery, known-pose recovery on
                    rendered pairs, first-order optimality, cost-grid minimum
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

TOO_FEW_POINTS = 1
NOT_PD = 2
DIVERGED = 4

PATTERN = np.array([[0, 0], [-2, 0], [2, 0], [0, -2], [0, 2], [-1, -1], [1, -1], [-1, 1]])


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` next to its source with gcc (FP contraction off
    so the x86 and Arm builds round identically)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Cam(ctypes.Structure):
    _fields_ = [("fx", ctypes.c_double), ("fy", ctypes.c_double), ("cx", ctypes.c_double),
                ("cy", ctypes.c_double)]


class _Config(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int), ("max_iters", ctypes.c_int * 8),
                ("huber_k", ctypes.c_double), ("lambda0", ctypes.c_double),
                ("lambda_up", ctypes.c_double), ("lambda_down", ctypes.c_double),
                ("eps_step", ctypes.c_double), ("eps_step_coarse", ctypes.c_double),
                ("eps_cost", ctypes.c_double),
                ("accept_step", ctypes.c_double), ("min_valid", ctypes.c_int),
                ("zmin", ctypes.c_double), ("ic", ctypes.c_int), ("pattern", ctypes.c_int),
                ("affine", ctypes.c_int), ("hcache", ctypes.c_int)]


class _Result(ctypes.Structure):
    _fields_ = [("T", ctypes.c_double * 12), ("a", ctypes.c_double), ("b", ctypes.c_double),
                ("cost", ctypes.c_double), ("n_valid", ctypes.c_int),
                ("iters_total", ctypes.c_int), ("iters", ctypes.c_int * 8),
                ("passes", ctypes.c_int), ("status", ctypes.c_int)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER
            d, i = ctypes.c_double, ctypes.c_int
            dp, u8p, fp, ip = P(ctypes.c_double), P(ctypes.c_uint8), P(ctypes.c_float), P(ctypes.c_int)
            lib.orc_pyr_down.argtypes = [u8p, i, i, i, u8p]
            lib.orc_build_pyramid.argtypes = [u8p, i, i, i, i, u8p]
            lib.orc_se3_exp.argtypes = [dp, dp]
            lib.orc_se3_log.argtypes = [dp, dp]
            lib.orc_se3_mul.argtypes = [dp, dp, dp]
            lib.orc_backproject.argtypes = [_Cam, fp, i, dp]
            lib.orc_ref_patch.argtypes = [dp, i, i, i, fp, i, dp, u8p]
            lib.orc_linearize.argtypes = [dp, i, i, _Cam, i, dp, dp, u8p, i, dp, d, d, d, d,
                                          dp, dp, dp, ip, dp, dp, dp, u8p]
            lib.orc_track.argtypes = [dp, i, i, _Cam, dp, dp, u8p, i, P(_Config), dp, d, d,
                                      P(_Result), dp, ip, dp, i]
            lib.orc_ic_jacobian.argtypes = [dp, i, i, _Cam, i, dp, fp, u8p, i, i, dp]
            lib.orc_linearize2.argtypes = [dp, i, i, _Cam, i, dp, dp, u8p, dp, i, i, dp, d, d, d,
                                           d, dp, dp, dp, ip, dp, dp, dp, u8p]
            lib.orc_ref_patch2.argtypes = [dp, i, i, i, fp, i, i, dp, u8p]
            lib.orc_ic_hessian.argtypes = [dp, u8p, i, i, dp]
            lib.orc_ic_hessian.restype = None
            lib.orc_pattern.argtypes = [i, ip, ip]
            lib.orc_pattern.restype = i
            lib.orc_ref_patch2.restype = None
            lib.orc_track2.argtypes = [dp, i, i, _Cam, dp, dp, u8p, dp, i, P(_Config), dp, d, d,
                                       P(_Result), dp, ip, dp, i]
            for fn in (lib.orc_pyr_down, lib.orc_build_pyramid, lib.orc_se3_exp, lib.orc_se3_log,
                       lib.orc_se3_mul, lib.orc_backproject, lib.orc_ref_patch,
                       lib.orc_linearize, lib.orc_track, lib.orc_ic_jacobian,
                       lib.orc_linearize2, lib.orc_track2):
                fn.restype = None
            _lib = lib
    return _lib


def _p(a, ct):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ct))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def level_dims(W: int, H: int, L: int):
    dims = []
    for _ in range(L):
        dims.append((W, H))
        W //= 2
        H //= 2
    return dims


# --------------------------------------------------------------------------
# pyramid
# --------------------------------------------------------------------------
def pyr_down(img: np.ndarray) -> np.ndarray:
    img = np.ascontiguousarray(img, np.uint8)
    H, W = img.shape
    out = np.zeros((H // 2, W // 2), np.uint8)
    _load().orc_pyr_down(_p(img, ctypes.c_uint8), W, H, W, _p(out, ctypes.c_uint8))
    return out


def pyramid(img: np.ndarray, L: int) -> list:
    img = np.ascontiguousarray(img, np.uint8)
    H, W = img.shape
    dims = level_dims(W, H, L)
    flat = np.zeros(sum(w * h for w, h in dims), np.uint8)
    _load().orc_build_pyramid(_p(img, ctypes.c_uint8), W, H, W, L, _p(flat, ctypes.c_uint8))
    out, o = [], 0
    for w, h in dims:
        out.append(flat[o:o + w * h].reshape(h, w).copy())
        o += w * h
    return out


# --------------------------------------------------------------------------
# SE(3)
# --------------------------------------------------------------------------
def se3_exp(xi) -> np.ndarray:
    xi = _f64(xi).reshape(6)
    T = np.zeros(12)
    _load().orc_se3_exp(_p(xi, ctypes.c_double), _p(T, ctypes.c_double))
    return T.reshape(3, 4)


def se3_log(T) -> np.ndarray:
    T = _f64(T).reshape(12)
    xi = np.zeros(6)
    _load().orc_se3_log(_p(T, ctypes.c_double), _p(xi, ctypes.c_double))
    return xi


def se3_mul(A, B) -> np.ndarray:
    A = _f64(A).reshape(12)
    B = _f64(B).reshape(12)
    C = np.zeros(12)
    _load().orc_se3_mul(_p(A, ctypes.c_double), _p(B, ctypes.c_double), _p(C, ctypes.c_double))
    return C.reshape(3, 4)


# --------------------------------------------------------------------------
# points, reference patches, linearisation
# --------------------------------------------------------------------------
def _cam(K) -> _Cam:
    fx, fy, cx, cy = K
    return _Cam(float(fx), float(fy), float(cx), float(cy))


def backproject(K, uvd) -> np.ndarray:
    uvd = np.ascontiguousarray(uvd, np.float32).reshape(-1, 3)
    N = uvd.shape[0]
    x = np.zeros((N, 3))
    _load().orc_backproject(_cam(K), _p(uvd, ctypes.c_float), N, _p(x, ctypes.c_double))
    return x


def pattern_offsets(pattern: int = 0):
    """(dx, dy) of the pattern's samples: 0 = the 8-pixel pattern, odd p = p x p."""
    dx = np.zeros(121, np.int32)
    dy = np.zeros(121, np.int32)
    K = _load().orc_pattern(int(pattern), _p(dx, ctypes.c_int), _p(dy, ctypes.c_int))
    if K == 0:
        raise ValueError(f"unknown pattern {pattern}")
    return dx[:K].copy(), dy[:K].copy()


def ref_patch(img_l, level: int, uvd, pattern: int = 0):
    """I0 [N, K] and validity [N] of one level (K samples of the pattern).
    img_l: the level image (any real dtype, converted exactly to double)."""
    img = _f64(img_l)
    H, W = img.shape
    uvd = np.ascontiguousarray(uvd, np.float32).reshape(-1, 3)
    N = uvd.shape[0]
    K = len(pattern_offsets(pattern)[0])
    I0 = np.zeros((N, K))
    valid = np.zeros(N, np.uint8)
    _load().orc_ref_patch2(_p(img, ctypes.c_double), W, H, level, _p(uvd, ctypes.c_float), N,
                           int(pattern), _p(I0, ctypes.c_double), _p(valid, ctypes.c_uint8))
    return I0, valid


def ic_jacobian(ref_l, K0, level, x_r, uvd, valid_l, pattern: int = 0):
    """Inverse-compositional cache of one level: [N, K, 6] reference-side
    pose Jacobian rows (zero for unusable points)."""
    img = _f64(ref_l)
    H, W = img.shape
    x_r = _f64(x_r)
    N = x_r.shape[0]
    uvd = np.ascontiguousarray(uvd, np.float32).reshape(-1, 3)
    valid_l = np.ascontiguousarray(valid_l, np.uint8)
    K = len(pattern_offsets(pattern)[0])
    out = np.zeros(N * K * 6)
    _load().orc_ic_jacobian(_p(img, ctypes.c_double), W, H, _cam(K0), int(level),
                            _p(x_r, ctypes.c_double), _p(uvd, ctypes.c_float),
                            _p(valid_l, ctypes.c_uint8), N, int(pattern), _p(out, ctypes.c_double))
    return out.reshape(N, K, 6)


def ic_hessian(Jic_l, valid_l) -> np.ndarray:
    """Per-reference Hessian [6, 6] of one level from its IC cache [N, K, 6]."""
    J = _f64(Jic_l)
    N, K = J.shape[0], J.shape[1]
    valid_l = np.ascontiguousarray(valid_l, np.uint8)
    H6 = np.zeros(36)
    _load().orc_ic_hessian(_p(J, ctypes.c_double), _p(valid_l, ctypes.c_uint8), N, K,
                           _p(H6, ctypes.c_double))
    return H6.reshape(6, 6)


def linearize(img_l, K0, level, x_r, I0_l, valid_l, T, a, b, huber_k=9.0, zmin=1e-3,
              per_sample=True, Jic=None, pattern=0):
    img = _f64(img_l)
    H, W = img.shape
    x_r = _f64(x_r)
    N = x_r.shape[0]
    K = len(pattern_offsets(pattern)[0])
    I0_l = _f64(I0_l).reshape(N * K)
    valid_l = np.ascontiguousarray(valid_l, np.uint8)
    T = _f64(T).reshape(12)
    Hm = np.zeros(64)
    g = np.zeros(8)
    E = ctypes.c_double()
    n = ctypes.c_int()
    res = jac = wts = pv = None
    if per_sample:
        res = np.zeros(N * K)
        jac = np.zeros(N * K * 8)
        wts = np.zeros(N * K)
        pv = np.zeros(N, np.uint8)
    Jic = None if Jic is None else _f64(Jic).reshape(N * K * 6)
    _load().orc_linearize2(_p(img, ctypes.c_double), W, H, _cam(K0), int(level),
                          _p(x_r, ctypes.c_double), _p(I0_l, ctypes.c_double),
                          _p(valid_l, ctypes.c_uint8), _p(Jic, ctypes.c_double), N,
                          int(pattern), _p(T, ctypes.c_double), float(a),
                          float(b), float(huber_k), float(zmin), _p(Hm, ctypes.c_double),
                          _p(g, ctypes.c_double), ctypes.byref(E), ctypes.byref(n),
                          _p(res, ctypes.c_double), _p(jac, ctypes.c_double),
                          _p(wts, ctypes.c_double), _p(pv, ctypes.c_uint8))
    out = {"H": Hm.reshape(8, 8), "g": g, "E": E.value, "n": n.value}
    if per_sample:
        out.update(res=res.reshape(N, K), J=jac.reshape(N, K, 8), w=wts.reshape(N, K),
                   point_valid=pv.astype(bool))
    return out


# --------------------------------------------------------------------------
# configuration and tracking
# --------------------------------------------------------------------------
DEFAULT_CONFIG = dict(levels=4, max_iters=[10] * 8, huber_k=9.0, lambda0=1e-4, lambda_up=4.0,
                      lambda_down=0.5, eps_step=1e-6, eps_step_coarse=3e-4, eps_cost=0.0, accept_step=1e-3,
                      min_valid=16, zmin=1e-3, jacobian="forward", pattern=0, affine=True,
                      hessian="pass")


def make_config(**kw) -> dict:
    c = dict(DEFAULT_CONFIG)
    c.update(kw)
    mi = list(c["max_iters"])
    c["max_iters"] = (mi + [mi[-1]] * 8)[:8]
    return c


def _cconfig(c: dict) -> _Config:
    cc = _Config()
    cc.levels = int(c["levels"])
    for i in range(8):
        cc.max_iters[i] = int(c["max_iters"][i])
    cc.huber_k = float(c["huber_k"])
    cc.lambda0 = float(c["lambda0"])
    cc.lambda_up = float(c["lambda_up"])
    cc.lambda_down = float(c["lambda_down"])
    cc.eps_step = float(c["eps_step"])
    cc.eps_step_coarse = float(c["eps_step_coarse"])
    cc.eps_cost = float(c["eps_cost"])
    cc.accept_step = float(c["accept_step"])
    cc.min_valid = int(c["min_valid"])
    cc.zmin = float(c["zmin"])
    cc.ic = {"forward": 0, "ic": 1}[c["jacobian"]]
    cc.pattern = int(c["pattern"])
    cc.affine = 1 if c["affine"] else 0
    cc.hcache = {"pass": 0, "cached": 1}[c["hessian"]]
    return cc


def track(cur_levels, K0, x_r, I0, valid, cfg: dict, T_init, a0=0.0, b0=0.0, Jic=None) -> dict:
    """cur_levels: list of level images; I0 [L, N, 8]; valid [L, N]; Jic
    [L, N, 8, 6] (inverse-compositional cache, needed when cfg jacobian = ic)."""
    L = int(cfg["levels"])
    H0, W0 = np.asarray(cur_levels[0]).shape
    flat = np.concatenate([_f64(cur_levels[l]).ravel() for l in range(L)])
    x_r = _f64(x_r)
    N = x_r.shape[0]
    K = len(pattern_offsets(cfg["pattern"])[0])
    I0 = _f64(I0).reshape(L, N, K)
    valid = np.ascontiguousarray(valid, np.uint8).reshape(L, N)
    T = _f64(T_init).reshape(12)
    cc = _cconfig(cfg)
    r = _Result()
    mt = L * (1 + max(cfg["max_iters"][:L]))
    tc = np.zeros(max(mt, 1))
    ti = np.zeros(max(mt, 1), np.int32)
    ts = np.zeros(max(mt, 1))
    if cfg["jacobian"] == "ic" and Jic is None:
        raise ValueError("the inverse-compositional solve needs its Jacobian cache")
    Jic = None if Jic is None else _f64(Jic).reshape(L * N * K * 6)
    _load().orc_track2(_p(flat, ctypes.c_double), W0, H0, _cam(K0), _p(x_r, ctypes.c_double),
                      _p(I0, ctypes.c_double), _p(valid, ctypes.c_uint8), _p(Jic, ctypes.c_double),
                      N, ctypes.byref(cc),
                      _p(T, ctypes.c_double), float(a0), float(b0), ctypes.byref(r),
                      _p(tc, ctypes.c_double), _p(ti, ctypes.c_int), _p(ts, ctypes.c_double), mt)
    n = min(r.passes, mt)
    trace = [dict(cost=float(tc[k]), level=int(ti[k]) >> 2, accepted=bool(ti[k] & 2),
                  candidate=bool(ti[k] & 1), step=float(ts[k])) for k in range(n)]
    return {"T": np.array(r.T[:]).reshape(3, 4), "a": r.a, "b": r.b, "cost": r.cost,
            "n_valid": r.n_valid, "iters_total": r.iters_total, "iters": list(r.iters[:L]),
            "passes": r.passes, "status": r.status, "trace": trace}


class OracleTracker:
    """The oracle behind the same calls as the CUDA library's tracker:
    build_pyramid(slot, img), set_map_points(uvd), track_frame(T_init, ab_init),
    debug_linearize(level, T, a, b)."""

    REF, CUR = 0, 1

    def __init__(self, W, H, K, **cfg):
        self.W, self.H, self.K = int(W), int(H), tuple(float(k) for k in K)
        self.cfg = make_config(**cfg)
        self.L = int(self.cfg["levels"])
        self.pyr = [None, None]
        self.x_r = None
        self.I0 = None
        self.valid = None
        self.Jic = None

    def build_pyramid(self, slot: int, img) -> None:
        img = np.ascontiguousarray(img, np.uint8)
        assert img.shape == (self.H, self.W)
        self.pyr[slot] = pyramid(img, self.L)

    def set_map_points(self, uvd) -> None:
        if self.pyr[self.REF] is None:
            raise RuntimeError("reference pyramid not built")
        uvd = np.ascontiguousarray(uvd, np.float32).reshape(-1, 3)
        self.uvd = uvd
        self.x_r = backproject(self.K, uvd)
        N = uvd.shape[0]
        pat = self.cfg["pattern"]
        K = len(pattern_offsets(pat)[0])
        self.I0 = np.zeros((self.L, N, K))
        self.valid = np.zeros((self.L, N), np.uint8)
        for l in range(self.L):
            self.I0[l], self.valid[l] = ref_patch(self.pyr[self.REF][l], l, uvd, pat)
        self.Jic = None
        if self.cfg["jacobian"] == "ic":
            self.Jic = np.stack([ic_jacobian(self.pyr[self.REF][l], self.K, l, self.x_r, uvd,
                                             self.valid[l], pat) for l in range(self.L)])

    def cached_hessian(self, level):
        """The per-reference Hessian [6, 6] of a level (jacobian "ic")."""
        return ic_hessian(self.Jic[level], self.valid[level])

    def debug_linearize(self, level, T, a, b, per_sample=True):
        """The normal equations a pass of the solve uses: with hessian
        "cached", H is e^{2a} times the per-reference Hessian (pose block; the
        affine rows, unused, are zero) and g keeps its pose part."""
        out = linearize(self.pyr[self.CUR][level], self.K, level, self.x_r, self.I0[level],
                        self.valid[level], T, a, b, self.cfg["huber_k"], self.cfg["zmin"],
                        per_sample, Jic=None if self.Jic is None else self.Jic[level],
                        pattern=self.cfg["pattern"])
        if self.cfg["hessian"] == "cached":
            Hm = np.zeros((8, 8))
            Hm[:6, :6] = np.exp(2.0 * a) * self.cached_hessian(level)
            out["H"] = Hm
            out["g"] = out["g"].copy()
            out["g"][6:] = 0.0
        return out

    def track_frame(self, T_init, ab_init=(0.0, 0.0)) -> dict:
        return track(self.pyr[self.CUR], self.K, self.x_r, self.I0, self.valid, self.cfg,
                     T_init, float(ab_init[0]), float(ab_init[1]), Jic=self.Jic)
