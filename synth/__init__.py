"""Seeded synthetic inputs shared by the FP64 oracle tests and the CUDA path.

What lives here manufactures inputs only: rendered uint8 frames of a textured
box room, exact depth, sparse map points, smooth camera trajectories and
per-frame exposure.  None of the tracker's arithmetic (pyramid, projection
Jacobians, residuals, solver, SE(3) exponential) is implemented here; poses
are built from unit quaternions and composed as plain 3x4 matrices.

The renderer is C (``render.c``) compiled on first use with gcc, so that it
runs at the same speed on the x86 development host and the Arm GPU host.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "render.c")
_LIB_PATH = os.path.join(_HERE, "libsynth.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``libsynth.so`` next to its source (gcc, OpenMP if available)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    base = ["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-std=c11"]
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    try:
        subprocess.check_call(base + ["-fopenmp", "-o", tmp, _SRC, "-lm"])
    except subprocess.CalledProcessError:
        subprocess.check_call(base + ["-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Scene(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
                ("light", ctypes.c_double * 3), ("ambient", ctypes.c_double),
                ("base_freq", ctypes.c_double), ("lacunarity", ctypes.c_double),
                ("gain", ctypes.c_double), ("contrast", ctypes.c_double),
                ("octaves", ctypes.c_int), ("pad_", ctypes.c_int),
                ("tex_seed", ctypes.c_uint64)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            u8p = ctypes.POINTER(ctypes.c_uint8)
            fp = ctypes.POINTER(ctypes.c_float)
            sp = ctypes.POINTER(_Scene)
            d = ctypes.c_double
            lib.synth_render.argtypes = [sp, dp, d, d, d, d, ctypes.c_int, ctypes.c_int, d, d, d,
                                         ctypes.c_uint64, u8p, fp, fp, u8p]
            lib.synth_render.restype = ctypes.c_int
            lib.synth_depth_at.argtypes = [sp, dp, d, d, d, d, d, d]
            lib.synth_depth_at.restype = ctypes.c_double
            lib.synth_select_points.argtypes = [sp, dp, d, d, d, d, u8p, fp, u8p, ctypes.c_int,
                                                ctypes.c_int, ctypes.c_int, d, d, ctypes.c_int,
                                                ctypes.c_int, ctypes.c_uint64, fp]
            lib.synth_select_points.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


# --------------------------------------------------------------------------
# scenes and cameras
# --------------------------------------------------------------------------
@dataclass
class Scene:
    lo: tuple
    hi: tuple
    tex_seed: int = 7
    ambient: float = 0.3
    base_freq: float = 2.0
    lacunarity: float = 2.0
    gain: float = 0.5
    contrast: float = 2.0
    octaves: int = 4

    def c(self) -> _Scene:
        s = _Scene()
        for i in range(3):
            s.lo[i] = self.lo[i]
            s.hi[i] = self.hi[i]
            s.light[i] = 0.5 * (self.lo[i] + self.hi[i])
        s.ambient = self.ambient
        s.base_freq = self.base_freq
        s.lacunarity = self.lacunarity
        s.gain = self.gain
        s.contrast = self.contrast
        s.octaves = self.octaves
        s.tex_seed = self.tex_seed
        return s


# small deep room seen from the origin looking down +z: floor, ceiling, both
# side walls and the far wall are all in view, depths ~2.1-5 m
ROOM_SMALL = Scene(lo=(-1.5, -1.0, -1.0), hi=(1.5, 1.0, 5.0))
# larger room for the sequence workloads (depths up to ~8 m)
ROOM_LARGE = Scene(lo=(-4.0, -1.6, -3.0), hi=(4.0, 1.6, 6.5))


@dataclass
class Camera:
    W: int
    H: int
    fx: float
    fy: float
    cx: float
    cy: float

    @property
    def K(self):
        return (self.fx, self.fy, self.cx, self.cy)


def camera_for(W: int, H: int, f: float | None = None) -> Camera:
    if f is None:
        f = 0.8 * W
    return Camera(W, H, float(f), float(f), W / 2.0, H / 2.0)


# --------------------------------------------------------------------------
# poses (plain 3x4 matrices; rotations from unit quaternions)
# --------------------------------------------------------------------------
def rot_from_axis_angle(axis, angle) -> np.ndarray:
    axis = np.asarray(axis, dtype=np.float64)
    n = np.linalg.norm(axis)
    if n == 0 or angle == 0:
        return np.eye(3)
    axis = axis / n
    w = np.cos(angle / 2.0)
    x, y, z = np.sin(angle / 2.0) * axis
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)],
    ])


def rot_from_vec(v) -> np.ndarray:
    v = np.asarray(v, dtype=np.float64)
    return rot_from_axis_angle(v, float(np.linalg.norm(v)))


def pose(R, t) -> np.ndarray:
    T = np.zeros((3, 4))
    T[:, :3] = R
    T[:, 3] = t
    return T


def pose_mul(A, B) -> np.ndarray:
    return pose(A[:, :3] @ B[:, :3], A[:, :3] @ B[:, 3] + A[:, 3])


def pose_inv(A) -> np.ndarray:
    R = A[:, :3].T
    return pose(R, -R @ A[:, 3])


def rotation_angle(R) -> float:
    c = (np.trace(R) - 1.0) / 2.0
    s = np.linalg.norm([R[2, 1] - R[1, 2], R[0, 2] - R[2, 0], R[1, 0] - R[0, 1]]) / 2.0
    return float(np.arctan2(s, c))


def relative(T_wc_ref, T_wc_cur) -> np.ndarray:
    """T_cr: maps reference-camera coordinates to current-camera coordinates."""
    return pose_mul(pose_inv(T_wc_cur), T_wc_ref)


# --------------------------------------------------------------------------
# rendering and point selection
# --------------------------------------------------------------------------
def render(scene: Scene, T_wc, cam: Camera, a=0.0, b=0.0, sigma=0.0, noise_seed=0,
           want_rad=False, want_wall=False):
    """Returns (img uint8 HxW, depth float32 HxW[, radiance float32 HxW]
    [, wall id uint8 HxW])."""
    lib = _load()
    T = np.ascontiguousarray(T_wc, dtype=np.float64).reshape(12)
    img = np.zeros((cam.H, cam.W), np.uint8)
    dep = np.zeros((cam.H, cam.W), np.float32)
    rad = np.zeros((cam.H, cam.W), np.float32) if want_rad else None
    wall = np.zeros((cam.H, cam.W), np.uint8) if want_wall else None
    sc = scene.c()
    rc = lib.synth_render(ctypes.byref(sc), _ptr(T, ctypes.c_double), cam.fx, cam.fy, cam.cx,
                          cam.cy, cam.W, cam.H, float(a), float(b), float(sigma),
                          int(noise_seed) & (2**64 - 1), _ptr(img, ctypes.c_uint8),
                          _ptr(dep, ctypes.c_float),
                          _ptr(rad, ctypes.c_float) if want_rad else None,
                          _ptr(wall, ctypes.c_uint8) if want_wall else None)
    if rc != 0:
        raise ValueError("camera is outside the room")
    out = (img, dep)
    if want_rad:
        out = out + (rad,)
    if want_wall:
        out = out + (wall,)
    return out


def depth_at(scene: Scene, T_wc, cam: Camera, u, v) -> float:
    lib = _load()
    T = np.ascontiguousarray(T_wc, dtype=np.float64).reshape(12)
    sc = scene.c()
    return lib.synth_depth_at(ctypes.byref(sc), _ptr(T, ctypes.c_double), cam.fx, cam.fy,
                              cam.cx, cam.cy, float(u), float(v))


def select_points(scene: Scene, T_wc, cam: Camera, img, depth, wall, N, dmin, dmax, seed,
                  margin=4, plane_margin=8) -> np.ndarray:
    """Returns float32 [n, 3] rows (u0, v0, depth) at level-0 sub-pixel positions;
    points whose (2*plane_margin+1)^2 neighbourhood spans two walls are skipped."""
    lib = _load()
    T = np.ascontiguousarray(T_wc, dtype=np.float64).reshape(12)
    img = np.ascontiguousarray(img, np.uint8)
    depth = np.ascontiguousarray(depth, np.float32)
    wall = np.ascontiguousarray(wall, np.uint8)
    out = np.zeros((max(N, 1), 3), np.float32)
    sc = scene.c()
    n = lib.synth_select_points(ctypes.byref(sc), _ptr(T, ctypes.c_double), cam.fx, cam.fy,
                                cam.cx, cam.cy, _ptr(img, ctypes.c_uint8),
                                _ptr(depth, ctypes.c_float), _ptr(wall, ctypes.c_uint8), cam.W,
                                cam.H, int(N), float(dmin), float(dmax), int(margin),
                                int(plane_margin), int(seed) & (2**64 - 1),
                                _ptr(out, ctypes.c_float))
    return out[:n].copy()


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------
@dataclass
class Pair:
    """A reference/current frame pair with its ground truth."""
    cam: Camera
    ref: np.ndarray
    cur: np.ndarray
    uvd: np.ndarray
    T_cr: np.ndarray          # true reference->current motion
    a: float                  # true relative affine (cur ~ e^a ref + b)
    b: float
    ref_depth: np.ndarray = field(repr=False, default=None)


def _unit(rng):
    v = rng.normal(size=3)
    return v / np.linalg.norm(v)


def pair_c1(seed: int, sigma: float = 2.0, N: int = 500, W: int = 320, H: int = 240,
            f: float = 256.0, rot_deg: float = 2.0, trans_m: float = 0.03,
            a: float = 0.05, b: float = 3.0, scene: Scene = ROOM_SMALL) -> Pair:
    """Single pair: reference at the origin looking down +z, current moved by
    `rot_deg` about a seeded random axis and `trans_m` in a seeded direction."""
    rng = np.random.default_rng(10_000 + seed)
    cam = Camera(W, H, f, f, W / 2.0, H / 2.0)
    T_wc_ref = pose(np.eye(3), np.zeros(3))
    R_cr = rot_from_axis_angle(_unit(rng), np.deg2rad(rot_deg))
    t_cr = trans_m * _unit(rng)
    T_cr = pose(R_cr, t_cr)
    T_wc_cur = pose_mul(T_wc_ref, pose_inv(T_cr))
    ref, dref, wref = render(scene, T_wc_ref, cam, 0.0, 0.0, sigma, noise_seed=2 * seed + 1,
                             want_wall=True)
    cur, _ = render(scene, T_wc_cur, cam, a, b, sigma, noise_seed=2 * seed + 2)
    uvd = select_points(scene, T_wc_ref, cam, ref, dref, wref, N, 1.0, 5.0, seed=seed,
                        plane_margin=16)
    return Pair(cam, ref, cur, uvd, T_cr, a, b, dref)


@dataclass
class Sequence:
    cam: Camera
    scene: Scene
    T_wc: np.ndarray          # [F, 3, 4]
    a: np.ndarray             # [F] absolute exposure
    b: np.ndarray             # [F]
    sigma: float
    seed: int

    def __len__(self):
        return len(self.T_wc)

    def frame(self, k: int, want_wall=False):
        return render(self.scene, self.T_wc[k], self.cam, self.a[k], self.b[k], self.sigma,
                      noise_seed=(self.seed << 20) + k, want_wall=want_wall)

    def rel_affine(self, r: int, c: int):
        a = self.a[c] - self.a[r]
        return a, self.b[c] - np.exp(a) * self.b[r]


def trajectory(seed: int, frames: int, fps: float, speed: float, ang_speed_deg: float,
               scene: Scene, margin: float = 1.0):
    """Smooth seeded trajectory: per axis a sum of three sinusoids for the
    position and for the rotation vector (yaw-dominant), rescaled to the
    requested mean linear and angular speeds, kept `margin` from the walls."""
    rng = np.random.default_rng(seed)
    t = np.arange(frames) / fps
    lo, hi = np.array(scene.lo), np.array(scene.hi)
    centre = 0.5 * (lo + hi)
    half = 0.5 * (hi - lo) - margin
    freqs = rng.uniform(0.08, 0.35, size=(3, 3))
    phase = rng.uniform(0, 2 * np.pi, size=(3, 3))
    pos = np.zeros((frames, 3))
    for ax in range(3):
        for j in range(3):
            pos[:, ax] += half[ax] / 3.0 * np.sin(2 * np.pi * freqs[ax, j] * t + phase[ax, j])
    v = np.linalg.norm(np.diff(pos, axis=0), axis=1).mean() * fps
    pos *= speed / max(v, 1e-9)
    # keep inside the margin: shrink any axis that overflows (slows that axis)
    for ax in range(3):
        m = np.abs(pos[:, ax]).max()
        if m > half[ax]:
            pos[:, ax] *= half[ax] / m
    pos += centre
    rf = rng.uniform(0.08, 0.35, size=(3, 3))
    rp = rng.uniform(0, 2 * np.pi, size=(3, 3))
    amp = np.array([0.25, 1.0, 0.15])   # pitch (x), yaw (y), roll (z)
    rv = np.zeros((frames, 3))
    for ax in range(3):
        for j in range(3):
            rv[:, ax] += amp[ax] / 3.0 * np.sin(2 * np.pi * rf[ax, j] * t + rp[ax, j])
    Rs = [rot_from_vec(r) for r in rv]
    w = np.mean([rotation_angle(Rs[k].T @ Rs[k + 1]) for k in range(frames - 1)]) * fps
    rv *= np.deg2rad(ang_speed_deg) / max(w, 1e-12)
    # cap the yaw so the camera keeps facing the long (+z) axis of the room
    cap = np.array([0.35, 0.7, 0.25])
    for ax in range(3):
        m = np.abs(rv[:, ax]).max()
        if m > cap[ax]:
            rv[:, ax] *= cap[ax] / m
    T = np.stack([pose(rot_from_vec(rv[k]), pos[k]) for k in range(frames)])
    return T


def sequence(seed: int, frames: int, cam: Camera, scene: Scene, speed: float,
             ang_speed_deg: float, fps: float = 30.0, sigma: float = 2.0,
             a_range=(-0.1, 0.1), b_range=(-10.0, 10.0)) -> Sequence:
    T = trajectory(seed, frames, fps, speed, ang_speed_deg, scene)
    rng = np.random.default_rng(seed + 77)
    t = np.arange(frames) / fps
    fa, fb = rng.uniform(0.05, 0.25, 2)
    pa, pb = rng.uniform(0, 2 * np.pi, 2)
    a = 0.5 * (a_range[0] + a_range[1]) + 0.5 * (a_range[1] - a_range[0]) * np.sin(2 * np.pi * fa * t + pa)
    b = 0.5 * (b_range[0] + b_range[1]) + 0.5 * (b_range[1] - b_range[0]) * np.sin(2 * np.pi * fb * t + pb)
    return Sequence(cam, scene, T, a, b, sigma, seed)


def reference_points(seq: Sequence, k: int, N: int, dmin: float, dmax: float):
    """Renders frame k and picks N map points on it (reference refresh)."""
    img, dep, wall = seq.frame(k, want_wall=True)
    uvd = select_points(seq.scene, seq.T_wc[k], seq.cam, img, dep, wall, N, dmin, dmax,
                        seed=(seq.seed << 16) + k)
    return img, uvd
