"""Python binding of libglt.so: GB300-native pose-only direct photometric tracking.

Argument marshalling only.  Every step of the method runs in the library's
sm_103a kernels; PyTorch is used for device memory (``data_ptr()``) and
streams (``torch.cuda.current_stream().cuda_stream``).  The functions
``glt_*`` are the C entry points of ``include/glt.h`` under the same names;
``Tracker`` and ``Batch`` wrap them for numpy / torch callers.

The library is loaded on first use (a ``glt_*`` attribute, a wrapper object,
or ``load()``); if ``libglt.so`` has not been built that first use raises
ImportError.  There is no fallback of any kind.  The pure host modules of the
package (``tween``, ``proposal``'s feature and training helpers) import
without the library.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# GLT_LIBRARY=checked selects the bounds-checked build (libglt_checked.so)
LIB_PATH = os.path.join(_HERE, "libglt_checked.so" if os.environ.get("GLT_LIBRARY") == "checked"
                        else "libglt.so")

GLT_OK = 0
GLT_ERR_INVALID_ARG = -1
GLT_ERR_CUDA = -2
GLT_ERR_NO_REFERENCE = -3
GLT_ERR_CAPACITY = -4
GLT_ERR_UNSUPPORTED = -5
GLT_ERR_IO = -6
GLT_TRACK_TOO_FEW_POINTS = 1
GLT_TRACK_NOT_PD = 2
GLT_TRACK_DIVERGED = 4
GLT_TRACK_TIMEOUT = 8
GLT_SOLVE_FP64, GLT_SOLVE_FP32 = 0, 1
GLT_REF, GLT_CUR = 0, 1
GLT_FP32, GLT_MIXED = 0, 1
GLT_FORWARD, GLT_IC = 0, 1
GLT_HESSIAN_PASS, GLT_HESSIAN_CACHED = 0, 1
MAX_LEVELS = 8
GLT_NN_PARAMS = 189064
GLT_NN_INPUT = 1200
GLT_NN_MOTION = 6
GLT_NN_OUTPUT = 8


class glt_config(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int), ("height", ctypes.c_int), ("levels", ctypes.c_int),
                ("fx", ctypes.c_double), ("fy", ctypes.c_double), ("cx", ctypes.c_double),
                ("cy", ctypes.c_double), ("max_points", ctypes.c_int),
                ("max_iters", ctypes.c_int * MAX_LEVELS), ("huber_k", ctypes.c_double),
                ("lambda0", ctypes.c_double), ("lambda_up", ctypes.c_double),
                ("lambda_down", ctypes.c_double), ("eps_step", ctypes.c_double),
                ("eps_step_coarse", ctypes.c_double),
                ("eps_cost", ctypes.c_double), ("accept_step", ctypes.c_double),
                ("min_valid", ctypes.c_int),
                ("zmin", ctypes.c_double), ("precision", ctypes.c_int), ("cluster", ctypes.c_int),
                ("threads", ctypes.c_int), ("jacobian", ctypes.c_int), ("pattern", ctypes.c_int),
                ("affine", ctypes.c_int), ("hessian", ctypes.c_int), ("solve", ctypes.c_int)]


class glt_result(ctypes.Structure):
    _fields_ = [("T", ctypes.c_double * 12), ("a", ctypes.c_double), ("b", ctypes.c_double),
                ("cost", ctypes.c_double), ("n_valid", ctypes.c_int),
                ("iters_total", ctypes.c_int), ("iters", ctypes.c_int * MAX_LEVELS),
                ("passes", ctypes.c_int), ("status", ctypes.c_int)]


class glt_state(ctypes.Structure):
    _fields_ = [("T_cr", ctypes.c_double * 12), ("a", ctypes.c_double), ("b", ctypes.c_double),
                ("motion", ctypes.c_double * 12), ("reference", ctypes.c_uint),
                ("frames", ctypes.c_int)]


RESULT_BYTES = ctypes.sizeof(glt_result)
RESULT_DTYPE = np.dtype({"names": ["T", "a", "b", "cost", "n_valid", "iters_total", "iters",
                                   "passes", "status"],
                         "formats": [(np.float64, (12,)), np.float64, np.float64, np.float64,
                                     np.int32, np.int32, (np.int32, (MAX_LEVELS,)), np.int32,
                                     np.int32],
                         "offsets": [glt_result.T.offset, glt_result.a.offset,
                                     glt_result.b.offset, glt_result.cost.offset,
                                     glt_result.n_valid.offset, glt_result.iters_total.offset,
                                     glt_result.iters.offset, glt_result.passes.offset,
                                     glt_result.status.offset],
                         "itemsize": RESULT_BYTES})

# name -> (restype, argtypes) of every entry point declared in include/glt.h
_P = ctypes.POINTER
_vp = ctypes.c_void_p
_i = ctypes.c_int
_d = ctypes.c_double
SIGNATURES = {
    "glt_default_config": (None, [_P(glt_config), _i, _i, _d, _d, _d, _d]),
    "glt_create": (_i, [_P(glt_config), _P(_vp)]),
    "glt_destroy": (None, [_vp]),
    "glt_build_pyramid": (_i, [_vp, _i, _vp, _i, _i, _vp]),
    "glt_set_map_points": (_i, [_vp, _vp, _i, _i, _vp]),
    "glt_track_frame": (_i, [_vp, _P(_d), _P(_d), _P(glt_result), _vp]),
    "glt_track_frame_async": (_i, [_vp, _vp, _vp, _vp]),
    "glt_track_image_async": (_i, [_vp, _vp, _i, _vp, _vp, _vp]),
    "glt_track_image": (_i, [_vp, _vp, _i, _i, _P(_d), _P(_d), _P(glt_result), _vp]),
    "glt_debug_linearize": (_i, [_vp, _i, _P(_d), _d, _d, _P(_d), _P(_d), _P(_d), _P(_i),
                                 _P(ctypes.c_float), _vp]),
    "glt_debug_rcp": (_i, [_vp, _vp, _i, _vp]),
    "glt_debug_pass_floor": (_i, [_i, _i, _i, _i, _i, _P(ctypes.c_float), _vp]),
    "glt_debug_exchange_timeout": (_i, [_i, _i, _P(ctypes.c_int), _vp]),
    "glt_debug_checked_flags": (_i, [_P(ctypes.c_uint)]),
    "glt_debug_checked_probe": (_i, [_P(ctypes.c_uint)]),
    "glt_get_shape": (_i, [_vp, _P(_i), _P(_i)]),
    "glt_get_pyramid": (_i, [_vp, _i, _i, _P(ctypes.c_uint8), _vp]),
    "glt_get_trace": (_i, [_vp, _P(_d), _P(_i), _i, _P(_i), _vp]),
    "glt_state_predict": (_i, [_P(glt_state), _P(_d), _P(_d)]),
    "glt_state_update": (_i, [_P(glt_state), _P(glt_result)]),
    "glt_get_state": (_i, [_vp, _P(glt_state)]),
    "glt_set_state": (_i, [_vp, _P(glt_state)]),
    "glt_batch_create": (_i, [_P(_vp), _i, _P(_vp)]),
    "glt_batch_destroy": (None, [_vp]),
    "glt_batch_build_pyramid": (_i, [_vp, _vp, _vp]),
    "glt_batch_track": (_i, [_vp, _vp, _vp, _vp]),
    "glt_batch_capture": (_i, [_vp, _vp, _vp, _vp, _vp]),
    "glt_batch_replay": (_i, [_vp, _vp]),
    "glt_batch_autotune": (_i, [_vp, _vp, _vp, _i, _P(_i), _P(_i), _P(ctypes.c_float), _vp]),
    "glt_batch_set_shape": (_i, [_vp, _i, _i]),
    "glt_batch_set_classes": (_i, [_vp, _i, _i, _i, _i, _i]),
    "glt_batch_get_classes": (_i, [_vp, _P(_i), _P(_i), _P(_i), _P(_i), _P(_i)]),
    "glt_batch_set_proportional": (_i, [_vp, _i, _i]),
    "glt_batch_get_class_table": (_i, [_vp, _i, _P(_i), _P(_i), _P(_i), _P(_i)]),
    "glt_linearize_noalloc": (_i, [_vp, _i, _vp, _i, _i, _i, _i, _d, _d, _d, _d, _vp, _i, _P(_d),
                                   _d, _d, _d, _d, _vp, _vp]),
    "glt_nn_create": (_i, [_i, _P(_vp)]),
    "glt_nn_destroy": (None, [_vp]),
    "glt_nn_set_params": (_i, [_vp, _P(ctypes.c_float), _i]),
    "glt_nn_get_params": (_i, [_vp, _P(ctypes.c_float), _i]),
    "glt_nn_forward": (_i, [_vp, _vp, _vp, _vp, _i, _vp]),
    "glt_nn_gradient": (_i, [_vp, _vp, _vp, _vp, _i, _P(ctypes.c_float), _P(ctypes.c_float), _vp]),
    "glt_nn_train_step": (_i, [_vp, _vp, _vp, _vp, _i, ctypes.c_float, _vp, _vp]),
    "glt_nn_save": (_i, [_vp, ctypes.c_char_p]),
    "glt_nn_load": (_i, [_vp, ctypes.c_char_p]),
    "glt_batch_set_proposal": (_i, [_vp, _vp, _vp]),
    "glt_status_string": (ctypes.c_char_p, [_i]),
    "glt_last_error": (ctypes.c_char_p, []),
    "glt_version": (ctypes.c_char_p, []),
}


def _open():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is not built; run paper_2607_16897_gb300.build.build() "
            "(the CUDA library is required, there is no fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_handle = None


def load():
    """The loaded library (opened on the first call; ImportError if it is not
    built)."""
    global _handle
    if _handle is None:
        _handle = _open()
    return _handle


class _Lazy:
    """Forwards attribute access to the library, opening it on first use."""

    def __getattr__(self, name):
        return getattr(load(), name)


_lib = _Lazy()


def __getattr__(name):
    # module attributes glt_* are the C entry points (PEP 562)
    if name in SIGNATURES:
        return getattr(load(), name)
    raise AttributeError(f"module {__name__!r} has no attribute {name!r}")


class GltError(RuntimeError):
    pass


def _check(rc: int, what: str):
    if rc != GLT_OK:
        raise GltError(f"{what} failed ({rc}): {_lib.glt_last_error().decode()}")


def _stream_handle(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dptr(t) -> int:
    """Device address of a tensor (or an address given as an int)."""
    return int(t) if isinstance(t, int) else int(t.data_ptr())


def _is_cuda_tensor(x) -> bool:
    return hasattr(x, "is_cuda") and bool(x.is_cuda)


def default_config(width, height, K, **kw) -> glt_config:
    fx, fy, cx, cy = (float(k) for k in K)
    c = glt_config()
    _lib.glt_default_config(ctypes.byref(c), int(width), int(height), fx, fy, cx, cy)
    for k, v in kw.items():
        if k == "max_iters":
            v = list(v)
            v = (v + [v[-1]] * MAX_LEVELS)[:MAX_LEVELS]
            for i in range(MAX_LEVELS):
                c.max_iters[i] = int(v[i])
        elif k == "precision" and isinstance(v, str):
            c.precision = {"fp32": GLT_FP32, "mixed": GLT_MIXED}[v]
        elif k == "jacobian" and isinstance(v, str):
            c.jacobian = {"forward": GLT_FORWARD, "ic": GLT_IC}[v]
        elif k == "hessian" and isinstance(v, str):
            c.hessian = {"pass": GLT_HESSIAN_PASS, "cached": GLT_HESSIAN_CACHED}[v]
        elif k == "solve" and isinstance(v, str):
            c.solve = {"fp64": GLT_SOLVE_FP64, "fp32": GLT_SOLVE_FP32}[v]
        else:
            if not hasattr(c, k):
                raise KeyError(k)
            setattr(c, k, v)
    return c


def result_to_dict(r) -> dict:
    """glt_result (ctypes struct or numpy structured record) -> dict."""
    if isinstance(r, glt_result):
        T = np.array(r.T[:]).reshape(3, 4)
        return {"T": T, "a": r.a, "b": r.b, "cost": r.cost, "n_valid": r.n_valid,
                "iters_total": r.iters_total, "iters": list(r.iters[:]), "passes": r.passes,
                "status": r.status}
    return {"T": np.array(r["T"]).reshape(3, 4), "a": float(r["a"]), "b": float(r["b"]),
            "cost": float(r["cost"]), "n_valid": int(r["n_valid"]),
            "iters_total": int(r["iters_total"]), "iters": [int(x) for x in r["iters"]],
            "passes": int(r["passes"]), "status": int(r["status"])}


def parse_results(buf) -> list:
    """Device or host byte buffer of S glt_result structs -> list of dicts."""
    if _is_cuda_tensor(buf):
        buf = buf.cpu().numpy()
    arr = np.frombuffer(np.ascontiguousarray(buf).tobytes(), dtype=RESULT_DTYPE)
    return [result_to_dict(r) for r in arr]


class Tracker:
    """One camera stream: glt_create / glt_build_pyramid / glt_set_map_points /
    glt_track_frame / glt_debug_linearize on numpy or torch inputs."""

    def __init__(self, width, height, K, **cfg):
        self.cfg = default_config(width, height, K, **cfg)
        self.W, self.H, self.L = int(width), int(height), int(self.cfg.levels)
        h = ctypes.c_void_p()
        _check(_lib.glt_create(ctypes.byref(self.cfg), ctypes.byref(h)), "glt_create")
        self.handle = h
        self.N = 0

    def close(self):
        if getattr(self, "handle", None):
            _lib.glt_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check_frame(self, img):
        # the library reads height rows of width bytes: refuse smaller arrays
        if len(img.shape) != 2 or img.shape[0] < self.H or img.shape[1] < self.W:
            raise ValueError(f"frame of shape {tuple(img.shape)}; the tracker needs "
                             f"{self.H} x {self.W} uint8")

    def build_pyramid(self, slot, img, stream=None):
        self._check_frame(img)
        if _is_cuda_tensor(img):
            assert img.dtype.itemsize == 1 and img.is_contiguous()
            pitch = img.shape[-1]
            _check(_lib.glt_build_pyramid(self.handle, slot, _dptr(img), pitch, 1,
                                          _stream_handle(stream)), "glt_build_pyramid")
        else:
            a = np.ascontiguousarray(img, np.uint8)
            _check(_lib.glt_build_pyramid(self.handle, slot, a.ctypes.data, a.shape[1], 0,
                                          _stream_handle(stream)), "glt_build_pyramid")
            # pageable H2D copies are staged before the call returns

    def set_map_points(self, uvd, stream=None):
        if _is_cuda_tensor(uvd):
            n = uvd.shape[0]
            _check(_lib.glt_set_map_points(self.handle, _dptr(uvd), n, 1, _stream_handle(stream)),
                   "glt_set_map_points")
        else:
            a = np.ascontiguousarray(uvd, np.float32).reshape(-1, 3)
            n = a.shape[0]
            _check(_lib.glt_set_map_points(self.handle, a.ctypes.data, n, 0,
                                           _stream_handle(stream)), "glt_set_map_points")
        self.N = n

    def track_frame(self, T_init=None, ab_init=None, stream=None) -> dict:
        """T_init None: start from the tracker's constant-velocity prediction
        (and ab_init None from its last affine pair); ab_init None with a
        given T_init: (0, 0)."""
        Tp = abp = None
        if T_init is not None:
            T = np.ascontiguousarray(T_init, np.float64).reshape(12)
            Tp = T.ctypes.data_as(_P(_d))
            if ab_init is None:
                ab_init = (0.0, 0.0)
        if ab_init is not None:
            ab = np.ascontiguousarray(ab_init, np.float64).reshape(2)
            abp = ab.ctypes.data_as(_P(_d))
        r = glt_result()
        _check(_lib.glt_track_frame(self.handle, Tp, abp, ctypes.byref(r), _stream_handle(stream)),
               "glt_track_frame")
        return result_to_dict(r)

    def get_state(self) -> glt_state:
        st = glt_state()
        _check(_lib.glt_get_state(self.handle, ctypes.byref(st)), "glt_get_state")
        return st

    def set_state(self, st: glt_state):
        _check(_lib.glt_set_state(self.handle, ctypes.byref(st)), "glt_set_state")

    def track_frame_async(self, init_dev, out_dev, stream=None):
        _check(_lib.glt_track_frame_async(self.handle, _dptr(init_dev), _dptr(out_dev),
                                          _stream_handle(stream)), "glt_track_frame_async")

    def track_image(self, img, T_init=None, ab_init=None, stream=None) -> dict:
        """One frame end to end (glt_track_image): `img` is a host numpy array
        (uploaded by the library; pinned memory uploads fastest) or a CUDA
        tensor.  T_init None: the state's constant-velocity prediction."""
        Tp = abp = None
        if T_init is not None:
            T = np.ascontiguousarray(T_init, np.float64).reshape(12)
            Tp = T.ctypes.data_as(_P(_d))
            if ab_init is None:
                ab_init = (0.0, 0.0)
        if ab_init is not None:
            ab = np.ascontiguousarray(ab_init, np.float64).reshape(2)
            abp = ab.ctypes.data_as(_P(_d))
        r = glt_result()
        self._check_frame(img)
        if _is_cuda_tensor(img):
            assert img.dtype.itemsize == 1 and img.stride(1) == 1
            ptr, pitch, dev = img.data_ptr(), int(img.stride(0)), 1
        else:
            a = np.asarray(img)
            if a.dtype != np.uint8 or a.ndim != 2 or a.strides[1] != 1:
                a = np.ascontiguousarray(a, np.uint8)
            ptr, pitch, dev = a.ctypes.data, int(a.strides[0]), 0   # rows may be pitched
        _check(_lib.glt_track_image(self.handle, ctypes.c_void_p(ptr), pitch, dev, Tp, abp,
                                    ctypes.byref(r), _stream_handle(stream)), "glt_track_image")
        return result_to_dict(r)

    def track_image_async(self, frame_dev, init_dev, out_dev, pitch=None, stream=None):
        """Pyramid of the device frame chained with the solve (glt_track_image_async)."""
        if not isinstance(frame_dev, int):
            self._check_frame(frame_dev)
        pitch = self.W if pitch is None else int(pitch)
        _check(_lib.glt_track_image_async(self.handle, _dptr(frame_dev), pitch, _dptr(init_dev),
                                          _dptr(out_dev), _stream_handle(stream)),
               "glt_track_image_async")

    def debug_linearize(self, level, T, a, b, want_res=True, stream=None) -> dict:
        T = np.ascontiguousarray(T, np.float64).reshape(12)
        H = np.zeros(64)
        g = np.zeros(8)
        E = ctypes.c_double()
        n = ctypes.c_int()
        K = 8 if self.cfg.pattern == 0 else self.cfg.pattern ** 2
        res = np.zeros(max(self.N, 1) * K, np.float32) if want_res else None
        _check(_lib.glt_debug_linearize(self.handle, int(level), T.ctypes.data_as(_P(_d)),
                                        float(a), float(b), H.ctypes.data_as(_P(_d)),
                                        g.ctypes.data_as(_P(_d)), ctypes.byref(E),
                                        ctypes.byref(n),
                                        res.ctypes.data_as(_P(ctypes.c_float)) if want_res else None,
                                        _stream_handle(stream)), "glt_debug_linearize")
        out = {"H": H.reshape(8, 8), "g": g, "E": E.value, "n": n.value}
        if want_res:
            out["res"] = res[:self.N * K].reshape(self.N, K)
        return out

    def shape(self):
        """(cluster, threads) of the tracker's solve launch."""
        c, t = ctypes.c_int(), ctypes.c_int()
        _check(_lib.glt_get_shape(self.handle, ctypes.byref(c), ctypes.byref(t)), "glt_get_shape")
        return c.value, t.value

    def get_pyramid(self, slot, level, stream=None) -> np.ndarray:
        w, h = self.W >> level, self.H >> level
        out = np.zeros((h, w), np.uint8)
        _check(_lib.glt_get_pyramid(self.handle, slot, level, out.ctypes.data_as(_P(ctypes.c_uint8)),
                                    _stream_handle(stream)), "glt_get_pyramid")
        return out

    def get_trace(self, stream=None) -> list:
        m = self.L * (1 + max(self.cfg.max_iters[:self.L]))
        cost = np.zeros(max(m, 1))
        info = np.zeros(max(m, 1), np.int32)
        cnt = ctypes.c_int()
        _check(_lib.glt_get_trace(self.handle, cost.ctypes.data_as(_P(_d)),
                                  info.ctypes.data_as(_P(_i)), m, ctypes.byref(cnt),
                                  _stream_handle(stream)), "glt_get_trace")
        return [dict(cost=float(cost[k]), level=int(info[k]) >> 2, accepted=bool(info[k] & 2),
                     candidate=bool(info[k] & 1)) for k in range(cnt.value)]


class Batch:
    """S trackers tracked in one persistent launch (glt_batch_*)."""

    def __init__(self, trackers):
        self.trackers = list(trackers)
        arr = (ctypes.c_void_p * len(self.trackers))(*[t.handle for t in self.trackers])
        h = ctypes.c_void_p()
        _check(_lib.glt_batch_create(arr, len(self.trackers), ctypes.byref(h)), "glt_batch_create")
        self.handle = h
        self.S = len(self.trackers)

    def close(self):
        if getattr(self, "handle", None):
            _lib.glt_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def build_pyramid(self, frame_ptrs_dev, stream=None):
        _check(_lib.glt_batch_build_pyramid(self.handle, _dptr(frame_ptrs_dev),
                                            _stream_handle(stream)), "glt_batch_build_pyramid")

    def track(self, init_dev, out_dev, stream=None):
        _check(_lib.glt_batch_track(self.handle, _dptr(init_dev), _dptr(out_dev),
                                    _stream_handle(stream)), "glt_batch_track")

    def capture(self, frame_ptrs_dev, init_dev, out_dev, stream):
        _check(_lib.glt_batch_capture(self.handle, _dptr(frame_ptrs_dev), _dptr(init_dev),
                                      _dptr(out_dev), _stream_handle(stream)), "glt_batch_capture")

    def replay(self, stream=None):
        _check(_lib.glt_batch_replay(self.handle, _stream_handle(stream)), "glt_batch_replay")

    def set_shape(self, cluster, threads):
        _check(_lib.glt_batch_set_shape(self.handle, int(cluster), int(threads)),
               "glt_batch_set_shape")

    def set_classes(self, heavy, heavy_shape, light_shape):
        """Two launch classes: the first `heavy` streams of the launch order
        with heavy_shape = (cluster, threads), the rest with light_shape."""
        _check(_lib.glt_batch_set_classes(self.handle, int(heavy), int(heavy_shape[0]),
                                          int(heavy_shape[1]), int(light_shape[0]),
                                          int(light_shape[1])), "glt_batch_set_classes")

    def set_proportional(self, points_per_cta, threads=128):
        """Clusters in proportion to each stream's points (one class per
        cluster size, concurrent launches)."""
        _check(_lib.glt_batch_set_proportional(self.handle, int(points_per_cta), int(threads)),
               "glt_batch_set_proportional")

    def class_table(self) -> list:
        """[(first stream in launch order, count, cluster, threads)] per class."""
        k = 5
        first, cl, th = (ctypes.c_int * k)(), (ctypes.c_int * k)(), (ctypes.c_int * k)()
        n = ctypes.c_int()
        _check(_lib.glt_batch_get_class_table(self.handle, k, first, cl, th, ctypes.byref(n)),
               "glt_batch_get_class_table")
        out = []
        for i in range(n.value):
            end = first[i + 1] if i + 1 < n.value else self.S
            out.append((first[i], end - first[i], cl[i], th[i]))
        return out

    def classes(self) -> dict:
        v = [ctypes.c_int() for _ in range(5)]
        _check(_lib.glt_batch_get_classes(self.handle, *[ctypes.byref(x) for x in v]),
               "glt_batch_get_classes")
        return {"heavy": v[0].value, "heavy_shape": (v[1].value, v[2].value),
                "light_shape": (v[3].value, v[4].value)}

    def autotune(self, init_dev, out_dev, reps=3, stream=None):
        c, t, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_float()
        _check(_lib.glt_batch_autotune(self.handle, _dptr(init_dev), _dptr(out_dev), int(reps),
                                       ctypes.byref(c), ctypes.byref(t), ctypes.byref(ms),
                                       _stream_handle(stream)), "glt_batch_autotune")
        return c.value, t.value, ms.value

    def set_proposal(self, nn, motion_dev):
        """Attach a proposal network (``NN``) with each stream's last
        inter-frame motion motion_dev [S, 12] (row-major 3x4, float64, device,
        read at every track); ``nn=None`` detaches it."""
        self._nn = nn
        self._motion = motion_dev
        _check(_lib.glt_batch_set_proposal(self.handle, nn.handle if nn is not None else None,
                                           _dptr(motion_dev) if nn is not None else None),
               "glt_batch_set_proposal")


class NN:
    """Learned initial-pose proposal network (glt_nn_*): FP32 device arrays
    x [B, 1200], m [B, 6], y / t [B, 8]."""

    def __init__(self, max_batch, params=None):
        h = ctypes.c_void_p()
        _check(_lib.glt_nn_create(int(max_batch), ctypes.byref(h)), "glt_nn_create")
        self.handle = h
        self.max_batch = int(max_batch)
        if params is not None:
            self.set_params(params)

    def close(self):
        if getattr(self, "handle", None):
            _lib.glt_nn_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        _check(_lib.glt_nn_set_params(self.handle, p.ctypes.data_as(_P(ctypes.c_float)), p.size),
               "glt_nn_set_params")

    def get_params(self) -> np.ndarray:
        p = np.zeros(GLT_NN_PARAMS, np.float32)
        _check(_lib.glt_nn_get_params(self.handle, p.ctypes.data_as(_P(ctypes.c_float)), p.size),
               "glt_nn_get_params")
        return p

    def forward(self, x_dev, m_dev, y_dev, B, stream=None):
        _check(_lib.glt_nn_forward(self.handle, _dptr(x_dev), _dptr(m_dev), _dptr(y_dev), int(B),
                                   _stream_handle(stream)), "glt_nn_forward")

    def gradient(self, x_dev, m_dev, t_dev, B, stream=None):
        g = np.zeros(GLT_NN_PARAMS, np.float32)
        loss = ctypes.c_float()
        _check(_lib.glt_nn_gradient(self.handle, _dptr(x_dev), _dptr(m_dev), _dptr(t_dev), int(B),
                                    g.ctypes.data_as(_P(ctypes.c_float)), ctypes.byref(loss),
                                    _stream_handle(stream)), "glt_nn_gradient")
        return g, loss.value

    def save(self, path):
        """Training checkpoint: weights, Adam moments and step (glt_nn_save)."""
        _check(_lib.glt_nn_save(self.handle, os.fsencode(path)), "glt_nn_save")

    def load(self, path):
        """A checkpoint of save(), or a .npy weight file (glt_nn_load)."""
        _check(_lib.glt_nn_load(self.handle, os.fsencode(path)), "glt_nn_load")

    def train_step(self, x_dev, m_dev, t_dev, B, lr, loss_dev=None, stream=None):
        _check(_lib.glt_nn_train_step(self.handle, _dptr(x_dev), _dptr(m_dev), _dptr(t_dev), int(B),
                                      float(lr), _dptr(loss_dev) if loss_dev is not None else None,
                                      _stream_handle(stream)), "glt_nn_train_step")


def pass_floor(cluster, threads, cached=False, passes=400, stream=None, solve="fp64") -> float:
    """Microseconds per pass of the track kernel's fixed part (no points) for
    one stream's (cluster, threads) shape and solve mode (glt_debug_pass_floor)."""
    us = ctypes.c_float()
    mode = {"fp64": GLT_SOLVE_FP64, "fp32": GLT_SOLVE_FP32}.get(solve, solve)
    _check(_lib.glt_debug_pass_floor(int(cluster), int(threads), int(bool(cached)), int(mode),
                                     int(passes), ctypes.byref(us), _stream_handle(stream)),
           "glt_debug_pass_floor")
    return us.value


def version() -> str:
    return _lib.glt_version().decode()
