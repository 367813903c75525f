"""The C-ABI library loads and exports every entry point include/glt.h
declares, and the binding's structs match the C layout (no GPU needed)."""
import ctypes
import importlib.util
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "glt.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^[A-Za-z_][\w\s\*]*?\b(glt_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib_path():
    spec = importlib.util.spec_from_file_location(
        "_glt_build", os.path.join(ROOT, "paper_2607_16897_gb300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.build()


def test_header_declares_the_api():
    names = declared_functions()
    for must in ("glt_create", "glt_build_pyramid", "glt_set_map_points", "glt_track_frame",
                 "glt_debug_linearize", "glt_batch_track", "glt_batch_capture"):
        assert must in names
    assert len(names) >= 20


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_checked_library_exports_the_same_api():
    """The bounds-checked twin (GLT_CHECKED) is the same ABI."""
    spec = importlib.util.spec_from_file_location(
        "_glt_build", os.path.join(ROOT, "paper_2607_16897_gb300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    lib = ctypes.CDLL(mod.build(checked=True))
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    # no GPU is needed to see that it is the checked build: the call fails on
    # the device, not with "not a checked build"
    flags = ctypes.c_uint(0)
    lib.glt_debug_checked_flags.argtypes = [ctypes.POINTER(ctypes.c_uint)]
    lib.glt_last_error.restype = ctypes.c_char_p
    rc = lib.glt_debug_checked_flags(ctypes.byref(flags))
    assert rc != -5 or b"not a bounds-checked build" not in lib.glt_last_error()


def test_binding_covers_header_and_layouts(lib_path):
    import paper_2607_16897_gb300 as glt
    assert set(glt.SIGNATURES) == set(declared_functions())
    assert ctypes.sizeof(glt.glt_config) == 200
    # the C struct has the binding's layout: glt_default_config writes exactly
    # sizeof(glt_config) bytes and its last field lands where the binding has it
    buf = (ctypes.c_uint8 * 256)(*([0xA5] * 256))
    glt.glt_default_config(ctypes.cast(buf, ctypes.POINTER(glt.glt_config)), 640, 480, 525.0,
                           525.0, 320.0, 240.0)
    assert bytes(buf[200:]) == bytes([0xA5] * 56)
    cfg = glt.glt_config.from_buffer_copy(bytes(buf[:200]))
    assert cfg.affine == 1 and cfg.pattern == 0 and cfg.jacobian == 0 and cfg.width == 640
    assert cfg.hessian == glt.GLT_HESSIAN_PASS and cfg.solve == glt.GLT_SOLVE_FP64
    assert ctypes.sizeof(glt.glt_result) == 168
    assert glt.RESULT_DTYPE.itemsize == glt.RESULT_BYTES
    c = glt.default_config(640, 480, (525, 525, 320, 240))
    assert c.levels == 4 and c.max_iters[0] == 10 and c.huber_k == 9.0


def test_host_side_argument_checks(lib_path):
    """Config validation happens before any device call, so it runs without a GPU."""
    import paper_2607_16897_gb300 as glt
    bad = [dict(levels=0), dict(levels=9), dict(huber_k=0.0), dict(max_points=0),
           dict(precision=7), dict(cluster=17), dict(threads=100), dict(levels=7),
           dict(jacobian=3)]
    for kw in bad:
        c = glt.default_config(320, 240, (256, 256, 160, 120), **kw)
        h = ctypes.c_void_p()
        rc = glt.glt_create(ctypes.byref(c), ctypes.byref(h))
        assert rc == glt.GLT_ERR_INVALID_ARG, kw
        assert glt.glt_last_error()
    assert glt.glt_build_pyramid(None, 0, None, 0, 0, None) == glt.GLT_ERR_INVALID_ARG
    r = glt.glt_result()
    assert glt.glt_track_image(None, None, 0, 0, None, None, ctypes.byref(r), None) == glt.GLT_ERR_INVALID_ARG
    assert glt.glt_track_image_async(None, None, 0, None, None, None) == glt.GLT_ERR_INVALID_ARG
    assert glt.glt_track_frame(None, None, None, ctypes.byref(r), None) == glt.GLT_ERR_INVALID_ARG
    assert glt.glt_batch_create(None, 0, ctypes.byref(ctypes.c_void_p())) == glt.GLT_ERR_INVALID_ARG


def test_status_strings(lib_path):
    import paper_2607_16897_gb300 as glt
    assert glt.glt_status_string(0) == b"ok"
    assert glt.glt_status_string(glt.GLT_ERR_INVALID_ARG) == b"invalid argument"
    assert glt.glt_status_string(glt.GLT_ERR_CAPACITY) == b"capacity exceeded"
    assert glt.glt_status_string(glt.GLT_TRACK_NOT_PD) == b"not positive definite"
    assert glt.glt_status_string(3) == b"too few points|not positive definite"
    assert glt.glt_status_string(-99) == b"unknown"
