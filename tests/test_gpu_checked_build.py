"""The bounds-checked build (libglt_checked.so, GLT_CHECKED): the pyramid,
map-point, tracking and batch parity suites run against it in a child
process, where every test also asserts that no gather or table access left
its buffer (glt_debug_checked_flags); the normal build reports that it is
not a checked build; a positive control shows that a read past a buffer is
caught."""
import ctypes
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_normal_build_is_not_checked():
    import paper_2607_16897_gb300 as glt
    flags = ctypes.c_uint(7)
    assert glt.glt_debug_checked_flags(ctypes.byref(flags)) == glt.GLT_ERR_UNSUPPORTED
    assert flags.value == 0
    flags.value = 7
    assert glt.glt_debug_checked_probe(ctypes.byref(flags)) == glt.GLT_ERR_UNSUPPORTED
    assert flags.value == 0


def test_checked_build_flags_an_out_of_range_read():
    """Positive control, in a child process on the checked library: the
    probe's read past its buffer is redirected and flagged (flag 4), and the
    flags of the kernels are clear again afterwards."""
    code = ("import ctypes, paper_2607_16897_gb300 as glt\n"
            "f = ctypes.c_uint(0)\n"
            "assert glt.glt_debug_checked_probe(ctypes.byref(f)) == 0, glt.glt_last_error()\n"
            "assert f.value == 4, f.value\n"
            "assert glt.glt_debug_checked_flags(ctypes.byref(f)) == 0 and f.value == 0\n"
            "print('probe ok')\n")
    env = dict(os.environ, GLT_LIBRARY="checked")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0 and "probe ok" in r.stdout, r.stdout[-2000:] + r.stderr[-2000:]


def test_parity_suites_in_the_checked_build():
    lib = os.path.join(ROOT, "paper_2607_16897_gb300", "libglt_checked.so")
    assert os.path.exists(lib), "libglt_checked.so is built by __graft_entry__.build()"
    suites = ["test_gpu_pyramid.py", "test_gpu_linearize.py", "test_gpu_track.py", "test_gpu_batch.py",
              "test_gpu_ic.py", "test_gpu_paper_config.py", "test_gpu_hcache.py", "test_gpu_solve_modes.py"]
    env = dict(os.environ, GLT_LIBRARY="checked")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider",
                        *[os.path.join(ROOT, "tests", s) for s in suites]],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]
    import re
    m = re.search(r"(\d+) passed", r.stdout)
    assert m and int(m.group(1)) >= 100, r.stdout[-2000:]
