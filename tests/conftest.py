import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the sm_103a kernels)")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def syn():
    import synth
    synth.build()
    return synth


@pytest.fixture(autouse=True)
def _bounds_checked_build(request):
    """Under GLT_LIBRARY=checked (the bounds-checked library) every GPU test
    also asserts that no kernel it ran accessed memory outside its buffers."""
    yield
    if os.environ.get("GLT_LIBRARY") != "checked" or request.node.get_closest_marker("gpu") is None:
        return
    import ctypes
    import paper_2607_16897_gb300 as glt
    flags = ctypes.c_uint(0)
    assert glt.glt_debug_checked_flags(ctypes.byref(flags)) == 0, glt.glt_last_error()
    assert flags.value == 0, f"out-of-range accesses, check flags {flags.value:#x}"
