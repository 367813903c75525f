"""Failure detection on the GPU without a GPU fault: a start that is not
finite, and pass sums that overflow FP32, end the solve with the DIVERGED
status bit (the state before the failure is returned); the FP64 oracle
flags the same inputs.  A cluster exchange whose partial sums do not arrive
ends with the TIMEOUT status after its bounded wait.  Also the solver's FP64
reciprocal (one Newton-Raphson step on an FP32 seed) against IEEE division
across the exponent range."""
import numpy as np
import pytest

from helpers import I34

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def glt():
    import paper_2607_16897_gb300 as g
    return g


def _pair(glt, orc, syn):
    p = syn.pair_c1(3, sigma=2.0)
    trk = glt.Tracker(p.cam.W, p.cam.H, p.cam.K, levels=3, max_points=500)
    trk.build_pyramid(glt.GLT_REF, p.ref)
    trk.set_map_points(p.uvd)
    trk.build_pyramid(glt.GLT_CUR, p.cur)
    o = orc.OracleTracker(p.cam.W, p.cam.H, p.cam.K, levels=3)
    o.build_pyramid(0, p.ref)
    o.set_map_points(p.uvd)
    o.build_pyramid(1, p.cur)
    return trk, o


def _track_async(glt, trk, init):
    import torch
    init_dev = torch.tensor(np.asarray(init, np.float64)).cuda()
    out = torch.zeros(glt.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    trk.track_frame_async(init_dev, out)
    torch.cuda.synchronize()
    return glt.parse_results(out)[0]


def test_non_finite_start_is_flagged(glt, orc, syn):
    trk, o = _pair(glt, orc, syn)
    for bad in (np.nan, np.inf):
        init = np.concatenate([I34.ravel(), [0.0, 0.0]])
        init[3] = bad
        g = _track_async(glt, trk, init)
        assert g["status"] == glt.GLT_TRACK_DIVERGED and g["passes"] == 0
        r = o.track_frame(init[:12].reshape(3, 4), (0.0, 0.0))
        assert r["status"] == orc.DIVERGED and r["passes"] == 0
    # a degenerate rotation cannot be orthonormalised: the same outcome
    init = np.zeros(14)
    g = _track_async(glt, trk, init)
    assert g["status"] == glt.GLT_TRACK_DIVERGED and g["passes"] == 0
    assert o.track_frame(np.zeros((3, 4)))["status"] == orc.DIVERGED
    # the tracker is usable afterwards
    g = trk.track_frame(I34)
    assert g["status"] == 0 and g["passes"] > 3
    trk.close()


def test_overflowing_sums_are_flagged(glt, orc, syn):
    """e^a beyond the FP32 (and FP64) range makes every pass's sums infinite
    or NaN: each level start is unusable, the start is returned."""
    trk, o = _pair(glt, orc, syn)
    init = np.concatenate([I34.ravel(), [1000.0, 0.0]])
    g = _track_async(glt, trk, init)
    r = o.track_frame(I34, (1000.0, 0.0))
    assert g["status"] == glt.GLT_TRACK_DIVERGED, glt.glt_status_string(g["status"])
    assert r["status"] == orc.DIVERGED
    assert g["passes"] == r["passes"] == 3          # one unusable level start per level
    assert np.array_equal(g["T"], I34) and g["a"] == 1000.0
    assert glt.glt_status_string(g["status"]) == b"diverged"
    trk.close()


def test_reciprocal_against_ieee_division(glt):
    import torch
    rng = np.random.default_rng(0)
    e = rng.integers(-99, 100, 20000)
    m = rng.uniform(1.0, 2.0, 20000)
    d = np.ldexp(m, e) * rng.choice([-1.0, 1.0], 20000)
    # the edges of the Newton range and the division fallback beyond it
    edges = np.array([2.0 ** -100, np.nextafter(2.0 ** -100, 0), 2.0 ** 100,
                      np.nextafter(2.0 ** 100, 0), 2.0 ** -101, 2.0 ** 101, 1.0, -1.0,
                      np.nextafter(1.0, 2), np.nextafter(2.0, 0), 3.0, 1e-300, 1e300, 5e-324,
                      0.0, -0.0, np.inf, -np.inf, np.nan])
    d = np.concatenate([d, edges, -edges])
    dd = torch.from_numpy(d).cuda()
    rr = torch.empty_like(dd)
    assert glt.glt_debug_rcp(dd.data_ptr(), rr.data_ptr(), len(d), None) == glt.GLT_OK
    torch.cuda.synchronize()
    r = rr.cpu().numpy()
    with np.errstate(divide="ignore", over="ignore"):
        ref = 1.0 / d
    newton = (np.abs(d) >= 2.0 ** -100) & (np.abs(d) < 2.0 ** 100)
    rel = np.abs(r[newton] - ref[newton]) / np.abs(ref[newton])
    assert rel.max() < 1e-13, rel.max()
    # outside the Newton range the kernel divides: IEEE results, bit for bit
    out = ~newton
    assert np.array_equal(np.isnan(r[out]), np.isnan(ref[out]))
    ok = ~np.isnan(ref[out])
    assert np.array_equal(r[out][ok], ref[out][ok])
    assert glt.glt_debug_rcp(0, 0, -1, None) == glt.GLT_ERR_INVALID_ARG


def test_cluster_exchange_wait_runs_out_and_reports(glt):
    """A CTA that withholds its partial sums: every bounded wait of the
    cluster exchange runs out, the kernel reports GLT_TRACK_TIMEOUT, and the
    context stays usable (the next floor launch completes normally)."""
    import ctypes
    st = ctypes.c_int(-1)
    assert glt.glt_debug_exchange_timeout(4, 256, ctypes.byref(st), None) == 0
    assert st.value == glt.GLT_TRACK_TIMEOUT
    assert glt.glt_status_string(st.value) == b"timeout"
    assert glt.pass_floor(4, 256, passes=20) > 0.0
    with pytest.raises(Exception):
        glt.pass_floor(4, 300)
    assert glt.glt_debug_exchange_timeout(1, 256, ctypes.byref(st), None) == glt.GLT_ERR_INVALID_ARG
