"""Tween-frame switch (Sec. IV-D) on the GPU against the oracle: along
sequences fast and jumpy enough that the acceptance test rejects frames
(3 m/s, 135 deg/s, the exposure offset stepping by 40 gray levels every third
frame), every frame is tracked by the library and by the FP64 oracle from the
same start and reference; the acceptance test takes the same decision on
both results, so the direct / indirect schedules are identical."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed", [7100, 7101])
def test_switch_decisions_match_the_oracle(orc, syn, seed):
    import bench
    import paper_2607_16897_gb300 as glt
    F = 24
    wl = bench.Workload(seed=seed, frames=F, N=500, W=320, H=240, f=256.0, L=3, speed=3.0,
                        ang=135.0, render=False, label="tween switch test stream")
    wl.seq.b = wl.seq.b + 40.0 * ((np.arange(F) // 3) % 2)
    wl.frames = [wl.seq.frame(k)[0] for k in range(F)]
    trk = glt.Tracker(320, 240, wl.cam.K, levels=3, max_points=500)
    o = orc.OracleTracker(320, 240, wl.cam.K, levels=3)
    drv = bench.SequenceDriver(wl)
    mirror = bench.SequenceDriver(wl).switch           # replays the oracle's decisions
    decisions = []
    for k in range(1, F):
        if drv.refresh(k - 1):
            ref, uvd = wl.frames[drv.r], wl.ref_points(drv.r)
            trk.build_pyramid(glt.GLT_REF, ref)
            trk.set_map_points(uvd)
            o.build_pyramid(0, ref)
            o.set_map_points(uvd)
        T0, ab = drv.init_for(k), drv.ab_init()
        trk.build_pyramid(glt.GLT_CUR, wl.frames[k])
        o.build_pyramid(1, wl.frames[k])
        g = trk.track_frame(T0, ab)
        r = o.track_frame(T0, ab)
        ok_g = drv.switch.direct_ok(g, wl.N)
        ok_o = mirror.direct_ok(r, wl.N)
        assert ok_g == ok_o, (k, g["status"], r["status"], g["cost"], r["cost"], g["n_valid"],
                              r["n_valid"])
        mirror.after_direct(r, wl.N)
        drv.record(k, g)
        decisions.append(ok_g)
    assert drv.switch.history == mirror.history
    assert not all(decisions) and sum(decisions) > F // 2, decisions   # the test sees rejections
    trk.close()
