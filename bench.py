"""Benchmark: frames tracked per second on a synthetic sequence.

Default workload (config "c2"): one camera stream, 640x480 uint8 frames
(fx = fy = 525) from a 300-frame seeded sequence at 30 Hz (0.5 m/s, 30 deg/s,
exposure affine a in [-0.1, 0.1], b in [-10, 10], sigma 2 noise), 2000 map
points with depth 0.5-8 m, 4 pyramid levels, Huber k = 9, <= 10 LM iterations
per level, constant-velocity initial pose, a new reference every 8 frames (or
sooner if tracking degrades).  A step is one tracked frame: build the CUR
pyramid of the frame (already in device memory) and run the whole
coarse-to-fine solve.  Reference refreshes are timed separately.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
on the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FLOPS_PER_SAMPLE = 160      # algorithmic FP32 flops per residual sample per pass
# the cached-Hessian form: bilinear sample (7), residual and Huber weight (6), the
# two gradient-weighted sums (4), energy and count (2), the per-point fold amortised (1)
FLOPS_PER_SAMPLE_CACHED = 20


def samples_per_point(wl):
    p = wl.solver.get("pattern", 0)
    return 8 if p == 0 else p * p


def flops_per_sample(wl):
    return FLOPS_PER_SAMPLE_CACHED if wl.solver.get("hessian") == "cached" else FLOPS_PER_SAMPLE
# DRAM bytes (read + write) per track_kernel launch, measured with ncu
# (dram__bytes_read.sum + dram__bytes_write.sum, caches flushed before the
# launch as in the timed steps) on the workload named by the key; a value is
# removed whenever the kernel changes after it was taken.
TRACK_TRAFFIC = {"c2": 813568, "c2p": 6195968}
# the trained proposal network's parameters (data file; read here as plain
# numbers so that the oracle legs need nothing but oracle/ and synth/)
WEIGHTS_PATH = os.path.join(ROOT, "paper_2607_16897_gb300", "proposal_weights.npy")
I34 = np.hstack([np.eye(3), np.zeros((3, 1))])


# ---------------------------------------------------------------------------
# replicas over ranks: independent streams per GPU, the slowest rank's time
# ---------------------------------------------------------------------------
def max_over_ranks(values, dist=None, device="cpu"):
    """Entry-wise maximum of `values` over the ranks of the process group (the
    slowest rank bounds a step); the values themselves without a group."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return [float(v) for v in values]
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def aggregate_rate(units_per_rank, world, seconds):
    """Whole-job throughput: every rank processed `units_per_rank` units in at
    most `seconds` (weak scaling: the work per GPU is fixed)."""
    return world * units_per_rank / seconds


def step_percentiles(ms):
    """Median, 90th percentile and spread of the per-step device times (ms)."""
    a = np.asarray(ms, dtype=np.float64)
    return {"p50": float(np.percentile(a, 50)), "p90": float(np.percentile(a, 90)),
            "min": float(a.min()), "max": float(a.max())}


def stream_seed(kind, s, rank):
    """Seed of stream s of workload `kind` on `rank` (replicas get disjoint
    sequences)."""
    base = {"c2": 1, "c2p": 1, "c2e": 1, "c4": 2000, "c3": 1000, "c4b": 2000, "c5": 5000}[kind]
    return base + s + (100000 * rank if kind in ("c3", "c4b", "c5") else rank)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2", choices=["c2", "c3", "c4", "c4b", "c5", "c2p", "c2e"],
                    help="c2: 640x480 single stream FP32 (default); c3: 64 streams of mixed "
                         "sizes, batched; c4: 1280x720 mixed precision single stream; c4b: "
                         "64 streams of c4, batched; c5: 256 streams of 640x480 with the "
                         "learned proposal, against the plain form on the same streams; c2p / "
                         "c2e: single stream in the paper's configuration (7x7 / 11x11 patches, "
                         "IC Jacobians, 6 levels, fixed-count Gauss-Newton, no affine, no Huber) "
                         "at 640x480 / 752x480")
    ap.add_argument("--cpu-sample", type=int, default=0,
                    help="frames the oracle tracks for cpu_baseline (0 = auto, ~10-30 s)")
    ap.add_argument("--jacobian", default=None, choices=["forward", "ic"],
                    help="Jacobian form: forward (current image, default) or ic "
                         "(inverse compositional, reference-side rows cached per reference)")
    ap.add_argument("--hessian", default=None, choices=["pass", "cached"],
                    help="paper-configuration workloads (c2p / c2e): the normal matrix summed in "
                         "every pass, or cached per reference and level as in the paper (default)")
    ap.add_argument("--shape", default=None,
                    help="batched forms: fixed tile shape 'cluster,threads' instead of the "
                         "autotuner's pick (profiling runs, where the tuner's timings are distorted)")
    ap.add_argument("--precision", default=None, choices=["fp32", "mixed"],
                    help="storage precision of the levels: c4 / c4b default to mixed (FP16 "
                         "levels and gradients, Kahan sums), every other workload to fp32")
    ap.add_argument("--solve", default=None, choices=["fp64", "fp32"],
                    help="the tracker's 8x8 solve and SE(3) step: fp64 (default: FP64 L D L^T and "
                         "exponential) or fp32 (FP32 factors and exponential increment, FP64 "
                         "state and composition)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-launch-overhead", action="store_true",
                    help="skip the launch-overhead measurement (e.g. for a profiler's launch list)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--table3", action="store_true",
                    help="print the direct-tracking acceptance over a sweep of motion speeds and "
                         "exposure jumps (the Table III analogue) instead of a benchmark line")
    ap.add_argument("--no-batched", action="store_true",
                    help="default workload only: skip the batched forms (C3, C5 plain and "
                         "learned) that the line otherwise carries under 'batched'")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------
class Workload:
    """One camera stream: its frames, reference keyframes and map points."""

    def __init__(self, seed=1, frames=300, N=2000, W=640, H=480, f=525.0, L=4, speed=0.5,
                 ang=30.0, label="C2 single stream", render=True, exposure=True, solver=None,
                 jacobian="forward", max_cost=2.5):
        import synth
        self.cam = synth.camera_for(W, H, f)
        rng_ab = {} if exposure else dict(a_range=(0.0, 0.0), b_range=(0.0, 0.0))
        self.seq = synth.sequence(seed, frames, self.cam, synth.ROOM_LARGE, speed, ang, **rng_ab)
        self.solver = dict(solver or {})    # tracker configuration overrides
        self.max_cost = max_cost
        self.job = (seed, frames, W, H, f)
        self.speed, self.ang = speed, ang
        self.frames = [self.seq.frame(k)[0] for k in range(frames)] if render else None
        self.N, self.L = N, L
        self.refs = {}
        self._tw = {}
        self.jacobian = jacobian
        self.solve = "fp64"          # glt_config.solve of the GPU run (the oracle is FP64)
        if solver:
            self.name = (f"{label}: {W}x{H} uint8, fx=fy={f:g}, {frames}-frame sequence "
                         f"({speed:g} m/s, {ang:g} deg/s, no exposure change), N={N} points, "
                         f"L={L}, const-velocity init, reference every 8 frames")
        else:
            self.name = (f"{label}: {W}x{H} uint8, fx=fy={f:g}, {frames}-frame sequence "
                         f"({speed:g} m/s, {ang:g} deg/s), N={N} points, L={L}, Huber 9, "
                         f"<=10 LM iters/level, const-velocity init, reference every 8 frames")

    def ref_points(self, r):
        import synth
        if r not in self.refs:
            self.refs[r] = synth.reference_points(self.seq, r, self.N, 0.5, 8.0)[1]
        return self.refs[r]

    def T_ref_world(self, r):
        if r not in self._tw:
            self._tw[r] = pose_inv(self.seq.T_wc[r])
        return self._tw[r]


def pose_mul(A, B):
    out = np.empty((3, 4))
    np.matmul(A[:, :3], B, out=out)
    out[:, 3] += A[:, 3]
    return out


def orthonormalised(T):
    """Rotation projected back onto SO(3) (Gram-Schmidt on the rows): the
    constant-velocity extrapolation would otherwise amplify rounding."""
    r0, r1 = T[0, :3], T[1, :3]
    q0 = r0 / math.sqrt(r0 @ r0)
    q1 = r1 - (r1 @ q0) * q0
    q1 = q1 / math.sqrt(q1 @ q1)
    out = T.copy()
    out[0, :3] = q0
    out[1, :3] = q1
    out[2, :3] = (q0[1] * q1[2] - q0[2] * q1[1], q0[2] * q1[0] - q0[0] * q1[2],
                  q0[0] * q1[1] - q0[1] * q1[0])
    return out


def pose_inv(A):
    out = np.empty((3, 4))
    out[:, :3] = A[:, :3].T
    out[:, 3] = -(out[:, :3] @ A[:, 3])
    return out


class SequenceDriver:
    """Host-side loop around the tracker, shaped like the paper's tween-frame
    schedule (Sec. III, Sec. IV-D): constant-velocity initial pose, affine
    brightness carried over from the previous frame of the same reference; a
    frame is accepted if the tracker reports no failure, at least half of the
    8N samples are valid and the robust photometric error (mean Huber energy)
    is below `max_cost`.  A rejected frame, or the `interval`-th frame since
    the last reference, is handed to the indirect pipeline, which here is the
    renderer's true pose and depth: that frame becomes the new reference."""

    def __init__(self, wl: Workload, interval=8, max_cost=None):
        from paper_2607_16897_gb300.tween import TweenSwitch
        self.wl = wl
        self.interval = interval
        self.max_cost = wl.max_cost if max_cost is None else max_cost
        p = wl.solver.get("pattern", 0)
        self.switch = TweenSwitch(max_direct=interval, max_cost=self.max_cost,
                                  samples_per_point=8 if p == 0 else p * p)
        self.rejected = 0
        self.r = 0
        self.since = 0
        self.Tw = {0: wl.T_ref_world(0)}   # estimated world->camera per frame
        self.ab = (0.0, 0.0)
        self.need_refresh = True

    def motion(self, k):
        """The last inter-frame motion before frame k, T_{k-1} T_{k-2}^-1
        (identity before two tracked frames)."""
        Tpp = self.Tw.get(k - 2)
        return pose_mul(self.Tw[k - 1], pose_inv(Tpp)) if Tpp is not None else I34

    def init_for(self, k):
        return pose_mul(pose_mul(self.motion(k), self.Tw[k - 1]),
                        pose_inv(self.wl.T_ref_world(self.r)))

    def ab_init(self):
        return self.ab

    def record(self, k, res):
        self.Tw[k] = orthonormalised(pose_mul(res["T"], self.wl.T_ref_world(self.r)))
        self.ab = (float(res["a"]), float(res["b"]))
        self.Tw.pop(k - 3, None)
        self.since += 1
        bad = not self.switch.direct_ok(res, self.wl.N)
        self.switch.after_direct(res, self.wl.N)
        if bad:
            # the indirect pipeline re-localises this frame
            self.Tw[k] = self.wl.T_ref_world(k)
            self.rejected += 1
        if self.since >= self.interval or bad:
            self.need_refresh = True

    def refresh(self, k):
        """The reference becomes frame k (its true pose, as the indirect
        pipeline would provide); returns True if a refresh happened."""
        if not self.need_refresh:
            return False
        self.r = k
        self.Tw[k] = self.wl.T_ref_world(k)
        self.ab = (0.0, 0.0)
        self.since = 0
        self.need_refresh = False
        return True


def poses_mul(A, B):
    """Batched pose_mul over the leading axis: (S, 3, 4) x (S, 3, 4)."""
    out = np.matmul(A[:, :, :3], B)
    out[:, :, 3] += A[:, :, 3]
    return out


def poses_inv(A):
    """Batched pose_inv: [R^T | -R^T t] for (S, 3, 4)."""
    Rt = np.transpose(A[:, :, :3], (0, 2, 1))
    return np.concatenate([Rt, -np.matmul(Rt, A[:, :, 3:])], axis=2)


def poses_orthonormalised(T):
    """Batched orthonormalised: Gram-Schmidt on the rotation rows."""
    out = np.array(T, np.float64, copy=True)
    r0, r1 = T[:, 0, :3], T[:, 1, :3]
    q0 = r0 / np.sqrt(np.sum(r0 * r0, axis=1, keepdims=True))
    q1 = r1 - np.sum(r1 * q0, axis=1, keepdims=True) * q0
    q1 = q1 / np.sqrt(np.sum(q1 * q1, axis=1, keepdims=True))
    out[:, 0, :3], out[:, 1, :3], out[:, 2, :3] = q0, q1, np.cross(q0, q1)
    return out


class BatchDriver:
    """SequenceDriver for S streams at once (numpy over the stream axis): the
    same constant-velocity start, affine carry-over, acceptance test and
    reference schedule, for the batched end-to-end loop, where one Python
    driver per stream would cost more host time than the GPU step."""

    def __init__(self, wls, interval=8, min_valid_frac=0.5):
        self.wls = wls
        self.S = len(wls)
        self.interval = interval
        self.min_valid = np.array([min_valid_frac * (8 if w.solver.get("pattern", 0) == 0
                                                     else w.solver["pattern"] ** 2) * w.N
                                   for w in wls])
        self.max_cost = np.array([w.max_cost for w in wls], np.float64)
        self.reset()

    def truth(self, idx, k):
        return np.stack([self.wls[s].T_ref_world(k) for s in idx]) if len(idx) else np.zeros((0, 3, 4))

    def reset(self):
        S = self.S
        self.r = np.zeros(S, np.int64)
        self.since = np.zeros(S, np.int64)
        self.need = np.ones(S, bool)
        self.Tk1 = self.truth(range(S), 0)       # world -> camera of the last frame
        self.Tk2 = np.zeros((S, 3, 4))           # and of the one before (if has2)
        self.has2 = np.zeros(S, bool)
        self.Tref = self.Tk1.copy()              # world -> camera of each reference
        self.ab = np.zeros((S, 2))
        self.rejected = np.zeros(S, np.int64)
        self.accepted = np.zeros(S, np.int64)

    def refresh(self, k):
        """Streams that need a new reference take frame k (its true pose, as
        the indirect pipeline would provide); returns their indices."""
        idx = np.nonzero(self.need)[0]
        if len(idx):
            T = self.truth(idx, k)
            self.r[idx] = k
            self.Tk1[idx] = T
            self.Tref[idx] = T
            self.ab[idx] = 0.0
            self.since[idx] = 0
            self.need[idx] = False
        return idx

    def motion(self):
        """A = T_{k-1} T_{k-2}^-1 per stream (identity before two frames)."""
        A = np.broadcast_to(I34, (self.S, 3, 4)).copy()
        if self.has2.any():
            h = self.has2
            A[h] = poses_mul(self.Tk1[h], poses_inv(self.Tk2[h]))
        return A

    def init_for(self):
        return poses_mul(poses_mul(self.motion(), self.Tk1), poses_inv(self.Tref))

    def record(self, k, T, a, b, status, n_valid, cost):
        Tw = poses_orthonormalised(poses_mul(T, self.Tref))
        self.ab = np.stack([a, b], 1).astype(np.float64)
        self.since += 1
        ok = (status == 0) & (n_valid >= self.min_valid) & np.isfinite(cost) & (cost <= self.max_cost)
        bad = np.nonzero(~ok)[0]
        if len(bad):
            Tw[bad] = self.truth(bad, k)
        self.rejected += ~ok
        self.accepted += ok
        self.Tk2, self.Tk1, self.has2 = self.Tk1, Tw, np.ones(self.S, bool)
        self.need |= (self.since >= self.interval) | ~ok


def pose_error(wl, k, r, T):
    import synth
    Tt = synth.relative(wl.seq.T_wc[r], wl.seq.T_wc[k])
    dR = T[:, :3].T @ Tt[:, :3]
    s = 0.5 * np.linalg.norm([dR[2, 1] - dR[1, 2], dR[0, 2] - dR[2, 0], dR[1, 0] - dR[0, 1]])
    return float(np.arctan2(s, 0.5 * (np.trace(dR) - 1))), float(np.linalg.norm(T[:, 3] - Tt[:, 3]))


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def proposal_weights():
    w = np.load(WEIGHTS_PATH).astype(np.float32)
    if w.size != 189064:
        raise ValueError(f"{WEIGHTS_PATH}: {w.size} values, expected 189064")
    return w


def fp32_peak_tflops(sm_mhz):
    # 152 SMs x 128 FP32 lanes x 2 flops (FMA) per clock
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


# ---------------------------------------------------------------------------
# oracle timing (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------
def oracle_track_sequence(wl, frames, inits=None, proposal=None, motions=None):
    """Tracks frames 1..frames with the FP64 oracle; returns (seconds spent in
    pyramid+track, results, inits used).  inits: optional {k: (r, T_init, ab)}
    to replay exactly the GPU's initial states and references.  proposal:
    optional oracle network parameters (BF16-rounded, FP64) applied to each
    initial state, with motions[k] the inter-frame motion (3x4) behind the
    network's motion input."""
    import oracle
    K = wl.cam.K
    trk = oracle.OracleTracker(wl.cam.W, wl.cam.H, K, levels=wl.L, jacobian=wl.jacobian, **wl.solver)
    drv = SequenceDriver(wl)
    t_track = 0.0
    out, used = {}, {}
    cur_ref = None
    ref_coarse = None
    for k in range(1, frames + 1):
        if inits is not None:
            r, T_init, ab = inits[k]
        else:
            drv.refresh(k - 1)
            r, T_init, ab = drv.r, drv.init_for(k), drv.ab_init()
        if r != cur_ref:
            trk.build_pyramid(0, wl.frames[r])
            trk.set_map_points(wl.ref_points(r))
            if proposal is not None:
                ref_coarse = oracle.pyramid(wl.frames[r], wl.L)[-1].astype(np.float64)
            cur_ref = r
        t0 = time.perf_counter()
        trk.build_pyramid(1, wl.frames[k])
        if proposal is not None:
            # the oracle network in front of the oracle tracker: its inputs and
            # the composition of its output are the oracle's own arithmetic
            from oracle import nn as onn
            if motions is not None:
                # the inter-frame motion the GPU run handed to its proposal stage
                mk = onn.motion_input(np.asarray(motions[k], np.float64).reshape(3, 4))
            else:
                mk = onn.motion_feature(drv.Tw.get(k - 1), drv.Tw.get(k - 2))
            x = (oracle.pyramid(wl.frames[k], wl.L)[-1].astype(np.float64) - ref_coarse) / 64.0
            y, _ = onn.forward(proposal, x[None, None], mk[None])
            T_init, ab = onn.apply_output(T_init, ab, y[0])
        res = trk.track_frame(T_init, ab)
        t_track += time.perf_counter() - t0
        out[k] = res
        used[k] = (r, T_init, ab)
        if inits is None:
            drv.record(k, res)
    return t_track, out, used


def run_reference(args):
    """The reference arm: the FP64 oracle on the host cores, same workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    W, K = args.warmup, args.steps
    if args.workload in ("c3", "c4b", "c5"):
        import concurrent.futures
        from synth import jobs as rj
        pool = rj.render_pool()
        wls = batch_workloads(args.workload, rank, pool=pool)
        pool.close()
        pool.join()
        for w in wls:
            apply_overrides(w, args)
        pw = None
        if args.workload == "c5":
            from oracle import nn as onn
            pw = onn.unflatten(onn.to_bf16(proposal_weights()))
        F = len(wls[0].frames)
        n = min(F - 1, W + K)
        workers = os.cpu_count() or 1
        t0 = time.perf_counter()
        with concurrent.futures.ThreadPoolExecutor(max_workers=workers) as ex:
            list(ex.map(lambda w: oracle_track_sequence(w, n, proposal=pw), wls))
        t = time.perf_counter() - t0
        frames = n * len(wls)
        name = f"{args.workload.upper()} batched, {len(wls)} streams"
        sample = f"frames 1..{n} of each of the {len(wls)} streams, one host thread per stream"
        cores = workers
        jac = wls[0].jacobian
    else:
        wl = single_workload(args.workload, rank)
        apply_overrides(wl, args)
        n = min(len(wl.frames) - 1, W + K)
        t, _, _ = oracle_track_sequence(wl, n)
        frames = n
        name = wl.name
        sample = f"frames 1..{n} of the sequence, pyramid + track per frame"
        cores = 1
        jac = wl.jacobian
    fps = frames / t
    line = {"metric": "frames tracked/s", "value": fps, "unit": "frames/s", "n_gpus": args.gpus,
            "steps": K, "warmup": W, "ms_per_step": 1000.0 * t / frames, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference", "config": {"workload": name, "jacobian": jac},
            "cpu_baseline": {"value": fps, "unit": "frames/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": fps, "unit": "frames/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import torch
    import paper_2607_16897_gb300 as glt

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = process_group(world)
    wl = single_workload(args.workload, rank)   # replicas: one independent stream per GPU
    apply_overrides(wl, args)
    precision = args.precision or ("mixed" if args.workload == "c4" else "fp32")
    Wd, Hd, L, N = wl.cam.W, wl.cam.H, wl.L, wl.N
    stream = torch.cuda.Stream()
    sh = stream.cuda_stream
    trk = glt.Tracker(Wd, Hd, wl.cam.K, levels=L, max_points=N, precision=precision,
                      jacobian=wl.jacobian, solve=wl.solve, **wl.solver)
    frames_dev = torch.from_numpy(np.stack(wl.frames)).to(f"cuda:{local}")
    frames_pin = torch.from_numpy(np.stack(wl.frames)).pin_memory()
    init_dev = torch.zeros(14, dtype=torch.float64, device=f"cuda:{local}")
    init_pin = torch.zeros(14, dtype=torch.float64).pin_memory()
    out_dev = torch.zeros(glt.RESULT_BYTES, dtype=torch.uint8, device=f"cuda:{local}")
    out_pin = torch.zeros(glt.RESULT_BYTES, dtype=torch.uint8).pin_memory()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=f"cuda:{local}")
    uvd_dev = {}

    def prepare_ref(r):
        # the caller's map points of reference r, on the device (host work,
        # kept outside the refresh events)
        if r not in uvd_dev:
            uvd_dev[r] = torch.from_numpy(wl.ref_points(r)).to(f"cuda:{local}")

    def refresh_dev(r):
        prepare_ref(r)
        trk.build_pyramid(glt.GLT_REF, frames_dev[r], stream=sh)
        trk.set_map_points(uvd_dev[r], stream=sh)

    nF = len(wl.frames)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    ev_ref = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]

    def run_steps(nsteps, timed, record):
        drv = SequenceDriver(wl)
        k = 0
        n_ref = 0
        for i in range(nsteps):
            k += 1
            if k >= nF:            # restart the sequence
                k = 1
                drv = SequenceDriver(wl)
            did = drv.refresh(k - 1)
            r_used = drv.r
            if did:
                prepare_ref(drv.r)
                with torch.cuda.stream(stream):
                    if timed:
                        ev_ref[n_ref][0].record(stream)
                    refresh_dev(drv.r)
                    if timed:
                        ev_ref[n_ref][1].record(stream)
                n_ref += 1
            T_init, ab = drv.init_for(k), drv.ab_init()
            init_pin.copy_(torch.from_numpy(np.concatenate([T_init.ravel(), list(ab)])))
            with torch.cuda.stream(stream):
                init_dev.copy_(init_pin, non_blocking=True)
                flush.zero_()                    # L2 flushed between steps
                if timed:
                    ev[i][0].record(stream)
                # the pyramid kernels and the solve, chained on the device
                trk.track_image_async(frames_dev[k], init_dev, out_dev, stream=sh)
                if timed:
                    ev[i][1].record(stream)
                out_pin.copy_(out_dev, non_blocking=True)
            stream.synchronize()
            res = glt.parse_results(out_pin.numpy())[0]
            drv.record(k, res)
            if record is not None:
                record.append((k, r_used, T_init, ab, res))
        return n_ref

    # warm-up (untimed), then the timed steps
    run_steps(max(args.warmup, 3), False, None)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    torch.cuda.synchronize()
    rec = []
    t_wall0 = time.perf_counter()
    n_ref = run_steps(args.steps, True, rec)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    # the chain overlaps the pyramid kernels with the track kernel's setup:
    # one interval per step
    step_ms = [e0.elapsed_time(e1) for e0, e1 in ev]
    trk_ms = step_ms
    ref_ms = [a.elapsed_time(b) for a, b in ev_ref[:n_ref]]
    dev_s = sum(step_ms) / 1000.0
    dev_s, t_wall = max_over_ranks([dev_s, t_wall], dist, f"cuda:{local}")
    value = aggregate_rate(args.steps, world, dev_s)
    passes = [r[4]["passes"] for r in rec]

    # accuracy vs ground truth along the sequence
    gt = [pose_error(wl, k, r, res["T"]) for (k, r, _, _, res) in rec]
    accuracy = {"median_rot_deg": float(np.rad2deg(np.median([e[0] for e in gt]))),
                "median_trans_mm": float(1000 * np.median([e[1] for e in gt])),
                "max_rot_deg": float(np.rad2deg(max(e[0] for e in gt))),
                "max_trans_mm": float(1000 * max(e[1] for e in gt)),
                "status_nonzero": int(sum(1 for r in rec if r[4]["status"]))}
    launch = None
    if not args.no_launch_overhead:
        launch = launch_overhead(stream, lambda: trk.track_image_async(frames_dev[1], init_dev, out_dev,
                                                                       stream=sh))
        launch["library_call"] = f"glt_track_image_async ({L - 1} pyramid launches + the track launch)"
    # one frame's upload from pinned host memory, timed on its own
    up = torch.empty_like(frames_dev[0])
    u0, u1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        up.copy_(frames_pin[1], non_blocking=True)
        u0.record(stream)
        for _ in range(20):
            up.copy_(frames_pin[1], non_blocking=True)
        u1.record(stream)
    stream.synchronize()
    h2d_frame_ms = u0.elapsed_time(u1) / 20
    # e2e through the C ABI with host buffers (pinned), H2D + D2H inside
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, glt, trk, wl, frames_pin, stream)

    # oracle on a bounded sample, same initial states and references
    cpu = None
    parity = None
    lin_err = None
    if rank == 0 and not args.no_cpu:
        cpu, parity = run_cpu_baseline(args, wl, rec)
        lin_err = linearization_error(glt, wl, rec[-1], precision)

    # roofline of the dominant kernel (the persistent tracker)
    mean_trk = statistics.mean(trk_ms) / 1000.0
    samples_per_launch = statistics.mean(p * samples_per_point(wl) * N for p in passes)
    achieved = flops_per_sample(wl) * samples_per_launch / mean_trk / 1e12
    peaks, src = measured_peaks()
    peak = fp32_peak_tflops(peaks.get("sm_max_mhz", 2070.0))
    # the chain's own yardstick: the fixed part of a pass (reduction, cluster
    # barrier, distributed-shared-memory finish, FP64 tail) with no points
    cl, th = trk.shape()
    floor_us = glt.pass_floor(cl, th, cached=wl.solver.get("hessian") == "cached", stream=sh,
                              solve=wl.solve)
    floor_ms = statistics.mean(passes) * floor_us / 1000.0
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": TRACK_TRAFFIC.get(args.workload),
            "kernel": "track_kernel",
            "peak_source": f"FP32 FMA peak from unit counts (152 SMs x 128 lanes x 2) at "
                           f"{peaks.get('sm_max_mhz', 2070.0):g} MHz ({src} clock)",
            "launch_ms": statistics.mean(trk_ms), "passes_per_launch": statistics.mean(passes),
            "samples_per_launch": samples_per_launch, "flops_per_sample": flops_per_sample(wl),
            "latency_floor": {"us_per_pass": floor_us, "shape": [cl, th],
                              "floor_ms_per_launch": floor_ms,
                              "frac": floor_ms / statistics.mean(trk_ms),
                              "what": "passes x (block reduction + cluster barrier + "
                                      "distributed-shared-memory finish + FP64 tail) with no "
                                      "points (glt_debug_pass_floor), over the measured launch"}}
    if rank == 0:
        line = {"metric": "frames tracked/s", "value": value, "unit": "frames/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1000.0 * dev_s / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f16 storage / f32 math" if precision == "mixed" else "f32",
                "data": "synthetic",
                "config": {"workload": wl.name, "jacobian": wl.jacobian,
                           "hessian": wl.solver.get("hessian", "pass"), "solve": wl.solve,
                           "global_batch": world,
                           "streams_per_gpu": 1,
                           "parallelism": f"replicas x{world}",
                           "l2": "flushed between steps (256 MB write, outside the step events)",
                           "timing": "sum of per-step CUDA-event times (pyramid + track)"},
                "step_ms_percentiles": step_percentiles(step_ms),
                "breakdown_ms": {"pyramid": "chained with the track launch (inside 'track')",
                                 "track": statistics.mean(trk_ms),
                                 "reference_refresh": statistics.mean(ref_ms) if ref_ms else None,
                                 "h2d_frame_upload": h2d_frame_ms,
                                 "wall_per_step": 1000.0 * t_wall / args.steps},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
                "gpu_launches": args.steps * (L + (1 if precision == "mixed" else 0)) + n_ref * L,
                "launch_overhead": launch,
                "parity_vs_oracle": parity, "accuracy_vs_truth": accuracy,
                "linearization_error_vs_oracle": lin_err}
        return line
    return None


def run_e2e(args, glt, trk, wl, frames_pin, stream):
    """Same frames through the C ABI with HOST (pinned) buffers, the way a
    per-frame caller uses the library: every frame is one glt_track_image call
    started from the tracker's own constant-velocity state (frame upload,
    chained pyramid + solve, result read back, state update); the host keeps
    the tween-frame schedule (acceptance test, reference every 8 frames) and
    hands a new reference in through glt_build_pyramid / glt_set_map_points
    with host buffers and glt_set_state (the reference's pose from the
    indirect pipeline, as SequenceDriver does)."""
    import torch
    from paper_2607_16897_gb300.tween import TweenSwitch
    sh = stream.cuda_stream
    nF = len(wl.frames)
    h2d = d2h = 0
    refs_pin = {}
    steps = args.steps
    # map points the caller holds in pinned memory, like the frames (prepared
    # before the timed loop: every reference the device-timed run used)
    for r in sorted(set(range(0, nF, 8)) | set(wl.refs)):
        refs_pin[r] = torch.from_numpy(wl.ref_points(r)).pin_memory()
    frames_np = [f.numpy() for f in frames_pin]
    p = wl.solver.get("pattern", 0)
    interval = 8

    def new_reference(k, motion):
        """Frame k becomes the reference; the state restarts there with the
        given camera motion (identity at a sequence start)."""
        nonlocal h2d
        if k not in refs_pin:
            refs_pin[k] = torch.from_numpy(wl.ref_points(k)).pin_memory()
        trk.build_pyramid(glt.GLT_REF, frames_np[k], stream=sh)
        trk.set_map_points(refs_pin[k].numpy(), stream=sh)
        h2d += wl.frames[k].nbytes + refs_pin[k].numel() * 4
        st = trk.get_state()
        for i in range(12):
            st.motion[i] = motion[i // 4, i % 4]
        trk.set_state(st)

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    k, r, since = 1, 0, 0
    switch = TweenSwitch(max_direct=interval, max_cost=wl.max_cost,
                         samples_per_point=8 if p == 0 else p * p)
    new_reference(0, I34)
    prev = None                      # (frame, pose relative to its reference, reference)
    for i in range(steps):
        res = trk.track_image(frames_np[k], stream=sh)
        h2d += wl.frames[k].nbytes + 14 * 8
        d2h += glt.RESULT_BYTES
        ok = switch.direct_ok(res, wl.N)
        switch.after_direct(res, wl.N)
        since += 1
        kn = k + 1 if k + 1 < nF else 1
        if kn == 1:                  # the sequence starts over
            new_reference(0, I34)
            r, since, prev = 0, 0, None
        elif not ok or since >= interval:
            # frame k becomes the reference at its true pose; the motion is
            # that pose against the previous frame's estimate (or truth)
            Tw_k = wl.T_ref_world(k)
            if prev is None or prev[0] == prev[2]:
                Tw_prev = wl.T_ref_world(k - 1)
            else:
                Tw_prev = orthonormalised(pose_mul(prev[1], wl.T_ref_world(prev[2])))
            new_reference(k, pose_mul(Tw_k, pose_inv(Tw_prev)))
            r, since, prev = k, 0, (k, None, k)
        else:
            prev = (k, res["T"], r)
        k = kn
    torch.cuda.synchronize()
    t = time.perf_counter() - t0
    return {"value": steps / t, "unit": "frames/s", "h2d_bytes_per_step": h2d / steps,
            "d2h_bytes_per_step": d2h / steps,
            "note": "one glt_track_image call per frame from pinned host memory, started from the "
                    "tracker's constant-velocity state (upload, chained pyramid + solve, result read "
                    "back), reference refreshes through the C ABI with host buffers, tween-frame "
                    "schedule on the host"}


def launch_overhead(stream, enqueue, reps=1000):
    """Launch cost, measured apart from the timed steps: the device time per
    empty kernel inside a graph of 100 (events around 20 replays), the device
    time per replay of a one-kernel graph issued back to back, and the host
    time to enqueue one call of the library (`enqueue`, the median over
    `reps` // 10 calls; the kernels it launches are not waited for)."""
    import torch

    def graph_of(n):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            for _ in range(n):
                torch.cuda._sleep(0)
        return g

    def per_replay(g, n):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            g.replay()
            e0.record(stream)
            for _ in range(n):
                g.replay()
            e1.record(stream)
        stream.synchronize()
        return 1000.0 * e0.elapsed_time(e1) / n

    g100, g1 = graph_of(100), graph_of(1)
    out = {"empty_kernel_in_graph_us": per_replay(g100, 20) / 100,
           "empty_graph_replay_us": per_replay(g1, reps)}
    host = []
    for _ in range(max(reps // 10, 5)):
        t0 = time.perf_counter()
        enqueue()
        host.append(time.perf_counter() - t0)
    stream.synchronize()
    out["library_call_host_us"] = 1e6 * statistics.median(host)
    return out


def run_cpu_baseline(args, wl, rec):
    """The oracle on the first n timed frames with the GPU run's initial
    states and references: frames/s on one host core, and the pose
    difference GPU vs oracle for the same inputs."""
    n = args.cpu_sample if args.cpu_sample > 0 else 299
    n = min(n, len(rec))
    inits = {k: (r, T_init, ab) for (k, r, T_init, ab, _) in rec[:n]}
    assert sorted(inits) == list(range(1, n + 1))
    t, out, _ = oracle_track_sequence(wl, n, inits=inits)
    gpu = {k: res for (k, _, _, _, res) in rec[:n]}
    rot, trans = [], []
    for k in range(1, n + 1):
        dR = gpu[k]["T"][:, :3].T @ out[k]["T"][:, :3]
        s = 0.5 * np.linalg.norm([dR[2, 1] - dR[1, 2], dR[0, 2] - dR[2, 0], dR[1, 0] - dR[0, 1]])
        rot.append(float(np.arctan2(s, 0.5 * (np.trace(dR) - 1))))
        trans.append(float(np.linalg.norm(gpu[k]["T"][:, 3] - out[k]["T"][:, 3])))
    cpu = {"value": n / t, "unit": "frames/s", "cores": 1, "kind": "oracle",
           "sample": f"frames 1..{n} of the sequence (pyramid + track each, FP64 C oracle, "
                     f"same initial states and references as the GPU run)"}
    parity = {"frames": n, "max_rot_rad": max(rot), "max_trans_m": max(trans),
              "tolerance": {"rot_rad": 1e-5, "trans_m": 1e-5}}
    return cpu, parity


def linearization_error(glt, wl, rec_entry, precision):
    """H, g and E of one linearisation on every level, GPU (this precision)
    against the FP64 oracle, at the initial state of the given frame:
    |dH|_F / |H|_F, |dg| / |g|, |dE| / E, and whether the sample counts match."""
    import oracle
    k, r, T_init, ab, _ = rec_entry
    trk = glt.Tracker(wl.cam.W, wl.cam.H, wl.cam.K, levels=wl.L, max_points=wl.N, precision=precision,
                      jacobian=wl.jacobian, solve=wl.solve, **wl.solver)
    trk.build_pyramid(glt.GLT_REF, wl.frames[r])
    trk.set_map_points(wl.ref_points(r))
    trk.build_pyramid(glt.GLT_CUR, wl.frames[k])
    o = oracle.OracleTracker(wl.cam.W, wl.cam.H, wl.cam.K, levels=wl.L, jacobian=wl.jacobian,
                             **wl.solver)
    o.build_pyramid(0, wl.frames[r])
    o.set_map_points(wl.ref_points(r))
    o.build_pyramid(1, wl.frames[k])
    out = {"frame": k, "state": "constant-velocity initial state", "levels": []}
    for l in range(wl.L):
        gd = trk.debug_linearize(l, T_init, ab[0], ab[1], want_res=False)
        od = o.debug_linearize(l, T_init, ab[0], ab[1], per_sample=False)
        out["levels"].append({
            "level": l,
            "H_rel": float(np.linalg.norm(gd["H"] - od["H"]) / np.linalg.norm(od["H"])),
            "g_rel": float(np.linalg.norm(gd["g"] - od["g"]) / np.linalg.norm(od["g"])),
            "E_rel": float(abs(gd["E"] - od["E"]) / od["E"]),
            "n_equal": bool(gd["n"] == od["n"])})
    trk.close()
    return out


# the paper's configuration: p x p patches, IC Jacobians with the Hessian
# cached per reference and level, plain Gauss-Newton with 10 iterations on each
# of 6 levels, no affine brightness, no Huber weights
PAPER_SOLVER = dict(affine=False, lambda0=0.0, accept_step=1e30, eps_step=0.0,
                    eps_step_coarse=0.0, huber_k=1e30, hessian="cached")


def apply_overrides(wl, args):
    """--jacobian / --hessian / --solve on a workload (the cached Hessian
    exists only with the inverse-compositional rows)."""
    if args.jacobian:
        wl.jacobian = args.jacobian
    if getattr(args, "hessian", None) and "hessian" in wl.solver:
        wl.solver["hessian"] = args.hessian
    if getattr(args, "solve", None):
        wl.solve = args.solve
    if wl.jacobian != "ic" and wl.solver.get("hessian") == "cached":
        wl.solver["hessian"] = "pass"


def single_workload(kind, rank=0):
    if kind == "c2p":
        return Workload(seed=stream_seed(kind, 0, rank), frames=300, N=2000, W=640, H=480, f=525.0, L=6,
                        exposure=False, solver=dict(PAPER_SOLVER, pattern=7), jacobian="ic",
                        max_cost=50.0,
                        label="C2 in the paper's configuration (TUM-like, 7x7 patches, IC rows "
                              "and the Hessian cached per reference, 6 levels, 10 GN iterations "
                              "per level, no affine, no Huber)")
    if kind == "c2e":
        return Workload(seed=stream_seed(kind, 0, rank), frames=300, N=2000, W=752, H=480, f=458.0, L=6,
                        exposure=False, solver=dict(PAPER_SOLVER, pattern=11), jacobian="ic",
                        max_cost=50.0,
                        label="752x480 in the paper's configuration (EuRoC-like, 11x11 patches, "
                              "IC rows and the Hessian cached per reference, 6 levels, 10 GN "
                              "iterations per level, no affine, no Huber)")
    if kind == "c4":
        return Workload(seed=stream_seed(kind, 0, rank), frames=300, N=8000, W=1280, H=720, f=1050.0, L=5,
                        speed=1.0, ang=60.0, label="C4 single stream")
    return Workload(seed=stream_seed("c2", 0, rank))


def batch_workloads(kind, rank=0, nstreams=None, frames=24, pool=None):
    """C3: 64 streams, sizes uniform over {320x240, 640x480, 752x480, 1280x720}
    (f = 0.8 W), N uniform in [300, 4000], L = 4.  C4b: 64 streams of the C4
    configuration (1280x720, N = 8000, L = 5, 1 m/s, 60 deg/s).  C5: 256
    streams of 640x480 (f = 525), N = 2000, L = 5 (40 x 30 coarsest level),
    held-out seeds 5000..5255 with the proposal's training motion range (mean
    speed 0.5-2 m/s, 30-90 deg/s per stream).  With a process pool the
    frames and the references at multiples of 8 are rendered in parallel."""
    from synth import jobs as rj
    rng = np.random.default_rng(1000 + rank)
    sizes = [(320, 240), (640, 480), (752, 480), (1280, 720)]
    nstreams = nstreams or (256 if kind == "c5" else 64)
    wls = []
    for s in range(nstreams):
        if kind == "c4b":
            wls.append(Workload(seed=stream_seed(kind, s, rank), frames=frames, N=8000, W=1280, H=720,
                                f=1050.0, L=5, speed=1.0, ang=60.0, label="C4b stream",
                                render=pool is None))
        elif kind == "c5":
            seed = stream_seed(kind, s, rank)
            v, w = rj.stream_motion(seed)
            wls.append(Workload(seed=seed, frames=frames, N=2000, W=640, H=480, f=525.0, L=5,
                                speed=v, ang=w, label="C5 stream", render=pool is None))
        else:
            W, H = sizes[int(rng.integers(4))]
            N = int(rng.integers(300, 4001))
            wls.append(Workload(seed=stream_seed(kind, s, rank), frames=frames, N=N, W=W, H=H,
                                f=0.8 * W, L=4, label="C3 stream", render=pool is None))
    if pool is not None:
        jobs = [w.job + (k, 0, w.speed, w.ang) for w in wls for k in range(frames)]
        imgs = pool.map(rj._render_job, jobs, chunksize=8)
        for i, w in enumerate(wls):
            w.frames = [imgs[i * frames + k][0] for k in range(frames)]
        refs = [(i, r) for i in range(len(wls)) for r in range(0, frames - 1, 8)]
        pts = pool.map(rj._render_job, [wls[i].job + (r, wls[i].N, wls[i].speed, wls[i].ang)
                                          for i, r in refs], chunksize=4)
        for (i, r), (_, uvd) in zip(refs, pts):
            wls[i].refs[r] = uvd
    return wls


def run_batch(args):
    """Batched form: every stream's next frame tracked by one graph replay
    (pyramids of all streams + one persistent track launch).  C5 runs the same
    streams twice, plain and with the learned proposal stage in the graph."""
    import torch
    import paper_2607_16897_gb300 as glt
    from paper_2607_16897_gb300 import proposal as prop

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    from synth import jobs as rj
    pool = rj.render_pool()            # spawned before the first CUDA call
    wls = batch_workloads(args.workload, rank, pool=pool)
    pool.close()
    pool.join()
    for w in wls:
        apply_overrides(w, args)
    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    dist = process_group(world)
    precision = args.precision or ("mixed" if args.workload == "c4b" else "fp32")
    use_prop = args.workload == "c5"
    S = len(wls)
    F = len(wls[0].frames)
    stream = torch.cuda.Stream()
    sh = stream.cuda_stream
    trks = [glt.Tracker(w.cam.W, w.cam.H, w.cam.K, levels=w.L, max_points=w.N, precision=precision,
                        jacobian=w.jacobian, solve=w.solve, **w.solver) for w in wls]
    batch = glt.Batch(trks)
    frames_dev = [torch.from_numpy(np.stack(w.frames)).to(dev) for w in wls]
    # host frames in pinned memory, laid out per step (every stream's frame k
    # contiguous), so that a step's upload is one copy; per-stream views serve
    # the reference refreshes
    frame_off = np.concatenate([[0], np.cumsum([w.cam.W * w.cam.H for w in wls])]).astype(np.int64)
    step_np = np.empty((F, int(frame_off[-1])), np.uint8)
    for s_, w in enumerate(wls):
        for k_ in range(F):
            step_np[k_, frame_off[s_]:frame_off[s_ + 1]] = w.frames[k_].ravel()
    step_pin = torch.from_numpy(step_np).pin_memory()
    del step_np
    frames_pin = [[step_pin[k_, frame_off[s_]:frame_off[s_ + 1]].view(w.cam.H, w.cam.W) for k_ in range(F)]
                  for s_, w in enumerate(wls)]
    ptr_dev = torch.zeros(S, dtype=torch.int64, device=dev)
    ptr_pin = torch.zeros(S, dtype=torch.int64).pin_memory()
    init_dev = torch.zeros((S, 14), dtype=torch.float64, device=dev)
    init_pin = torch.zeros((S, 14), dtype=torch.float64).pin_memory()
    # each stream's last inter-frame motion (3x4): the proposal stage's input
    motion_dev = torch.zeros((S, 12), dtype=torch.float64, device=dev)
    motion_pin = torch.zeros((S, 12), dtype=torch.float64).pin_memory()
    out_dev = torch.zeros(S * glt.RESULT_BYTES, dtype=torch.uint8, device=dev)
    out_pin = torch.zeros(S * glt.RESULT_BYTES, dtype=torch.uint8).pin_memory()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    net = glt.NN(S, prop.load_weights()) if use_prop else None
    uvd_dev = {}

    uvd_pin = {}

    def pin_refs():
        # map points the caller holds in pinned memory, like the frames
        for s_, w in enumerate(wls):
            for r in w.refs:
                if (s_, r) not in uvd_pin:
                    uvd_pin[(s_, r)] = torch.from_numpy(w.refs[r]).pin_memory()

    def refresh(s, r, host=False):
        t = trks[s]
        if host:
            # pinned host buffers through the C ABI (asynchronous uploads)
            key = (s, r)
            if key not in uvd_pin:
                uvd_pin[key] = torch.from_numpy(wls[s].ref_points(r)).pin_memory()
            t.build_pyramid(glt.GLT_REF, frames_pin[s][r].numpy(), stream=sh)
            t.set_map_points(uvd_pin[key].numpy(), stream=sh)
        else:
            key = (s, r)
            if key not in uvd_dev:
                uvd_dev[key] = torch.from_numpy(wls[s].ref_points(r)).to(dev)
            t.build_pyramid(glt.GLT_REF, frames_dev[s][r], stream=sh)
            t.set_map_points(uvd_dev[key], stream=sh)

    drvs = [SequenceDriver(w) for w in wls]

    def restart():
        for d in drvs:
            d.__init__(d.wl)
        for s in range(S):
            drvs[s].refresh(0)
            refresh(s, 0)

    init_np, motion_np, ptr_np = init_pin.numpy(), motion_pin.numpy(), ptr_pin.numpy()
    frame_ptrs = [[f[k].data_ptr() for k in range(F)] for f in frames_dev]

    def prepare(k):
        for s in range(S):
            d = drvs[s]
            init_np[s, :12] = d.init_for(k).ravel()
            init_np[s, 12:] = d.ab_init()
            if use_prop:
                motion_np[s] = d.motion(k).ravel()
            ptr_np[s] = frame_ptrs[s][k]

    def finish(k, record):
        res = glt.parse_results(out_pin.numpy())
        n_ref = 0
        for s in range(S):
            if record is not None:
                record.append((s, k, drvs[s].r, init_pin[s].numpy().copy(), res[s],
                               motion_pin[s].numpy().copy()))
            drvs[s].record(k, res[s])
            if k + 1 < F and drvs[s].refresh(k):
                refresh(s, k)
                n_ref += 1
        return res, n_ref

    def run_steps(nsteps, timed, record):
        """Device-resident steps: frames already in HBM, L2 flushed before each
        replay (outside its events), one SequenceDriver per stream."""
        restart()
        stream.synchronize()
        k = 0
        dev_ms, n_ref_total = [], 0
        for i in range(nsteps):
            k += 1
            if k >= F:
                k = 1
                restart()
            prepare(k)
            with torch.cuda.stream(stream):
                flush.zero_()
                ptr_dev.copy_(ptr_pin, non_blocking=True)
                init_dev.copy_(init_pin, non_blocking=True)
                motion_dev.copy_(motion_pin, non_blocking=True)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                batch.replay(stream=sh)
                e1.record(stream)
                out_pin.copy_(out_dev, non_blocking=True)
            stream.synchronize()
            if timed:
                dev_ms.append(e0.elapsed_time(e1))
            _, nr = finish(k, record)
            n_ref_total += nr
        return dev_ms, n_ref_total

    def run_e2e_steps(nsteps):
        """The end-to-end loop: host frames and states in, results out, every
        step; the drivers of all streams advance together (BatchDriver, the
        same schedule as SequenceDriver)."""
        bd = BatchDriver(wls)
        step_dev = torch.empty(int(frame_off[-1]), dtype=torch.uint8, device=dev)
        ptr_np[:] = step_dev.data_ptr() + frame_off[:-1]
        h2d = d2h = 0

        def refresh_streams(idx, k):
            nonlocal h2d
            for s_ in idx:
                refresh(int(s_), k, host=True)
                h2d += wls[s_].cam.W * wls[s_].cam.H + uvd_pin[(int(s_), k)].numel() * 4

        with torch.cuda.stream(stream):
            ptr_dev.copy_(ptr_pin, non_blocking=True)
        refresh_streams(bd.refresh(0), 0)
        k = 1
        res = np.frombuffer(out_pin.numpy(), dtype=glt.RESULT_DTYPE)
        for _ in range(nsteps):
            init_np[:, :12] = bd.init_for().reshape(S, 12)
            init_np[:, 12:] = bd.ab
            if use_prop:
                motion_np[:] = bd.motion().reshape(S, 12)
            with torch.cuda.stream(stream):
                step_dev.copy_(step_pin[k], non_blocking=True)
                init_dev.copy_(init_pin, non_blocking=True)
                if use_prop:
                    motion_dev.copy_(motion_pin, non_blocking=True)
                batch.replay(stream=sh)
                out_pin.copy_(out_dev, non_blocking=True)
            h2d += step_pin[k].numel() + init_pin.numel() * 8 + (motion_pin.numel() * 8 if use_prop else 0)
            d2h += out_pin.numel()
            stream.synchronize()
            bd.record(k, res["T"].reshape(S, 3, 4), res["a"], res["b"], res["status"], res["n_valid"],
                      res["cost"])
            if k + 1 < F:
                refresh_streams(bd.refresh(k), k)
                k += 1
            else:
                bd.reset()
                refresh_streams(bd.refresh(0), 0)
                k = 1
        return h2d, d2h

    # every stream starts on its frame 0 as reference; autotune the tile shape
    # on frame 1 (plain form)
    restart()
    prepare(1)
    with torch.cuda.stream(stream):
        ptr_dev.copy_(ptr_pin, non_blocking=True)
        init_dev.copy_(init_pin, non_blocking=True)
        batch.build_pyramid(ptr_dev, stream=sh)
    stream.synchronize()
    if args.shape:
        c, t = (int(v) for v in args.shape.split(","))
        batch.set_shape(c, t)
        shape = (c, t, None)
    else:
        shape = batch.autotune(init_dev, out_dev, reps=3, stream=sh)
    classes = batch.classes()
    class_table = batch.class_table()

    def measure(form):
        """Captures the step graph of `form` ("plain" / "proposal") and times it."""
        batch.set_proposal(net if form == "proposal" else None, motion_dev if form == "proposal" else None)
        batch.capture(ptr_dev, init_dev, out_dev, stream)
        run_steps(max(args.warmup, 3), False, None)
        if dist:
            dist.barrier()
        clocks = ClockSampler(local)
        clocks.start()
        torch.cuda.synchronize()
        rec = []
        t0 = time.perf_counter()
        dev_ms, n_ref = run_steps(args.steps, True, rec)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t0
        clk = clocks.stop()
        dev_s = sum(dev_ms) / 1000.0
        dev_s, t_wall = max_over_ranks([dev_s, t_wall], dist, dev)
        gt = [pose_error(wls[r[0]], r[1], r[2], r[4]["T"]) for r in rec]
        acc = {"median_rot_deg": float(np.rad2deg(np.median([e[0] for e in gt]))),
               "median_trans_mm": float(1000 * np.median([e[1] for e in gt])),
               "p99_trans_mm": float(1000 * np.percentile([e[1] for e in gt], 99)),
               "status_nonzero": int(sum(1 for r in rec if r[4]["status"])),
               "rejected_frames": int(sum(d.rejected for d in drvs)),
               "direct_acceptance": float(
                   sum(d.switch.direct_accepted for d in drvs)
                   / max(1, sum(d.switch.direct_accepted + d.switch.direct_rejected for d in drvs)))}
        return dict(dev_ms=dev_ms, dev_s=dev_s, t_wall=t_wall, clk=clk, rec=rec, n_ref=n_ref,
                    value=aggregate_rate(S * args.steps, world, dev_s), accuracy=acc,
                    iters_per_frame=float(np.mean([r[4]["iters_total"] for r in rec])),
                    passes_per_frame=float(np.mean([r[4]["passes"] for r in rec])))

    forms = ["plain", "proposal"] if use_prop else ["plain"]
    runs = {f: measure(f) for f in forms}
    head = runs[forms[-1]]
    launch = None
    if not args.no_launch_overhead:
        launch = launch_overhead(stream, lambda: batch.replay(stream=sh), reps=200)
        launch["library_call"] = "glt_batch_replay (the whole step graph)"
    value, dev_s, dev_ms, rec = head["value"], head["dev_s"], head["dev_ms"], head["rec"]
    e2e = None
    if not args.no_e2e:
        pin_refs()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        h2d, d2h = run_e2e_steps(args.steps)
        torch.cuda.synchronize()
        te = time.perf_counter() - t1
        e2e = {"value": S * args.steps / te, "unit": "frames/s",
               "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
               "note": "every step copies all streams' frames from pinned host memory (one copy), "
                       "replays the graph, reads all results back and runs the sequence drivers of "
                       "all streams at once (BatchDriver); reference refreshes through the C ABI "
                       "with host buffers"}
    cpu = parity = None
    if rank == 0 and not args.no_cpu:
        pw = None
        if use_prop:
            from oracle import nn as onn
            pw = onn.unflatten(onn.to_bf16(proposal_weights()))
        cpu, parity = batch_cpu_baseline(wls, rec, proposal=pw)
    # roofline of the persistent tracker (the graph's dominant kernel)
    samples = sum(r[4]["passes"] * samples_per_point(wls[r[0]]) * wls[r[0]].N for r in rec) / args.steps
    achieved = sum(r[4]["passes"] * samples_per_point(wls[r[0]]) * wls[r[0]].N * flops_per_sample(wls[r[0]])
                   for r in rec) / args.steps / (dev_s / args.steps) / 1e12
    peaks, src = measured_peaks()
    peak = fp32_peak_tflops(peaks.get("sm_max_mhz", 2070.0))
    if rank == 0:
        L = max(w.L for w in wls)
        if args.workload == "c4b":
            desc = "1280x720, N=8000, L=5, 1 m/s, 60 deg/s"
        elif use_prop:
            desc = ("640x480 (f=525), N=2000, L=5, held-out seeds 5000-5255, mean speed 0.5-2 m/s "
                    "and 30-90 deg/s per stream; learned proposal (3 conv + 2 fc, BF16 weights) "
                    "in the graph ahead of the track launch")
        else:
            desc = "sizes uniform over 320x240/640x480/752x480/1280x720, N uniform 300-4000, L=4"
        # L - 1 pyramid levels, the FP16 packing, the proposal stage, the track kernel
        launches = L + (1 if precision == "mixed" else 0) + (1 if use_prop else 0)
        line = {"metric": "frames tracked/s", "value": value, "unit": "frames/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1000.0 * dev_s / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f16 storage / f32 math" if precision == "mixed" else "f32",
                "data": "synthetic",
                "config": {"workload": (f"{args.workload.upper()} batched: {S} streams in one graph "
                                        f"replay (pyramids + one persistent track launch); " + desc
                                        + f", {F}-frame sequences, reference every 8 frames"),
                           "jacobian": wls[0].jacobian, "solve": wls[0].solve,
                           "global_batch": world * S, "streams_per_gpu": S,
                           "parallelism": f"replicas x{world}",
                           "autotuned_shape": {"cluster": shape[0], "threads": shape[1],
                                               "ms": shape[2],
                                               "heavy_streams": classes["heavy"],
                                               "light_shape": list(classes["light_shape"]),
                                               "classes": [{"first": f, "streams": n, "cluster": c,
                                                            "threads": t} for f, n, c, t in class_table]},
                           "l2": "flushed between steps (256 MB write, outside the step events)",
                           "timing": "sum of per-step CUDA-event times around the graph replay"},
                "step_ms_percentiles": step_percentiles(dev_ms),
                "breakdown_ms": {"replay": statistics.mean(dev_ms),
                                 "wall_per_step": 1000.0 * head["t_wall"] / args.steps},
                "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                             "frac": achieved / peak, "traffic": TRACK_TRAFFIC.get(args.workload),
                             "kernel": "track_kernel",
                             "peak_source": f"FP32 FMA peak from unit counts at "
                                            f"{peaks.get('sm_max_mhz', 2070.0):g} MHz ({src} clock)",
                             "samples_per_step": samples},
                "cpu_baseline": cpu, "e2e": e2e, "clocks": head["clk"],
                "gpu_launches": args.steps * launches + head["n_ref"] * L, "launch_overhead": launch,
                "parity_vs_oracle": parity, "accuracy_vs_truth": head["accuracy"],
                "iters_per_frame": head["iters_per_frame"],
                "passes_per_frame": head["passes_per_frame"]}
        if use_prop:
            pl = runs["plain"]
            agree = []
            for a, b in zip(pl["rec"], head["rec"]):
                if a[:3] == b[:3]:
                    dR = a[4]["T"][:, :3].T @ b[4]["T"][:, :3]
                    agree.append((np.arccos(np.clip(0.5 * (np.trace(dR) - 1), -1, 1)),
                                  np.linalg.norm(a[4]["T"][:, 3] - b[4]["T"][:, 3])))
            line["plain_same_streams"] = {
                "value": pl["value"], "unit": "frames/s", "ms_per_step": 1000.0 * pl["dev_s"] / args.steps,
                "iters_per_frame": pl["iters_per_frame"], "passes_per_frame": pl["passes_per_frame"],
                "accuracy_vs_truth": pl["accuracy"], "clocks": pl["clk"]}
            line["proposal_gain"] = {
                "iters_saved_per_frame": pl["iters_per_frame"] - head["iters_per_frame"],
                "passes_saved_per_frame": pl["passes_per_frame"] - head["passes_per_frame"],
                "speedup": value / pl["value"],
                "frames_compared": len(agree),
                "final_pose_agreement_with_plain": {
                    "within_1e-5": int(sum(1 for a in agree if a[0] <= 1e-5 and a[1] <= 1e-5)),
                    "median_rot_rad": float(np.median([a[0] for a in agree])) if agree else None,
                    "median_trans_m": float(np.median([a[1] for a in agree])) if agree else None}}
        return line
    return None


def batch_cpu_baseline(wls, rec, frames_per_stream=8, proposal=None):
    """The oracle on the first frames of every stream, one host thread per
    stream over all cores, with the GPU run's initial states, references and
    (with `proposal`, the oracle network's parameters) motion inputs."""
    import concurrent.futures
    S = len(wls)
    per = {}
    for (s, k, r, init, res, mot) in rec:
        if k <= frames_per_stream and (s, k) not in per:
            per[(s, k)] = (r, init[:12].reshape(3, 4), (float(init[12]), float(init[13])), res, mot)

    def one(s):
        ks = [k for k in range(1, frames_per_stream + 1) if (s, k) in per]
        inits = {k: per[(s, k)][:3] for k in ks}
        motions = {k: per[(s, k)][4] for k in ks}
        t, out, _ = oracle_track_sequence(wls[s], len(ks), inits=inits, proposal=proposal,
                                          motions=motions)
        diffs = []
        for k in ks:
            gr = per[(s, k)][3]
            g = gr["T"]
            o = out[k]["T"]
            dR = g[:, :3].T @ o[:, :3]
            sn = 0.5 * np.linalg.norm([dR[2, 1] - dR[1, 2], dR[0, 2] - dR[2, 0], dR[1, 0] - dR[0, 1]])
            diffs.append((float(np.arctan2(sn, 0.5 * (np.trace(dR) - 1))),
                          float(np.linalg.norm(g[:, 3] - o[:, 3])),
                          {"stream": s, "frame": k, "size": [wls[s].cam.W, wls[s].cam.H],
                           "N": wls[s].N, "gpu_iters": gr["iters"][:wls[s].L],
                           "oracle_iters": out[k]["iters"], "gpu_status": gr["status"],
                           "oracle_status": out[k]["status"], "gpu_cost": gr["cost"],
                           "oracle_cost": out[k]["cost"]}))
        return len(ks), diffs

    workers = os.cpu_count() or 1
    t0 = time.perf_counter()
    with concurrent.futures.ThreadPoolExecutor(max_workers=workers) as ex:
        outs = list(ex.map(one, range(S)))
    t = time.perf_counter() - t0
    n = sum(o[0] for o in outs)
    diffs = [d for o in outs for d in o[1]]
    cpu = {"value": n / t, "unit": "frames/s", "cores": workers, "kind": "oracle",
           "sample": f"frames 1..{frames_per_stream} of each of the {S} streams (FP64 C oracle, one "
                     f"host thread per stream, same initial states and references as the GPU run)"}
    worst = sorted(diffs, key=lambda d: -d[1])[:3]
    parity = {"frames": n, "max_rot_rad": max(d[0] for d in diffs),
              "max_trans_m": max(d[1] for d in diffs),
              "within_tolerance": int(sum(1 for d in diffs if d[0] <= 1e-5 and d[1] <= 1e-5)),
              "worst": [dict(w[2], rot_rad=w[0], trans_m=w[1]) for w in worst],
              "tolerance": {"rot_rad": 1e-5, "trans_m": 1e-5}}
    return cpu, parity


# the sweep behind the Table III analogue: mean camera speeds (m/s, deg/s)
# and exposure jumps (gray levels added to, then taken off, the offset b every
# third frame)
TABLE3_MOTION = [(0.5, 30.0), (1.0, 45.0), (2.0, 90.0), (3.0, 135.0), (4.0, 180.0)]
TABLE3_JUMPS = [0.0, 40.0]


def table3(args):
    """Direct-tracking acceptance on sequences of rising difficulty, the
    quantity of the paper's Table III (Sec. IV-D): per setting, 16 streams of
    640x480 (f 525, 2000 points, 4 levels, 24 frames) tracked by the batched
    GPU tracker with the tween-frame switch of the sequence driver (a frame is
    accepted if its status is clean, at least half of its samples are valid
    and its mean Huber energy is at most 2.5; a rejected frame and every 8th
    frame go to the indirect pipeline, which here is the renderer's truth)."""
    import torch
    import paper_2607_16897_gb300 as glt
    S, F = 16, 24
    out = torch.zeros(S * glt.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    rows = []
    for speed, ang in TABLE3_MOTION:
        for jump in TABLE3_JUMPS:
            wls = [Workload(seed=7000 + s, frames=F, N=2000, W=640, H=480, f=525.0, L=4,
                            speed=speed, ang=ang, render=False, label="Table III sweep stream")
                   for s in range(S)]
            for w in wls:
                if jump:
                    w.seq.b = w.seq.b + jump * ((np.arange(F) // 3) % 2)
                w.frames = [w.seq.frame(k)[0] for k in range(F)]
            trks = [glt.Tracker(640, 480, w.cam.K, levels=4, max_points=2000) for w in wls]
            batch = glt.Batch(trks)
            frames = [torch.from_numpy(np.stack(w.frames)).cuda() for w in wls]
            bd = BatchDriver(wls)
            errs = []
            for k in range(1, F):
                for s in bd.refresh(k - 1):
                    trks[s].build_pyramid(glt.GLT_REF, frames[s][bd.r[s]])
                    trks[s].set_map_points(wls[s].ref_points(int(bd.r[s])))
                init = np.concatenate([bd.init_for().reshape(S, 12), bd.ab], 1)
                ptrs = torch.tensor([frames[s][k].data_ptr() for s in range(S)], dtype=torch.int64,
                                    device="cuda")
                batch.build_pyramid(ptrs)
                batch.track(torch.from_numpy(init).cuda(), out)
                res = glt.parse_results(out)
                before = bd.accepted.copy()
                ref_used = bd.r.copy()
                bd.record(k, np.stack([r["T"] for r in res]), np.array([r["a"] for r in res]),
                          np.array([r["b"] for r in res]), np.array([r["status"] for r in res]),
                          np.array([r["n_valid"] for r in res]), np.array([r["cost"] for r in res]))
                for s in np.nonzero(bd.accepted > before)[0]:
                    errs.append(pose_error(wls[s], k, int(ref_used[s]), res[s]["T"]))
            step = [np.linalg.norm(w.seq.T_wc[k + 1][:, 3] - w.seq.T_wc[k][:, 3]) for w in wls
                    for k in range(F - 1)]
            acc, rej = int(bd.accepted.sum()), int(bd.rejected.sum())
            rows.append({"speed_mps": speed, "ang_dps": ang, "exposure_jump": jump,
                         "mean_step_cm": 100.0 * float(np.mean(step)),
                         "frames": acc + rej, "accepted": acc, "rejected": rej,
                         "acceptance": acc / max(1, acc + rej),
                         "accepted_median_trans_mm": 1000.0 * float(np.median([e[1] for e in errs]))
                         if errs else None})
            batch.close()
            for t in trks:
                t.close()
    print(json.dumps({"metric": "direct-tracking acceptance (Table III analogue)", "unit": "fraction",
                      "data": "synthetic", "streams_per_setting": S, "frames_per_stream": F,
                      "rows": rows}), flush=True)


_GROUP = {}


def process_group(world):
    """The replicas' process group (NCCL, one rank per GPU), created once per
    run and shared by every workload the run measures; None for one GPU."""
    if world <= 1:
        return None
    import torch.distributed as dist
    if not _GROUP:
        dist.init_process_group("nccl")
        _GROUP["dist"] = dist
    return dist


# the batched forms measured with the default (single-stream) workload
BATCHED_FORMS = ("c3", "c5")


def nested_batched(args):
    """The batched workloads' records (C3: 64 mixed streams; C5: 256 streams,
    plain and with the learned proposal), measured in the same run with the
    same step counts, keyed by workload."""
    out = {}
    for kind in BATCHED_FORMS:
        sub = argparse.Namespace(**vars(args))
        sub.workload = kind
        sub.precision = None
        rec = run_batch(sub)
        if rec is not None:
            for k in ("metric", "n_gpus", "steps", "warmup", "higher_is_better", "scaling",
                      "vs_baseline", "data"):
                rec.pop(k, None)
            out[kind] = rec
    return out


def nested_solve_fp32(args):
    """The default workload with the FP32 solve (--solve fp32), measured in the
    same run with the same step counts: its frames/s, roofline and latency
    floor, and its pose difference against the oracle."""
    sub = argparse.Namespace(**vars(args))
    sub.solve = "fp32"
    sub.no_e2e = True
    sub.no_launch_overhead = True
    rec = run_ours(sub)
    if rec is None:
        return None
    keep = ("value", "unit", "ms_per_step", "dtype", "config", "roofline", "cpu_baseline",
            "parity_vs_oracle", "accuracy_vs_truth", "passes_per_frame", "clocks", "gpu_launches")
    return {k: rec[k] for k in keep if k in rec}


def main():
    args = parse()
    if args.table3:
        table3(args)
        return
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload in ("c3", "c4b", "c5"):
        line = run_batch(args)
    else:
        line = run_ours(args)
        if args.workload == "c2" and args.solve is None and not args.no_batched:
            variant = nested_solve_fp32(args)
            if line is not None and variant is not None:
                line["solve_fp32"] = variant
        if args.workload == "c2" and not args.no_batched:
            batched = nested_batched(args)
            if line is not None:
                line["batched"] = batched
    if line is not None:
        print(json.dumps(line), flush=True)
    dist = _GROUP.get("dist")
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
