"""Rendering jobs for worker processes: seeded sequences of the large box room
rendered frame by frame, with map points at reference frames.  Input
generation only (no tracker arithmetic); both the tests' oracle runs and the
CUDA path's drivers draw their frames from here."""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np


def stream_motion(seed: int):
    """Per-sequence mean speed and angular speed, up to 2 m/s and 90 deg/s."""
    rng = np.random.default_rng(seed + 4242)
    return float(rng.uniform(0.5, 2.0)), float(rng.uniform(30.0, 90.0))


_SEQ_CACHE = {}


def _sequence(seed, frames, W, H, f, speed=None, ang=None):
    import synth
    key = (seed, frames, W, H, f, speed, ang)
    if key not in _SEQ_CACHE:
        if speed is None:
            speed, ang = stream_motion(seed)
        cam = synth.camera_for(W, H, f)
        _SEQ_CACHE[key] = synth.sequence(seed, frames, cam, synth.ROOM_LARGE, speed, ang)
    return _SEQ_CACHE[key]


def _render_job(job):
    """(seed, frames, W, H, f, k, N[, speed, ang]) -> (frame k, map points if
    N > 0); speed and ang default to ``stream_motion(seed)``."""
    import synth
    seed, frames, W, H, f, k, N = job[:7]
    speed, ang = (job[7], job[8]) if len(job) > 7 else (None, None)
    seq = _sequence(seed, frames, W, H, f, speed, ang)
    if N > 0:
        img, uvd = synth.reference_points(seq, k, N, 0.5, 8.0)
        return img, uvd
    return seq.frame(k)[0], None


def render_pool(workers: int | None = None):
    """Spawned worker pool for the CPU renderer (safe next to a CUDA context)."""
    return mp.get_context("spawn").Pool(processes=workers or os.cpu_count() or 1)
