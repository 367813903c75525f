"""Tween-frame switch between the direct tracker and an indirect pipeline
(GLidE-SLAM Sec. III and Sec. IV-D "Indirect Tracking Switch").

Host-side policy only; the tracking itself is the library's.  The paper tracks
the frames between indirect keyframes ("tween frames") with the direct
tracker and hands control back to the indirect pipeline when

* the direct tracker fails (here: a failure status bit, or fewer than
  ``min_valid_frac`` of the 8N (or K N) residual samples usable),
* its robust photometric error exceeds the failure threshold (here: the mean
  Huber energy ``cost`` above ``max_cost``), or
* the maximum number of direct frames since the last reference is reached.

A frame the direct tracker rejects is re-tracked by the indirect pipeline,
which also provides the next reference (pose, image and map points); after a
successful switch back the direct pipeline is refreshed with that reference.
``acceptance_rate`` is the share of frames the direct tracker kept (the
quantity of the paper's Table III).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field


@dataclass
class TweenSwitch:
    max_direct: int = 8            # direct frames per reference before switching back
    max_cost: float = 2.5          # failure threshold on the mean Huber energy
    min_valid_frac: float = 0.5    # minimum share of usable residual samples
    samples_per_point: int = 8     # K of the pattern
    since_reference: int = 0
    direct_accepted: int = 0
    direct_rejected: int = 0
    indirect_frames: int = 0
    history: list = field(default_factory=list)

    def direct_ok(self, result: dict, n_points: int) -> bool:
        """The acceptance test on one direct-tracking result (a dict with
        ``status``, ``n_valid`` and ``cost`` as returned by the tracker)."""
        if result["status"] != 0:
            return False
        if result["n_valid"] < self.min_valid_frac * self.samples_per_point * n_points:
            return False
        cost = result["cost"]
        return cost == cost and not math.isinf(cost) and cost <= self.max_cost

    def after_direct(self, result: dict, n_points: int) -> bool:
        """Records a direct-tracked frame; returns True if the next frame must
        go to the indirect pipeline (this frame was rejected, or the direct
        budget of the current reference is used up)."""
        ok = self.direct_ok(result, n_points)
        self.since_reference += 1
        if ok:
            self.direct_accepted += 1
        else:
            self.direct_rejected += 1
        self.history.append("direct" if ok else "rejected")
        return (not ok) or self.since_reference >= self.max_direct

    def after_indirect(self) -> None:
        """The indirect pipeline tracked a frame and provided a new reference."""
        self.indirect_frames += 1
        self.since_reference = 0
        self.history.append("indirect")

    @property
    def frames(self) -> int:
        return self.direct_accepted + self.direct_rejected + self.indirect_frames

    @property
    def acceptance_rate(self) -> float:
        """Share of all frames whose pose came from the direct tracker."""
        return self.direct_accepted / self.frames if self.frames else 0.0
