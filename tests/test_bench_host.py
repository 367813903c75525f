"""Host-side helpers of bench.py (no GPU): step-time percentiles, the
aggregate rate and the single-process max over ranks."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    sys.path.insert(0, ROOT)
    import bench as b
    return b


def test_step_percentiles(bench):
    p = bench.step_percentiles([5.0, 1.0, 3.0, 2.0, 4.0])
    assert p == {"p50": 3.0, "p90": pytest.approx(4.6), "min": 1.0, "max": 5.0}


def test_rates_and_single_rank_max(bench):
    assert bench.aggregate_rate(100, 4, 2.0) == pytest.approx(200.0)
    assert bench.max_over_ranks([1.5, 2.5]) == [1.5, 2.5]
    # distinct sequences per replica, stable per stream
    assert bench.stream_seed("c3", 3, 0) != bench.stream_seed("c3", 3, 1)
    assert bench.stream_seed("c3", 3, 0) == bench.stream_seed("c3", 3, 0)
