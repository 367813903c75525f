"""The N > 1 path of the benchmark (replicas: each rank tracks its own
streams, no collective on the data path) with world_size 2 over gloo on the
CPU: the slowest rank's time is what the job reports, the rate aggregates over
ranks, every rank gets its own sequences, and the reference arm runs on rank 0
only."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import contextlib
    import io
    import types

    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank 1 is the slow one on the first entry, rank 0 on the second
    times = [1.0 + rank, 5.0 - rank]
    got = bench.max_over_ranks(times, dist, "cpu")
    rate = bench.aggregate_rate(100, world, got[0])
    # single-stream workloads use stream 0 only; batches 3 streams here
    seeds = {k: [bench.stream_seed(k, s, rank) for s in range(1 if k in ("c2", "c4") else 3)]
             for k in ("c2", "c3", "c4", "c4b", "c5")}
    # the reference arm prints nothing on ranks other than 0
    buf = io.StringIO()
    args = types.SimpleNamespace(warmup=1, steps=1, workload="c2", gpus=world, jacobian=None)
    if rank != 0:
        with contextlib.redirect_stdout(buf):
            bench.run_reference(args)
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, got, rate, seeds, buf.getvalue()))


def test_two_ranks_over_gloo():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict((r, (g, rate, seeds, out)) for r, g, rate, seeds, out in (q.get(timeout=120) for _ in procs))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        got, rate, seeds, out = res[r]
        assert got == [2.0, 5.0]                # the maximum over the two ranks
        assert rate == pytest.approx(2 * 100 / 2.0)
    assert res[1][3] == ""                      # no reference line from rank 1
    for k in res[0][2]:
        a, b = set(res[0][2][k]), set(res[1][2][k])
        assert not (a & b), k                   # replicas never share a sequence
    assert res[0][2]["c2"][0] == 1 and res[0][2]["c3"][:2] == [1000, 1001]
