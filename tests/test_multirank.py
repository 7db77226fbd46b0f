"""The N > 1 host path of bench.py with world_size-2 gloo process groups on the CPU: each rank gets
its own realization (no data-path collective), the timing is the maximum over ranks, and the
aggregate throughput counts every rank's units."""
from __future__ import annotations

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sh = bench.shard_for_rank(rank)
        local_ms = 100.0 + 50.0 * rank  # the slower rank defines the job time
        mx = bench.max_over_ranks(local_ms, dist, "cpu")
        rate = bench.aggregate_rate(1_000_000, world, mx)
        gathered = [None] * world
        dist.all_gather_object(gathered, sh)
        if rank == 0:
            out.put((mx, rate, gathered))
    finally:
        dist.destroy_process_group()


def test_two_rank_weak_scaling_host_logic():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    mx, rate, shards = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert mx == 150.0
    assert rate == pytest.approx(2 * 1_000_000 / (150.0 * 1e6))
    assert [s["realization"] for s in shards] == [0, 1]
    assert len({s["field_seed"] for s in shards}) == 2
