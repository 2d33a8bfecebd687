"""The N > 1 path of bench.py on CPU: world_size-2 gloo process group, each
rank a replica with its own timing; the line reports the slowest rank's time
and the steps of all ranks over it (the replicas exchange nothing else)."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, out):
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        total_ms, value = bench.aggregate_over_ranks(times[rank], 12, world, device="cpu")
        out.put((rank, total_ms, value))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("times", [(1500.0, 1800.0), (2000.0, 900.0)])
def test_two_replicas_report_the_slowest_rank(times):
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, times, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    slowest = max(times)
    for rank, total_ms, value in res:
        assert total_ms == slowest
        assert abs(value - world * 12 / (slowest * 1e-3)) <= 1e-12 * value


def test_single_rank_needs_no_process_group():
    import bench

    total_ms, value = bench.aggregate_over_ranks(2400.0, 12, 1)
    assert total_ms == 2400.0 and value == 5.0
