"""The host side of spatial sharding on CPU ranks (gloo, world sizes 2 and
4): the slab partition, the ring halo exchange and the all-reduce that the
library's shards call (paper_2503_18056_gb300.shard.RingExchanger).  The
sharded step itself is checked on CPU ranks against the single-rank oracle
step in test_oracle_shard.py."""
import os

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def test_shard_planes_partition_axis_zero():
    from paper_2503_18056_gb300.shard import shard_planes

    for n0 in (1, 5, 12, 128):
        for world in range(1, min(n0, 9) + 1):
            parts = [shard_planes(n0, world, r) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == n0
            assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))
            sizes = [p1 - p0 for p0, p1 in parts]
            assert min(sizes) >= 1 and max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard_planes(3, 4, 0)


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2503_18056_gb300.shard import RingExchanger

        ex = RingExchanger()
        count = 5
        send_lo = torch.full((count,), 100.0 * rank + 1.0, dtype=torch.float64)
        send_hi = torch.full((count,), 100.0 * rank + 2.0, dtype=torch.float64)
        recv_lo = torch.zeros(count, dtype=torch.float64)
        recv_hi = torch.zeros(count, dtype=torch.float64)
        ex.halo_(send_lo, send_hi, recv_lo, recv_hi)
        g = torch.arange(6, dtype=torch.float64) * (rank + 1) + 0.25
        ex.sum_(g)
        out[rank] = (recv_lo.tolist(), recv_hi.tolist(), g.tolist())
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_ring_halo_and_sum_on_gloo_ranks(world):
    port = 29500 + 17 * world + os.getpid() % 1000
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        lo, hi, g = out[r]
        below, above = (r - 1) % world, (r + 1) % world
        assert lo == [100.0 * below + 2.0] * 5   # the lower shard's top layer
        assert hi == [100.0 * above + 1.0] * 5   # the upper shard's bottom layer
        want = np.arange(6) * sum(range(1, world + 1)) + 0.25 * world
        assert np.array_equal(np.array(g), want)
        assert g == out[0][2]                     # the same bits on every rank
