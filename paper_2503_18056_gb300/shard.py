"""Spatial sharding of the TT-S_N step over several processes (or threads).

The grouped layout's spatial core X holds one row per cell, so a shard keeps
the rows of a slab of whole layers along axis 0 and the step needs two
exchanges (include/ttsn.h, tt_create_shard): a halo of the slab's first and
last layers for the upwind stencil (Sec. 4.3 with the ghost layers of
Sec. 4.5), and the sum over shards of the partial left Gram matrices of the
spatial core, G_A = sum_s X*_s^T X*_s, for the Gram-SVD rounding (App. A.2).
Everything else is row-local or replicated, so every shard takes the same
rank decisions.

This module holds the host side of that exchange: the slab partition, the
exchangers that move the data (``RingExchanger`` over torch.distributed, one
process per GPU; ``LocalRing`` for shards driven by threads of one process),
and the C callback that hands the library's device buffers to them.
"""
import ctypes
import threading

import torch

from . import _native


def shard_planes(n0, world, rank):
    """Layers [p0, p1) of axis 0 held by shard ``rank`` of ``world``: contiguous
    slabs whose sizes differ by at most one layer, lower ranks first."""
    n0, world, rank = int(n0), int(world), int(rank)
    if not (1 <= world <= n0) or not (0 <= rank < world):
        raise ValueError("need 1 <= world <= n0 layers and 0 <= rank < world")
    base, extra = divmod(n0, world)
    p0 = rank * base + min(rank, extra)
    return p0, p0 + base + (1 if rank < extra else 0)


class RingExchanger:
    """The two exchanges over a torch.distributed process group (NCCL for
    device buffers, gloo for host tensors): ``sum_`` is an all-reduce, and
    ``halo_`` fills recv_lo with the send_hi block of the rank below and
    recv_hi with the send_lo block of the rank above, on the ring of ranks
    (rank 0's lower neighbour is the last rank)."""

    def __init__(self, group=None):
        import torch.distributed as dist

        self.dist = dist
        self.group = group
        self.world = dist.get_world_size(group)
        self.rank = dist.get_rank(group)

    def _peer(self, r):
        # global rank of group rank r
        if self.group is None:
            return r
        return self.dist.get_global_rank(self.group, r)

    def sum_(self, t):
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM, group=self.group)

    def halo_(self, send_lo, send_hi, recv_lo, recv_hi):
        if self.world == 1:
            recv_lo.copy_(send_hi)
            recv_hi.copy_(send_lo)
            return
        dist = self.dist
        down = self._peer((self.rank - 1) % self.world)
        up = self._peer((self.rank + 1) % self.world)
        # the same issue order on every rank, so that messages between the
        # same pair of ranks (world 2: down == up) match in order as well as
        # by tag: tag 0 carries a send_hi upward, tag 1 a send_lo downward
        ops = [dist.P2POp(dist.isend, send_hi, up, self.group, 0),
               dist.P2POp(dist.isend, send_lo, down, self.group, 1),
               dist.P2POp(dist.irecv, recv_lo, down, self.group, 0),
               dist.P2POp(dist.irecv, recv_hi, up, self.group, 1)]
        for req in dist.batch_isend_irecv(ops):
            req.wait()


class LocalRing:
    """A ring of ``n`` shards in one process, each stepped by its own thread
    (several shards on one GPU, or one GPU per thread).  ``member(i)`` is the
    exchanger of shard i.  The exchanges meet at a barrier: no device-side
    wait is involved, each callback runs after its shard's stream has
    drained."""

    def __init__(self, n, timeout=120.0):
        self.n = int(n)
        self.barrier = threading.Barrier(self.n, timeout=timeout)
        self.slots = [None] * self.n

    def member(self, i):
        return _LocalMember(self, int(i))


class _LocalMember:
    def __init__(self, ring, i):
        self.ring, self.i = ring, i

    def _sync(self, t):
        if t.is_cuda:
            torch.cuda.current_stream(t.device).synchronize()

    def sum_(self, t):
        ring = self.ring
        ring.slots[self.i] = t
        ring.barrier.wait()
        acc = ring.slots[0].clone()
        for j in range(1, ring.n):  # the same order on every shard: the same bits
            acc += ring.slots[j]
        self._sync(acc)
        ring.barrier.wait()  # everyone has read every slot
        t.copy_(acc)
        self._sync(t)

    def halo_(self, send_lo, send_hi, recv_lo, recv_hi):
        ring = self.ring
        ring.slots[self.i] = (send_lo, send_hi)
        ring.barrier.wait()
        recv_lo.copy_(ring.slots[(self.i - 1) % ring.n][1])
        recv_hi.copy_(ring.slots[(self.i + 1) % ring.n][0])
        self._sync(recv_hi)
        ring.barrier.wait()  # nobody's send blocks change before all copied


class _DeviceArray:
    """A view of count doubles of device memory for torch.as_tensor."""

    def __init__(self, ptr, count):
        self.__cuda_array_interface__ = {"shape": (int(count),), "typestr": "<f8",
                                         "data": (int(ptr), False), "version": 3, "strides": None}


def device_view(ptr, count):
    """A float64 CUDA tensor aliasing count doubles at device address ptr."""
    return torch.as_tensor(_DeviceArray(ptr, count), device="cuda")


def exchange_callback(exchanger):
    """The tt_exchange_fn handed to tt_create_shard: views the library's
    device buffer as tensors and calls exchanger.sum_ or exchanger.halo_.
    Returns the ctypes function object (keep it alive with the handle)."""

    def cb(ctx, kind, buf, count, stream):
        try:
            if kind == _native.TT_XCHG_SUM:
                exchanger.sum_(device_view(buf, count))
            elif kind == _native.TT_XCHG_HALO:
                v = device_view(buf, 4 * count)
                exchanger.halo_(v[:count], v[count:2 * count], v[2 * count:3 * count], v[3 * count:])
            else:
                return 2
            torch.cuda.current_stream().synchronize()
            return 0
        except Exception:  # reported to the library as a failed exchange
            import traceback

            traceback.print_exc()
            return 1

    return _native.EXCHANGE_FN(cb)
