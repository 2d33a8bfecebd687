"""Handles created with a caller-supplied device allocator (tt_create_ex):
results identical to the default pool, the memory visibly drawn from and
returned to torch's caching allocator; borrowed core views (tt_get_cores);
refused allocations reported as TT_ERR_OOM."""
import gc

import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ttsn():
    assert torch.cuda.is_available()
    import paper_2503_18056_gb300 as m

    return m


def _problem():
    return workloads.problem("small_2d", n=(24, 20), n_theta=8, n_phi=16, eps=1e-6)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_torch_allocator_gives_identical_results(ttsn, precision):
    p = _problem()
    prec = ttsn.TT_FP64 if precision == "fp64" else ttsn.TT_MIXED
    a = ttsn.TTSN.from_problem(p, precision=prec)
    b = ttsn.TTSN.from_problem(p, precision=prec, allocator="torch")
    for _ in range(5):
        ia = a.step()
        ib = b.step()
        assert ia["ranks"] == ib["ranks"]
    assert torch.equal(a.full(), b.full())
    assert torch.equal(a.energy()[1], b.energy()[1])


def test_torch_allocator_memory_is_torch_memory(ttsn):
    gc.collect()
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    g = ttsn.TTSN.from_problem(_problem(), allocator="torch")
    g.step(3)
    torch.cuda.synchronize()
    held = torch.cuda.memory_allocated() - base
    # at least the cores, the grown cores and the Gram workspaces
    r = g.ranks()
    assert held >= 8 * 24 * 20 * r[1]
    del g
    gc.collect()
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == base


def test_borrowed_core_views_match_ranks(ttsn):
    g = ttsn.TTSN.from_problem(_problem())
    g.step(2)
    r = g.ranks()
    views = g.core_views()
    assert [shape for _, shape in views] == [(r[0], 480, r[1]), (r[1], 8, r[2]), (r[2], 16, r[3])]
    assert all(ptr for ptr, _ in views)
    # the views are the same memory the owned copies come from
    cores = g.cores()
    assert [tuple(c.shape) for c in cores] == [shape for _, shape in views]


class _Budget:
    """Torch's caching allocator behind a byte budget: requests beyond it are
    refused (alloc returns 0), as a full device would refuse them."""

    def __init__(self, limit):
        self.limit, self.held, self.peak, self.unknown = limit, {}, 0, 0

    def alloc(self, nbytes, stream):
        if sum(self.held.values()) + nbytes > self.limit:
            return 0
        ptr = torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
        self.held[ptr] = nbytes
        self.peak = max(self.peak, sum(self.held.values()))
        return ptr

    def free(self, ptr, nbytes, stream):
        torch.cuda.caching_allocator_delete(ptr)
        self.unknown += self.held.pop(ptr, None) is None


def test_refused_allocation_is_out_of_memory_and_leaks_nothing(ttsn):
    """Failure detection without a device fault: an allocator that refuses a
    request makes the call that needed it return TT_ERR_OOM with a message;
    the handle's memory is all returned when it is destroyed, and a handle
    given just the memory the run needed computes the same result."""
    p = _problem()
    ample = _Budget(1 << 40)
    ref = ttsn.TTSN.from_problem(p, allocator=ample)
    for _ in range(4):
        ref.step()
    peak = ample.peak
    for frac in (0.05, 0.25):
        tight = _Budget(int(frac * peak))
        with pytest.raises(ttsn.TTError) as e:
            g = ttsn.TTSN.from_problem(p, allocator=tight)
            for _ in range(4):
                g.step()
        assert e.value.status == -2 and "allocation" in str(e.value)
        g = e = None  # the traceback holds the failed step's frame, and so the handle
        gc.collect()
        torch.cuda.synchronize()
        assert not tight.held and tight.unknown == 0
    again = ttsn.TTSN.from_problem(p, allocator=_Budget(peak))
    for _ in range(4):
        again.step()
    assert torch.equal(again.full(), ref.full())
