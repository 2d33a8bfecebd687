"""Handles created with a caller-supplied device allocator (tt_create_ex):
results identical to the default pool, the memory visibly drawn from and
returned to torch's caching allocator; borrowed core views (tt_get_cores)."""
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
