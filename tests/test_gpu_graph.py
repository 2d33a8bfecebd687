"""Captured steps (tt_set_graph): one step recorded as a CUDA graph whose
kernels read the device-decided sizes, replayed for every later step.  The
replays must give the same bits as host-driven steps, follow the ranks as they
grow and shrink, leave the handle usable for every other call, and the batch
form must replay every problem's graph with the same results."""
import numpy as np
import pytest
import torch

import workloads
from oracle.ttstep import PERIODIC, VACUUM

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ttsn():
    assert torch.cuda.is_available()
    import paper_2503_18056_gb300 as m

    return m


def _pair(ttsn, p, **over):
    a = ttsn.TTSN.from_problem(p, **over)
    b = ttsn.TTSN.from_problem(p, **over)
    b.set_graph(True)
    return a, b


@pytest.mark.parametrize("n,bc,flux,cap", [((16, 12), PERIODIC, "upwind", 24), ((14, 10), VACUUM, "rusanov", 12),
                                           ((6, 5, 4), VACUUM, "upwind", 16), ((13,), PERIODIC, "upwind", 8)])
def test_replayed_steps_equal_host_steps_bit_for_bit(ttsn, n, bc, flux, cap):
    p = workloads.problem("small_2d", n=n, n_theta=4, n_phi=8, eps=1e-6, bc=bc)
    p["max_rank"] = cap
    a, b = _pair(ttsn, p, flux=flux)
    for _ in range(6):
        ia, ib = a.step(), b.step()
        assert ia["ranks"] == ib["ranks"] and ia["grown"] == ib["grown"]
        assert ia["capped"] == ib["capped"] and ia["norm"] == ib["norm"]
        assert ia["discarded"] == ib["discarded"]
    assert torch.equal(a.full(), b.full())
    Ea, Ta, ta = a.energy()
    Eb, Tb, tb = b.energy()
    assert torch.equal(Ta, Tb) and torch.equal(Ea, Eb) and ta == tb


def test_several_replays_per_call_and_host_calls_in_between(ttsn):
    p = workloads.problem("small_2d", n=(16, 16), n_theta=4, n_phi=8, eps=1e-5)
    p["max_rank"] = 20
    a, b = _pair(ttsn, p)
    a.step(4)
    b.step(4)                       # four replays, one synchronisation
    assert a.ranks() == b.ranks()
    assert torch.equal(a.full(), b.full())
    # the host replaces the state in between: replays restart from its ranks
    st = a.state_dict()
    b.load_state_dict(st)
    a.step(2)
    b.step(2)
    assert torch.equal(a.full(), b.full())
    # a host-driven step in between (forced ranks are not captured)
    r = a.step(forced=[5, 4])["ranks"]
    assert b.step(forced=[5, 4])["ranks"] == r
    a.step(3)
    b.step(3)
    assert torch.equal(a.full(), b.full())


def test_replay_launch_count_and_refusals(ttsn):
    p = workloads.problem("small_2d", n=(12, 12), n_theta=4, n_phi=8, eps=1e-6)
    p["max_rank"] = 16
    g = ttsn.TTSN.from_problem(p)
    g.set_graph(True)
    g.step()                        # records and replays
    k0 = ttsn.kernel_launches()
    g.step(3)
    per = (ttsn.kernel_launches() - k0) / 3
    assert per > 20                 # the recorded step's library kernels, counted per replay
    # handles that cannot be captured
    for kw in (dict(max_rank=0), dict(precision=ttsn.TT_MIXED), dict(rounds_per_step=2), dict(flux="hll")):
        q = dict(p)
        h = ttsn.TTSN.from_problem(q, **kw)
        with pytest.raises(ttsn.TTError):
            h.set_graph(True)
    s = ttsn.TTSN.from_problem(p, layout=ttsn.TT_LAYOUT_SPLIT)
    with pytest.raises(ttsn.TTError):
        s.set_graph(True)
    # a setting that breaks the conditions later is refused at the next step
    g.set_precision(ttsn.TT_MIXED)
    with pytest.raises(ttsn.TTError):
        g.step()
    g.set_precision(ttsn.TT_FP64)
    g.step()


def test_batch_replays_equal_host_driven_batch(ttsn):
    probs = workloads.batch_problems(count=6, seed=3)
    a = ttsn.TTSNBatch(probs)
    b = ttsn.TTSNBatch(probs)
    b.set_graph(True)
    ia = a.step(3)
    ib = b.step(3)
    for x, y in zip(ia, ib):
        assert x["ranks"] == y["ranks"]
    for i in range(len(probs)):
        assert torch.equal(a.problem(i).full(), b.problem(i).full())
