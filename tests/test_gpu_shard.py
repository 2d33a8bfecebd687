"""Spatial shards on the GPU (tt_create_shard): slabs of layers along axis 0,
each a library handle stepped by its own thread, exchanging the halo layers
and the partial left Grams through an in-process ring (no device-side wait).
The sharded run must take the unsharded run's rank decisions and reproduce
its tensor, temperature and energy totals."""
import threading

import numpy as np
import pytest
import torch

import workloads
from oracle.ttstep import OUTFLOW, PERIODIC, VACUUM

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ttsn():
    assert torch.cuda.is_available()
    import paper_2503_18056_gb300 as m

    return m


def _problem(n, bc, eps=1e-5, seed=5):
    f = workloads.random_fields(n, seed)
    return dict(n=n, L=[1.0] * len(n), n_theta=4, n_phi=8, c=1.0, a_r=1.0,
                dt=0.4 * min(1.0 / m for m in n), bc=[bc] * len(n), sigma_a=f["sigma_a"].reshape(-1),
                cv=f["cv"].reshape(-1), T0=f["T0"].reshape(-1), Tr0=f["T0"].reshape(-1), eps=eps)


def _run_shards(ttsn, kw, world, steps, forced=None):
    from paper_2503_18056_gb300.shard import LocalRing, shard_planes

    ring = LocalRing(world, timeout=60.0)
    shards = [ttsn.TTSN(shard=shard_planes(kw["n"][0], world, r) + (ring.member(r),), **kw)
              for r in range(world)]
    infos = [[None] * steps for _ in range(world)]
    errors = []

    def run(r):
        try:
            for m in range(steps):
                infos[r][m] = shards[r].step(forced=None if forced is None else forced[m])
        except Exception as e:  # reported after the join
            errors.append((r, e))

    threads = [threading.Thread(target=run, args=(r,)) for r in range(world)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    return shards, infos


@pytest.mark.parametrize("n,bc,world", [((12, 9), PERIODIC, 2), ((12, 9), VACUUM, 3), ((12, 9), OUTFLOW, 4),
                                        ((7, 5, 4), VACUUM, 3), ((6, 5, 4), PERIODIC, 1), ((9,), PERIODIC, 3)])
def test_shards_reproduce_the_unsharded_step(ttsn, n, bc, world):
    kw = _problem(n, bc)
    steps = 4
    ref = ttsn.TTSN(**kw)
    ref_infos = [ref.step() for _ in range(steps)]
    shards, infos = _run_shards(ttsn, kw, world, steps)
    for r in range(world):  # the same free rank decisions on every shard
        assert [i["ranks"] for i in infos[r]] == [i["ranks"] for i in ref_infos]
    F = torch.cat([s.full() for s in shards], dim=0).cpu().numpy()
    R = ref.full().cpu().numpy()
    assert np.linalg.norm(F - R) <= 1e-12 * np.linalg.norm(R)
    T = torch.cat([s.energy(totals=False)[1] for s in shards]).cpu().numpy()
    _, Tr, tot_ref = ref.energy()
    assert np.abs(T - Tr.cpu().numpy()).max() <= 1e-13
    # totals are the whole grid's on every shard (summed through the exchange)
    tots = []
    done = []

    def totals(r):
        tots.append((r, shards[r].energy()[2]))
        done.append(r)

    threads = [threading.Thread(target=totals, args=(r,)) for r in range(world)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    for _, tot in tots:
        assert abs(sum(tot) - sum(tot_ref)) <= 1e-13 * abs(sum(tot_ref))


def test_shards_with_rusanov_and_the_precision_form(ttsn):
    kw = _problem((10, 8), VACUUM)
    kw.update(flux="rusanov", rusanov_s=0.5, precision=ttsn.TT_MIXED)
    ref = ttsn.TTSN(**kw)
    ranks = [ref.step()["ranks"][1:-1] for _ in range(3)]
    shards, infos = _run_shards(ttsn, kw, 2, 3, forced=ranks)
    F = torch.cat([s.full() for s in shards], dim=0).cpu().numpy()
    R = ref.full().cpu().numpy()
    # the shards sum two partial Grams where the unsharded run sums row
    # blocks in one split: the same products, added in another order
    assert np.linalg.norm(F - R) <= 1e-10 * np.linalg.norm(R)


def test_shard_arguments_and_unsupported_forms_are_refused(ttsn):
    from paper_2503_18056_gb300.shard import LocalRing

    kw = _problem((8, 6), VACUUM)
    ring = LocalRing(1)
    with pytest.raises(ttsn.TTError):
        ttsn.TTSN(shard=(3, 3, ring.member(0)), **kw)   # empty slab
    with pytest.raises(ttsn.TTError):
        ttsn.TTSN(shard=(0, 9, ring.member(0)), **kw)   # beyond n[0]
    with pytest.raises(ttsn.TTError):
        ttsn.TTSN(shard=(0, 8, ring.member(0)), flux="hll", **kw)
    with pytest.raises(ttsn.TTError):
        ttsn.TTSN(shard=(0, 8, ring.member(0)), layout=ttsn.TT_LAYOUT_SPLIT,
                  **dict(kw, sigma_a=np.ones(48)))
    s = ttsn.TTSN(shard=(0, 8, ring.member(0)), **kw)
    with pytest.raises(ttsn.TTError):
        s.tape_begin(1)
    with pytest.raises(ttsn.TTError):
        s.set_sources([(np.ones(48), np.ones(4), np.ones(8))])


def test_a_failed_exchange_is_reported_and_no_shard_hangs(ttsn):
    """A shard whose exchange fails on the host (here: it raises instead of
    meeting its neighbour) makes its own step return TT_ERR_STATE, and the
    shard waiting for it gives up after the ring's timeout with the same
    status: the failure surfaces on the host between kernels, no kernel waits."""
    from paper_2503_18056_gb300.shard import LocalRing, shard_planes

    kw = _problem((8, 6), PERIODIC)
    ring = LocalRing(2, timeout=2.0)

    class Broken:
        def sum_(self, t):
            raise RuntimeError("planted exchange failure")

        def halo_(self, *blocks):
            raise RuntimeError("planted exchange failure")

    shards = [ttsn.TTSN(shard=shard_planes(8, 2, 0) + (ring.member(0),), **kw),
              ttsn.TTSN(shard=shard_planes(8, 2, 1) + (Broken(),), **kw)]
    status = [None, None]

    def run(r):
        try:
            shards[r].step()
            status[r] = 0
        except ttsn.TTError as e:
            status[r] = e.status

    threads = [threading.Thread(target=run, args=(r,)) for r in range(2)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=30.0)
    assert not any(t.is_alive() for t in threads)
    assert status == [-6, -6]
    torch.cuda.synchronize()  # the context stays usable
    G = ttsn.gram(torch.ones((10, 3), dtype=torch.float64, device="cuda"))
    assert float(G[0, 0]) == 10.0
