"""Batched form: independent problems of uneven sizes stepped concurrently give
exactly the results of stepping each problem alone (which the single-problem
tests compare with the oracle), and each conserves energy (periodic)."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ttsn():
    import torch

    assert torch.cuda.is_available()
    import paper_2503_18056_gb300 as m

    return m


def _problems():
    ps = []
    for (n, nt, npf, eps, cap) in [((12, 12), 4, 8, 1e-4, 16), ((16, 20), 8, 16, 1e-6, 40),
                                         ((24, 24), 4, 8, 1e-5, 8), ((9, 31), 8, 16, 1e-4, 96),
                                         ((20, 16), 4, 8, 1e-6, 24)]:
        p = workloads.problem("small_2d", n=n, n_theta=nt, n_phi=npf, eps=eps, max_rank=cap)
        ps.append(p)
    return ps


def test_batch_equals_individual_runs_bitwise(ttsn):
    ps = _problems()
    batch = ttsn.TTSNBatch(ps, threads=3)
    infos = batch.step(3)
    for i, p in enumerate(ps):
        alone = ttsn.TTSN.from_problem(p)
        info = alone.step(3)
        assert info["ranks"] == infos[i]["ranks"]
        Fa = alone.full().cpu().numpy()
        Fb = batch.problem(i).full().cpu().numpy()
        assert np.array_equal(Fa, Fb)
        _, Ta, _ = alone.energy()
        _, Tb, _ = batch.problem(i).energy()
        assert np.array_equal(Ta.cpu().numpy(), Tb.cpu().numpy())


def test_batch_conserves_energy_per_problem(ttsn):
    ps = _problems()
    batch = ttsn.TTSNBatch(ps)
    t0 = [sum(batch.problem(i).energy()[2]) for i in range(len(ps))]
    batch.step(4)
    for i in range(len(ps)):
        t1 = sum(batch.problem(i).energy()[2])
        assert abs(t1 - t0[i]) <= 1e-12 * t0[i]


def test_batch_of_the_64_problem_workload_builds_and_steps(ttsn):
    ps = workloads.batch_problems(64)[:8]  # the first 8 of the 64-problem workload
    batch = ttsn.TTSNBatch(ps)
    infos = batch.step(2)
    for i, (p, info) in enumerate(zip(ps, infos)):
        assert max(info["ranks"]) <= p["max_rank"]
        E, T, _ = batch.problem(i).energy()
        assert np.isfinite(E.cpu().numpy()).all() and np.isfinite(T.cpu().numpy()).all()
