"""Randomized rounding on the GPU (App. A.3; tt_set_sketch, tt_set_rounding)
against the oracle's randomized rounding with the same Gaussian sketch:
single roundings of bare TTs and rounded steps."""
import ctypes

import numpy as np
import pytest
import torch

import workloads
from oracle import tt
from oracle.rounding import round_randomized, round_ttsvd
from oracle.ttstep import TTSN as OracleTTSN

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ttsn():
    assert torch.cuda.is_available()
    import paper_2503_18056_gb300 as m

    return m


def _omega(modes, ranks, seed):
    rng = np.random.default_rng(seed)
    r = [1] + list(ranks) + [1]
    return [rng.standard_normal((r[k], m, r[k + 1])) for k, m in enumerate(modes)]


def _sub(omega, ranks):
    r = [1] + list(ranks) + [1]
    return [w[: r[k], :, : r[k + 1]] for k, w in enumerate(omega)]


def test_randomized_rounding_recovers_exact_low_rank(ttsn):
    modes, ranks = [40, 30, 20, 10], [3, 5, 4]
    A = workloads.random_tt(modes, ranks, seed=61)
    X = tt.add(tt.add(A, A), tt.scale(A, -1.0))
    h = ttsn.TensorTrain(X)
    h.set_sketch(_omega(modes, [6, 8, 6], 62))
    h.set_rounding("randomized")
    info = h.round(forced=ranks)
    assert info["ranks"][1:-1] == ranks
    F = tt.full(A)
    assert np.abs(h.full().cpu().numpy() - F).max() <= 1e-11 * np.abs(F).max()


@pytest.mark.parametrize("modes,ranks,target", [([300, 40, 30], [20, 15], [10, 8]),
                                                ([5000, 16, 32], [60, 12], [25, 12]),
                                                ([64, 32, 16, 8], [12, 20, 6], [8, 10, 6])])
def test_randomized_rounding_matches_oracle_with_the_same_sketch(ttsn, modes, ranks, target):
    rng = np.random.default_rng(sum(modes))
    r = [1] + ranks + [1]
    decay = [np.geomspace(1.0, 1e-4, r[k + 1]) for k in range(len(modes))]
    X = [rng.standard_normal((r[k], m, r[k + 1])) * decay[k][None, None, :] for k, m in enumerate(modes)]
    om = _omega(modes, [t + 4 for t in target], 63)
    ref = round_randomized(X, _sub(om, target))
    h = ttsn.TensorTrain(X)
    h.set_sketch(om)
    h.set_rounding("randomized")
    info = h.round(forced=target)
    assert info["ranks"][1:-1] == tt.ranks(ref)
    R = tt.full(ref)
    assert np.linalg.norm(h.full().cpu().numpy() - R) <= 1e-10 * np.linalg.norm(R)
    # and it is a near-optimal truncation
    T, _ = round_ttsvd(X, forced=target)
    F = tt.full(X)
    assert np.linalg.norm(R - F) <= 20 * np.linalg.norm(tt.full(T) - F) + 1e-13 * np.linalg.norm(F)


def test_rounded_steps_with_randomized_rounding_match_oracle(ttsn):
    p = workloads.problem("small_2d", n=(16, 12), n_theta=4, n_phi=8, eps=1e-5, bc=1)
    I0 = p["c"] * p["a_r"] * p["Tr0"] ** 4 / (4 * np.pi)
    om = _omega([16 * 12, 4, 8], [40, 8], 64)
    ref = OracleTTSN(p["n"], p["L"], p["n_theta"], p["n_phi"], p["c"], p["a_r"], p["dt"], p["bc"],
                     p["sigma_a"], p["cv"], p["T0"],
                     OracleTTSN.isotropic_cores(I0.reshape(-1), p["n_theta"], p["n_phi"]),
                     rounding="randomized", sketch=om)
    gram = ttsn.TTSN.from_problem(p)
    g = ttsn.TTSN.from_problem(p)
    g.set_sketch(om)
    g.set_rounding("randomized")
    for _ in range(5):
        ranks = gram.step()["ranks"][1:-1]  # the Gram-SVD run's ranks at eps
        forced = [min(r, m) for r, m in zip(ranks, (40, 8))]
        ref.step(forced=forced)
        info = g.step(forced=forced)
        assert info["ranks"][1:-1] == tt.ranks(ref.cores)
    R = ref.full()
    assert np.linalg.norm(g.full().cpu().numpy() - R) <= 1e-9 * np.linalg.norm(R)
    _, T, _ = g.energy()
    assert np.abs(T.cpu().numpy() - ref.T).max() <= 1e-9 * np.abs(ref.T).max()


def test_randomized_rounding_state_errors(ttsn):
    X = workloads.random_tt([6, 5, 4], [2, 2], seed=65)
    h = ttsn.TensorTrain(X)
    with pytest.raises(ttsn.TTError) as e:
        h.set_rounding("randomized")  # no sketch yet
    assert e.value.status == -6
    p = workloads.problem("small_2d", n=(6, 5), n_theta=4, n_phi=8, bc=1)
    g = ttsn.TTSN.from_problem(p)
    g.set_sketch(_omega([30, 4, 8], [6, 4], 66))
    g.set_rounding("randomized")
    assert ttsn.lib.tt_tape_begin(g._h, ctypes.c_int(1)) == -6
    g.step(forced=[4, 3])
    g.set_rounding("gram")
    g.step()
