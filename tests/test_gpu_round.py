"""GPU Gram-SVD rounding (tt_round) against the oracle (App. A)."""
import numpy as np
import pytest

import workloads
from oracle import tt
from oracle.rounding import round_gram, round_ttsvd

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ttsn():
    import torch

    assert torch.cuda.is_available()
    import paper_2503_18056_gb300 as m

    return m


def _decaying(modes, nterms, ratio, seed):
    rng = np.random.default_rng(seed)
    terms = []
    for j in range(nterms):
        vs = [rng.standard_normal(m) for m in modes]
        vs[0] = vs[0] * ratio ** (-j)
        terms.append(tt.rank_one(vs))
    return tt.add_many(terms)


def _rel(F, R):
    return np.linalg.norm(F - R) / np.linalg.norm(R)


@pytest.mark.parametrize("modes", [[40, 6, 9], [30, 5, 4, 7], [200, 8, 16]])
def test_forced_rank_rounding_matches_oracle(ttsn, modes):
    X = _decaying(modes, 12, 2.5, seed=len(modes))
    forced = [5] * (len(modes) - 1)
    ref, _ = round_gram(X, forced=forced)
    g = ttsn.TensorTrain(X)
    info = g.round(forced=forced)
    assert info["ranks"][1:-1] == forced
    F = g.full().cpu().numpy()
    assert _rel(F, tt.full(ref)) < 1e-10
    # left cores orthonormal (App. A.4: A' has orthonormal columns)
    for G in g.cores()[:-1]:
        G = G.cpu().numpy()
        A = G.reshape(-1, G.shape[2])
        assert np.abs(A.T @ A - np.eye(A.shape[1])).max() < 1e-9


@pytest.mark.parametrize("eps", [1e-2, 1e-4, 1e-6])
def test_eps_rounding_ranks_and_error_bound(ttsn, eps):
    X = _decaying([60, 7, 11], 14, 3.0, seed=5)
    ref, sig = round_ttsvd(X, eps=eps)
    g = ttsn.TensorTrain(X)
    info = g.round(eps=eps)
    F = g.full().cpu().numpy()
    FX = tt.full(X)
    assert np.linalg.norm(F - FX) <= eps * np.linalg.norm(FX) * (1 + 1e-6)
    # chosen ranks are valid for the tolerance rule: within one of the oracle's
    assert all(abs(a - b) <= 1 for a, b in zip(info["ranks"][1:-1], tt.ranks(ref)))
    assert abs(info["norm"] - np.linalg.norm(FX)) <= 1e-10 * np.linalg.norm(FX)


def test_exact_recovery_of_redundant_tt(ttsn):
    X = workloads.random_tt([25, 6, 7, 5], [4, 3, 2], seed=8)
    Y = tt.add_many([X, X, tt.scale(X, -1.0)])
    g = ttsn.TensorTrain(Y)
    info = g.round(eps=1e-9)
    assert info["ranks"] == [1, 4, 3, 2, 1]
    assert _rel(g.full().cpu().numpy(), tt.full(X)) < 1e-10


def test_rank_cap_reports_warning_state(ttsn):
    X = _decaying([50, 9, 10], 12, 1.2, seed=9)
    g = ttsn.TensorTrain(X)
    info = g.round(eps=1e-12, max_rank=3)
    assert info["capped"]
    assert max(info["ranks"]) <= 3


def test_zero_tensor(ttsn):
    X = [np.zeros((1, 4, 2)), np.zeros((2, 3, 2)), np.zeros((2, 5, 1))]
    g = ttsn.TensorTrain(X)
    info = g.round(eps=1e-6)
    assert info["ranks"] == [1, 1, 1, 1]
    assert np.abs(g.full().cpu().numpy()).max() == 0.0
