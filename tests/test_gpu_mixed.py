"""Precision form: exact-split BF16 contractions and the mixed TT-S_N step.

The split (six balanced base-256 digits per scaled value, exact BF16 products,
exact FP32 block sums, double-float accumulation) bounds the error of every
product term by a few 2^-48 of the scales involved, with zero-mean residuals;
the tests check that bound, a 1e-12 relative Frobenius error, and the step's
agreement with the FP64 GPU step at equal ranks (target <= 1e-6)."""
import numpy as np
import pytest

import workloads
from oracle import tt

pytestmark = pytest.mark.gpu

U = 2.0 ** -48


@pytest.fixture(scope="module")
def ttsn():
    import torch

    assert torch.cuda.is_available()
    import paper_2503_18056_gb300 as m

    return m


@pytest.mark.parametrize("m,n,spread", [(1, 1, 0), (37, 5, 0), (5000, 130, 0), (300000, 449, 0),
                                        (200000, 97, 8), (40000, 897, 3)])
def test_gram_mixed_within_split_bound(ttsn, m, n, spread):
    rng = np.random.default_rng(m + n)
    A = rng.standard_normal((m, n))
    if spread:  # rows spanning `spread` decades (background vs peak cells)
        A *= 10.0 ** rng.uniform(-spread, 0, (m, 1))
    G = ttsn.gram_mixed(A).cpu().numpy()
    ref = A.T @ A
    cm = np.abs(A).max(axis=0)
    bound = 8 * U * m * np.outer(cm, cm) + 1e-15 * np.abs(ref).max()
    assert np.array_equal(G, G.T)
    assert np.all(np.abs(G - ref) <= bound)
    assert np.linalg.norm(G - ref) <= 1e-12 * np.linalg.norm(ref)


@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (100, 7, 33), (70000, 128, 897), (5000, 37, 64)])
def test_gemm_nt_mixed_within_split_bound(ttsn, M, N, K):
    rng = np.random.default_rng(M + N + K)
    A = rng.standard_normal((M, K)) * 10.0 ** rng.uniform(-8, 0, (M, 1))
    B = rng.standard_normal((N, K))
    C = ttsn.gemm_nt_mixed(A, B).cpu().numpy()
    ref = A @ B.T
    bound = 8 * U * K * np.outer(np.abs(A).max(axis=1), np.abs(B).max(axis=1))
    assert np.all(np.abs(C - ref) <= bound + 1e-16 * np.abs(ref))


def _fp64_then_mixed(ttsn, p, steps):
    g64 = ttsn.TTSN.from_problem(p)
    ranks = []
    for _ in range(steps):
        info = g64.step()
        ranks.append(info["ranks"][1:-1])
    gmx = ttsn.TTSN.from_problem(p, precision=ttsn.TT_MIXED)
    for r in ranks:
        info = gmx.step(forced=r)
        assert info["ranks"][1:-1] == r
    return g64, gmx


def test_mixed_step_matches_fp64_at_fp64_ranks(ttsn):
    # 2D 48x40 cells, 16x32 ordinates, vacuum, eps = 1e-5: the precision form
    # replays the FP64 GPU run's ranks; stated error target 1e-6
    p = workloads.problem("small_2d", n=(48, 40), n_theta=16, n_phi=32, eps=1e-5,
                          bc=workloads.VACUUM, max_rank=96)
    g64, gmx = _fp64_then_mixed(ttsn, p, 6)
    F64 = g64.full().cpu().numpy()
    FMX = gmx.full().cpu().numpy()
    err = np.linalg.norm(FMX - F64) / np.linalg.norm(F64)
    E64, T64, _ = g64.energy()
    EMX, TMX, _ = gmx.energy()
    errT = (TMX - T64).abs().max().item() / T64.abs().max().item()
    print("mixed vs fp64: full-tensor rel. %.2e, T rel. %.2e" % (err, errT))
    assert err <= 1e-6
    assert errT <= 1e-6


def test_mixed_step_conserves_energy_periodic(ttsn):
    p = workloads.problem("small_2d", n=(24, 24), n_theta=8, n_phi=16, eps=1e-4)
    g = ttsn.TTSN.from_problem(p, precision=ttsn.TT_MIXED)
    _, _, t0 = g.energy()
    g.step(4)
    _, _, t1 = g.energy()
    assert abs(sum(t1) - sum(t0)) <= 1e-12 * sum(t0)


def test_mixed_rounding_matches_oracle_at_forced_ranks(ttsn):
    rng = np.random.default_rng(2)
    terms = []
    for j in range(12):
        vs = [rng.standard_normal(m) for m in (300, 9, 11)]
        vs[0] = vs[0] * 2.5 ** (-j)
        terms.append(tt.rank_one(vs))
    X = tt.add_many(terms)
    from oracle.rounding import round_ttsvd

    ref, _ = round_ttsvd(X, forced=[6, 6])
    g = ttsn.TensorTrain(X)
    g.set_precision(ttsn.TT_MIXED)
    g.round(forced=[6, 6])
    F = g.full().cpu().numpy()
    assert np.linalg.norm(F - tt.full(ref)) <= 1e-10 * np.linalg.norm(tt.full(ref))
