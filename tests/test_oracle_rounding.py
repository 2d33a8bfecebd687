"""Pins for the oracle's TT rounding (App. A): exact recovery, error bound,
brute-force unfolding SVDs, orthonormality, Gram vs TT-SVD agreement."""
import numpy as np
import pytest

import workloads
from oracle import tt
from oracle.rounding import EPS_MACH, choose_rank, round_gram, round_randomized, round_ttsvd, sketch_right

ROUNDERS = [("ttsvd", round_ttsvd, 1e-12), ("gram", round_gram, 1e-10)]


def _rel(A, B):
    return np.linalg.norm(tt.full(A) - tt.full(B)) / np.linalg.norm(tt.full(B))


@pytest.mark.parametrize("name,fn,tol", ROUNDERS)
@pytest.mark.parametrize("modes,ranks", [([20, 6, 9], [4, 3]), ([5, 4, 6, 3], [3, 5, 2])])
def test_exact_recovery_of_redundant_tt(name, fn, tol, modes, ranks):
    X = workloads.random_tt(modes, ranks, seed=4)
    Y = tt.add_many([X, X, tt.scale(X, -1.0)])  # X + X - X, ranks 3r
    assert tt.ranks(Y) == [3 * r for r in ranks]
    Z, _ = fn(Y, eps=1e-9)
    assert tt.ranks(Z) == ranks
    assert _rel(Z, X) < tol


@pytest.mark.parametrize("name,fn,tol", ROUNDERS)
@pytest.mark.parametrize("eps", [1e-1, 1e-2, 1e-4])
def test_error_bound(name, fn, tol, eps):
    # a tensor with a decaying spectrum: sum of rank-1 terms with weights 2^-j
    rng = np.random.default_rng(9)
    terms = []
    for j in range(12):
        vs = [rng.standard_normal(m) for m in (15, 8, 10)]
        vs[0] = vs[0] * 2.0 ** (-j)
        terms.append(tt.rank_one(vs))
    X = tt.add_many(terms)
    Z, _ = fn(X, eps=eps)
    err = np.linalg.norm(tt.full(Z) - tt.full(X))
    assert err <= eps * np.linalg.norm(tt.full(X)) * (1 + 1e-8)
    assert max(tt.ranks(Z)) < 12


@pytest.mark.parametrize("modes", [[3, 4, 2], [2, 3, 4, 3], [4, 2, 3, 2, 3]])
def test_ttsvd_bond_singular_values_equal_unfolding_svd(modes):
    # brute force: with no truncation, bond k's singular values are those of the
    # k-th unfolding of the full tensor (Oseledets 2011, Thm 2.1)
    X = workloads.random_tt(modes, [3] * (len(modes) - 1), seed=12)
    F = tt.full(X)
    _, sig = round_ttsvd(X, eps=0.0)
    for k in range(len(modes) - 1):
        U = F.reshape(int(np.prod(modes[: k + 1])), -1)
        s_ref = np.linalg.svd(U, compute_uv=False)
        m = len(sig[k])
        assert np.allclose(sig[k], s_ref[:m], rtol=1e-12, atol=1e-13 * s_ref[0])
        assert np.all(s_ref[m:] < 1e-12 * s_ref[0])


@pytest.mark.parametrize("name,fn,tol", ROUNDERS)
def test_left_cores_orthonormal(name, fn, tol):
    X = workloads.random_tt([30, 7, 8, 5], [6, 5, 4], seed=21)
    Z, _ = fn(X, eps=1e-3)
    for G in Z[:-1]:
        r0, n, r1 = G.shape
        A = G.reshape(r0 * n, r1)
        assert np.abs(A.T @ A - np.eye(r1)).max() < (1e-12 if name == "ttsvd" else 1e-9)


def test_gram_singular_values_match_ttsvd_to_sqrt_eps():
    X = workloads.random_tt([40, 9, 11], [7, 5], seed=31)
    _, s1 = round_ttsvd(X, eps=0.0)
    _, s2 = round_gram(X, eps=0.0)
    for a, b in zip(s1, s2):
        m = min(len(a), len(b))
        assert np.abs(a[:m] - b[:m]).max() <= 10 * np.sqrt(EPS_MACH) * a[0]


def test_gram_and_ttsvd_agree_at_forced_ranks():
    rng = np.random.default_rng(41)
    terms = []
    for j in range(10):
        vs = [rng.standard_normal(m) for m in (25, 6, 12)]
        vs[0] = vs[0] * 3.0 ** (-j)
        terms.append(tt.rank_one(vs))
    X = tt.add_many(terms)
    A, _ = round_ttsvd(X, forced=[4, 4])
    B, _ = round_gram(X, forced=[4, 4])
    assert tt.ranks(A) == tt.ranks(B) == [4, 4]
    assert _rel(B, A) < 1e-10


def test_choose_rank_rule():
    S = np.array([4.0, 2.0, 1.0, 0.5])
    # tails: r=1 -> 4+1+0.25=5.25, r=2 -> 1.25, r=3 -> 0.25, r=4 -> 0
    assert choose_rank(S, np.sqrt(1.25)) == 2
    assert choose_rank(S, np.sqrt(1.2)) == 3
    assert choose_rank(S, 0.0) == 4
    assert choose_rank(S, 100.0) == 1
    assert choose_rank(S, 0.0, max_rank=2) == 2
    assert choose_rank(S, 0.0, forced=9) == 4


def test_zero_tensor_rounds_to_rank_one_zero():
    X = [np.zeros((1, 4, 2)), np.zeros((2, 3, 2)), np.zeros((2, 5, 1))]
    Z, _ = round_gram(X, eps=1e-6)
    assert tt.ranks(Z) == [1, 1]
    assert np.abs(tt.full(Z)).max() == 0.0


def _omega(modes, ranks, seed):
    rng = np.random.default_rng(seed)
    r = [1] + list(ranks) + [1]
    return [rng.standard_normal((r[k], m, r[k + 1])) for k, m in enumerate(modes)]


def test_randomized_rounding_recovers_an_exact_low_rank_tt():
    """A TT of ranks r written redundantly (X + X - X, ranks 3r): a sketch of
    ranks >= r spans the exact column spaces with probability one, so the
    randomized rounding returns the same tensor (App. A.3)."""
    modes, ranks = [5, 6, 4, 7], [2, 3, 2]
    A = workloads.random_tt(modes, ranks, seed=11)
    X = tt.add(tt.add(A, A), tt.scale(A, -1.0))
    for sketch in ([2, 3, 2], [4, 5, 3]):
        Z = round_randomized(X, _omega(modes, sketch, 12))
        assert tt.ranks(Z) == sketch
        F = tt.full(A)
        assert np.abs(tt.full(Z) - F).max() <= 1e-12 * np.abs(F).max()


def test_randomized_rounding_error_near_optimal_with_oversampling():
    """For a tensor with decaying unfolding spectra the randomized projection
    at sketch rank r + p stays within a small factor of the best rank-r + p
    truncation's error (TT-SVD at the same ranks), and left cores are
    orthonormal."""
    modes = [8, 7, 6, 5]
    rng = np.random.default_rng(5)
    cores = [rng.standard_normal((1 if k == 0 else 6, m, 1 if k == 3 else 6)) * np.geomspace(1, 1e-3, 6)[None, None, :]
             if k < 3 else rng.standard_normal((6, m, 1)) for k, m in enumerate(modes)]
    F = tt.full(cores)
    sk = [4, 4, 4]
    Z = round_randomized(cores, _omega(modes, sk, 6))
    T, _ = round_ttsvd(cores, forced=sk)
    e_rand = np.linalg.norm(tt.full(Z) - F)
    e_opt = np.linalg.norm(tt.full(T) - F)
    assert e_rand <= 20 * e_opt + 1e-14 * np.linalg.norm(F), (e_rand, e_opt)
    for G in Z[:-1]:
        M = G.reshape(-1, G.shape[2])
        assert np.abs(M.T @ M - np.eye(M.shape[1])).max() <= 1e-12


def test_sketch_right_equals_full_contraction():
    """W_k of the backward sweep is the right unfolding of the tensor times the
    random TT's right part, contracted over all modes after bond k."""
    modes = [4, 3, 5, 2]
    X = workloads.random_tt(modes, [2, 3, 2], seed=21)
    Om = _omega(modes, [3, 2, 2], 22)
    W = sketch_right(X, Om)
    for k in range(3):
        # reference: contract cores k+1..d of X and of Omega directly
        Bx = X[k + 1]
        Bo = Om[k + 1]
        for j in range(k + 2, 4):
            Bx = np.tensordot(Bx, X[j], axes=([Bx.ndim - 1], [0]))
            Bo = np.tensordot(Bo, Om[j], axes=([Bo.ndim - 1], [0]))
        ax = list(range(1, Bx.ndim))
        ref = np.tensordot(Bx, Bo, axes=(ax, ax))
        assert np.allclose(W[k], ref, rtol=1e-12, atol=1e-12)
