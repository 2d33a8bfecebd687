"""QR-based TT-SVD rounding on the GPU (App. A.1; tt_set_rounding(TT_ROUND_TTSVD))
against the oracle's TT-SVD rounding: single roundings of bare TTs at forced
and tolerance-chosen ranks, singular values below the Gram-SVD resolution,
degenerate tensors, and rounded steps."""
import ctypes

import numpy as np
import pytest
import torch

import workloads
from oracle import tt
from oracle.rounding import round_ttsvd
from oracle.ttstep import TTSN as OracleTTSN

pytestmark = pytest.mark.gpu

EPS_MACH = np.finfo(float).eps


@pytest.fixture(scope="module")
def ttsn():
    assert torch.cuda.is_available()
    import paper_2503_18056_gb300 as m

    return m


def _graded_tt(modes, ranks, seed, low=1e-4):
    rng = np.random.default_rng(seed)
    r = [1] + list(ranks) + [1]
    decay = [np.geomspace(1.0, low, r[k + 1]) for k in range(len(modes))]
    return [rng.standard_normal((r[k], m, r[k + 1])) * decay[k][None, None, :] for k, m in enumerate(modes)]


@pytest.mark.parametrize("modes,ranks,target", [([300, 40, 30], [20, 15], [10, 8]),
                                                ([5000, 16, 32], [60, 12], [25, 12]),
                                                ([64, 32, 16, 8], [12, 20, 6], [8, 10, 6]),
                                                ([37, 5, 3, 9, 11], [7, 13, 9, 5], [4, 6, 5, 3])])
def test_ttsvd_matches_oracle_at_forced_ranks(ttsn, modes, ranks, target):
    X = _graded_tt(modes, ranks, seed=sum(modes))
    ref, sig = round_ttsvd(X, forced=target)
    h = ttsn.TensorTrain(X)
    h.set_rounding("ttsvd")
    info = h.round(forced=target)
    assert info["ranks"][1:-1] == tt.ranks(ref)
    R = tt.full(ref)
    assert np.linalg.norm(h.full().cpu().numpy() - R) <= 1e-10 * np.linalg.norm(R)
    # the discarded tails are the oracle's singular values beyond the cuts
    for k, (S, r) in enumerate(zip(sig, target)):
        tail = float(np.sqrt(np.sum(S[r:] ** 2)))
        assert abs(info["discarded"][k] - tail) <= 1e-12 * np.linalg.norm(S)


def _tt_with_bond_spectrum(n0, n1, n2, sigma, seed):
    """A 3-core TT whose first bond has exactly the singular values sigma:
    orthonormal left core, diag(sigma), right-orthonormal middle and last
    cores, then a well-conditioned gauge change at both bonds so that no core
    is orthonormal any more."""
    rng = np.random.default_rng(seed)
    r1 = len(sigma)
    r2 = 6
    Q0, _ = np.linalg.qr(rng.standard_normal((n0, r1)))
    Q2, _ = np.linalg.qr(rng.standard_normal((n2, r2)))
    Q1, _ = np.linalg.qr(rng.standard_normal((n1 * r2, r1)))
    G0 = Q0.reshape(1, n0, r1)
    G1 = (sigma[:, None] * Q1.T).reshape(r1, n1, r2)
    G2 = Q2.T.reshape(r2, n2, 1)
    T1 = np.eye(r1) + 0.3 * rng.standard_normal((r1, r1)) / np.sqrt(r1)
    T2 = np.eye(r2) + 0.3 * rng.standard_normal((r2, r2)) / np.sqrt(r2)
    G0 = np.tensordot(G0, T1, axes=([2], [0]))
    G1 = np.tensordot(np.linalg.inv(T1), G1, axes=([1], [0]))
    G1 = np.tensordot(G1, T2, axes=([2], [0]))
    G2 = np.tensordot(np.linalg.inv(T2), G2, axes=([1], [0]))
    return [G0, G1, G2]


def test_ttsvd_resolves_singular_values_below_the_gram_limit(ttsn):
    # bond singular values 1 .. 1e-13 (ratio sqrt(10) apart): a Gram matrix
    # resolves them only to sqrt(eps_mach) ~ 1.5e-8 of the largest (App. A.4),
    # the QR-based rounding to eps_mach.  At eps = 1e-11 the cut lies at
    # sigma ~ 1e-11: the GPU keeps the oracle's rank and the same tensor.
    sigma = np.geomspace(1.0, 1e-13, 27)
    X = _tt_with_bond_spectrum(4000, 24, 10, sigma, seed=5)
    eps = 1e-11
    ref, sig = round_ttsvd(X, eps=eps)
    h = ttsn.TensorTrain(X)
    h.set_rounding("ttsvd")
    info = h.round(eps=eps)
    assert info["ranks"][1:-1] == tt.ranks(ref)
    assert 20 <= tt.ranks(ref)[0] < 27
    R = tt.full(ref)
    err = np.linalg.norm(h.full().cpu().numpy() - R) / np.linalg.norm(R)
    # Both sides are backward stable: each computes the truncation of X + dX
    # with ||dX|| <= m u ||X|| (u = eps_mach, m = 4000 the longest inner
    # product: Gram entries, Q^T A).  Truncation at a cut with relative gap
    # sigma_r / (sigma_r - sigma_{r+1}) moves by at most (1 + that) ||dX||.
    r = tt.ranks(ref)[0]
    S = sig[0]
    bound = (1.0 + S[r - 1] / (S[r - 1] - S[r])) * 4000 * EPS_MACH
    assert err <= bound, (err, bound)
    tail = float(np.sqrt(np.sum(S[r:] ** 2)))
    assert abs(info["discarded"][0] - tail) <= 100 * EPS_MACH * np.linalg.norm(S)


def test_ttsvd_recovers_exact_low_rank_and_rounds_zero_to_zero(ttsn):
    modes, ranks = [40, 30, 20, 10], [3, 5, 4]
    A = workloads.random_tt(modes, ranks, seed=71)
    X = tt.add(tt.add(A, A), tt.scale(A, -1.0))  # ranks 9, 15, 12 holding a rank (3, 5, 4) tensor
    h = ttsn.TensorTrain(X)
    h.set_rounding("ttsvd")
    info = h.round(eps=1e-12)
    assert info["ranks"][1:-1] == ranks
    F = tt.full(A)
    assert np.abs(h.full().cpu().numpy() - F).max() <= 1e-11 * np.abs(F).max()
    Z = [np.zeros_like(c) for c in X]
    hz = ttsn.TensorTrain(Z)
    hz.set_rounding("ttsvd")
    info = hz.round(eps=1e-6)
    assert info["ranks"] == [1, 1, 1, 1, 1]
    assert float(hz.full().abs().max()) == 0.0


def _oracle(p, **kw):
    I0 = p["c"] * p["a_r"] * p["Tr0"] ** 4 / (4 * np.pi)
    return OracleTTSN(p["n"], p["L"], p["n_theta"], p["n_phi"], p["c"], p["a_r"], p["dt"], p["bc"],
                      p["sigma_a"], p["cv"], p["T0"],
                      OracleTTSN.isotropic_cores(I0.reshape(-1), p["n_theta"], p["n_phi"]),
                      eps=p["eps"], max_rank=p.get("max_rank"), rounding="ttsvd", **kw)


def test_ttsvd_steps_choose_the_oracles_ranks_and_match(ttsn):
    # free rank decisions on both sides (the same tolerance rule on the same
    # singular values), 16 x 12 cells, 4 x 8 ordinates, eps = 1e-5
    p = workloads.problem("small_2d", n=(16, 12), n_theta=4, n_phi=8, eps=1e-5, bc=1)
    ref = _oracle(p)
    g = ttsn.TTSN.from_problem(p)
    g.set_rounding("ttsvd")
    for _ in range(4):
        ref.step()
        info = g.step()
        assert info["ranks"][1:-1] == tt.ranks(ref.cores)
    R = ref.full()
    assert np.linalg.norm(g.full().cpu().numpy() - R) <= 1e-10 * np.linalg.norm(R)
    _, T, _ = g.energy()
    assert np.abs(T.cpu().numpy() - ref.T).max() <= 1e-12


def _gap_ranks(sig, ranks, ratio=1.05):
    out = []
    for S, r in zip(sig, ranks):
        while r < len(S) and S[r] > 0 and S[r - 1] / S[r] < ratio:
            r += 1
        out.append(r)
    return out


@pytest.mark.parametrize("eps", [1e-8, 1e-6])
def test_small_2d_workload_at_gap_cuts_with_ttsvd(ttsn, eps):
    # The 32 x 32 pulse (8 x 16 ordinates, 10 steps) at its stated tolerances,
    # every cut moved to the next clear gap (the problem's symmetry makes
    # exactly equal singular-value pairs).  With the QR-based rounding the
    # cut at sigma ~ 1e-8 sigma_1 is far above the resolution (eps_mach), so
    # the run holds the 1e-10 parity bar where the Gram path is limited by
    # its sqrt(eps_mach) resolution.
    p = workloads.problem("small_2d", eps=eps)
    ref = _oracle(p)
    g = ttsn.TTSN.from_problem(p)
    g.set_rounding("ttsvd")
    for _ in range(p["steps"]):
        grown, _, _ = ref.source(ref.transport(ref.cores))
        Z, sig = round_ttsvd(grown, eps=p["eps"])
        forced = _gap_ranks(sig, tt.ranks(Z))
        ref.step(forced=forced)
        info = g.step(forced=forced)
        assert info["ranks"][1:-1] == tt.ranks(ref.cores)
    R = ref.full()
    err = np.linalg.norm(g.full().cpu().numpy() - R) / np.linalg.norm(R)
    print("small_2d eps %.0e, TT-SVD rounding at gap cuts: rel. difference %.2e" % (eps, err))
    assert err <= 1e-10


def test_ttsvd_is_refused_where_the_gram_factors_are_needed(ttsn):
    from paper_2503_18056_gb300 import _native

    p = workloads.problem("small_2d", n=(8, 6), n_theta=4, n_phi=8, eps=1e-5, bc=1)
    g = ttsn.TTSN.from_problem(p)
    g.tape_begin(2)
    with pytest.raises(_native.TTError) as e:
        g.set_rounding("ttsvd")
    assert e.value.status == -6  # TT_ERR_STATE: the tape records Gram-SVD factors
    g.tape_clear()
    g.set_rounding("ttsvd")
    with pytest.raises(_native.TTError):
        g.set_graph(True)
    assert _native.lib.tt_set_rounding(g._h, 7) == -1
