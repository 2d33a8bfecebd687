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


# (100, 7, 33), (5000, 37, 64) and (161, 161, 5184) -- an R x R right Gram
# over a long contraction -- have few output tiles and run split-K
@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (100, 7, 33), (70000, 128, 897), (5000, 37, 64), (161, 161, 5184)])
def test_gemm_nt_mixed_within_split_bound(ttsn, M, N, K):
    rng = np.random.default_rng(M + N + K)
    A = rng.standard_normal((M, K)) * 10.0 ** rng.uniform(-8, 0, (M, 1))
    B = rng.standard_normal((N, K))
    C = ttsn.gemm_nt_mixed(A, B).cpu().numpy()
    ref = A @ B.T
    bound = 8 * U * K * np.outer(np.abs(A).max(axis=1), np.abs(B).max(axis=1))
    assert np.all(np.abs(C - ref) <= bound + 1e-16 * np.abs(ref))


# Worst-case level sums.  A value whose seven balanced base-128 digits are
# all 63 (the largest the split produces below the leading one) makes every
# digit product of a level w equal 63^2, so a block of R contraction indices
# sums (w + 1) 63^2 R at level w: 14.2M at w = 6 and 10.2M at w = 4 for
# R = 512, above 2^23 and below 2^24.  The tensor cores must add these
# integers exactly; a lost unit at level w <= 4 moves a term by >= 2^-38 of
# its size, far above the double-float drain's rounding (the tolerance
# below).  The expected value is the truncated scheme's own exact result:
# sum over levels w <= 6 of (w + 1) 63^2 128^-(w+2), times 2^(e_j + e_k),
# computed in rationals.
_F63 = sum(63 * 128 ** (6 - s) for s in range(7))  # digits 63, 63, ..., 63


def _digit63_values(count, seed):
    """Values +-F 2^(k - 47) (F = _F63, so |v| in [1, 2) 2^k) with their split exponents e = k + 2."""
    rng = np.random.default_rng(seed)
    k = rng.integers(-6, 7, count)
    sign = rng.choice([-1.0, 1.0], count)
    v = sign * np.ldexp(float(_F63), k - 47)
    assert np.all(np.abs(v) * 2.0 ** -(k + 2) < 0.5) and np.all(np.abs(v) * 2.0 ** -(k + 2) >= 0.25)
    return v, sign, k + 2


def _trunc_products(sign_a, e_a, sign_b, e_b):
    from fractions import Fraction

    unit = sum(Fraction((w + 1) * 63 * 63, 128 ** (w + 2)) for w in range(7))
    out = np.empty((len(sign_a), len(sign_b)))
    for i in range(len(sign_a)):
        for j in range(len(sign_b)):
            out[i, j] = float(int(sign_a[i] * sign_b[j]) * unit * Fraction(2) ** int(e_a[i] + e_b[j]))
    return out


def test_gram_mixed_exact_block_sums_at_the_digit_bound(ttsn):
    m, n = 512 * 8 + 96, 70  # eight full 512-row blocks and a ragged one; two column tiles
    v, sign, e = _digit63_values(n, 11)
    A = np.tile(v, (m, 1))
    G = ttsn.gram_mixed(A).cpu().numpy()
    ref = m * _trunc_products(sign, e, sign, e)
    assert np.all(np.abs(G - ref) <= 2.0 ** -44 * np.abs(ref))
    exact = m * np.outer(v, v)  # the untruncated product: the split's stated bound
    assert np.all(np.abs(G - exact) <= 8 * U * m * np.outer(np.abs(v), np.abs(v)))


def test_gemm_nt_mixed_exact_block_sums_at_the_digit_bound(ttsn):
    M, N, K = 300, 130, 512 * 2 + 40
    va, sa, ea = _digit63_values(M, 12)
    vb, sb, eb = _digit63_values(N, 13)
    A = np.tile(va[:, None], (1, K))
    B = np.tile(vb[:, None], (1, K))
    C = ttsn.gemm_nt_mixed(A, B).cpu().numpy()
    ref = K * _trunc_products(sa, ea, sb, eb)
    assert np.all(np.abs(C - ref) <= 2.0 ** -44 * np.abs(ref))


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
