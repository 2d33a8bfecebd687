"""GPU checks of the rounding building blocks (through the C ABI):
FP64 GEMM, split-K left Gram, Jacobi eigensolver."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ttsn():
    import torch

    assert torch.cuda.is_available()
    import paper_2503_18056_gb300 as m

    return m


@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (7, 9, 5), (64, 64, 16), (130, 67, 301), (333, 129, 77)])
@pytest.mark.parametrize("ta,tb", [(False, False), (True, False), (False, True), (True, True)])
def test_dgemm_matches_numpy(ttsn, M, N, K, ta, tb):
    rng = np.random.default_rng(M * 1000 + N + K)
    A = rng.standard_normal((K, M) if ta else (M, K))
    B = rng.standard_normal((N, K) if tb else (K, N))
    ref = (A.T if ta else A) @ (B.T if tb else B)
    C = ttsn.dgemm(A, B, trans_a=ta, trans_b=tb).cpu().numpy()
    assert np.abs(C - ref).max() <= 1e-13 * max(1.0, np.abs(ref).max()) * np.sqrt(K)


@pytest.mark.parametrize("m,n", [(1, 1), (5, 3), (1000, 64), (4099, 130), (200000, 37), (3000, 897)])
def test_gram_matches_numpy_and_is_symmetric(ttsn, m, n):
    rng = np.random.default_rng(m + n)
    A = rng.standard_normal((m, n))
    G = ttsn.gram(A).cpu().numpy()
    ref = A.T @ A
    assert np.array_equal(G, G.T)
    assert np.abs(G - ref).max() <= 1e-13 * np.abs(ref).max() * np.sqrt(m)
    G2 = ttsn.gram(A).cpu().numpy()
    assert np.array_equal(G, G2)  # reproducible


@pytest.mark.parametrize("n", [1, 2, 3, 8, 33, 64, 95, 96, 97, 100, 257, 640])
def test_syev_reconstructs_and_matches_numpy(ttsn, n):
    rng = np.random.default_rng(n)
    X = rng.standard_normal((n + 5, n))
    G = X.T @ X
    lam, Vt, sweeps = ttsn.syev(G)
    lam, Vt = lam.cpu().numpy(), Vt.cpu().numpy()
    ref = np.sort(np.linalg.eigvalsh(G))[::-1]
    assert np.all(np.diff(lam) <= 0)
    assert np.abs(lam - ref).max() <= 1e-13 * ref[0] * max(1, np.sqrt(n))
    assert np.abs(Vt @ Vt.T - np.eye(n)).max() <= 1e-12 * max(1, np.sqrt(n))
    R = Vt.T @ np.diag(lam) @ Vt
    assert np.abs(R - G).max() <= 1e-12 * ref[0] * max(1, np.sqrt(n))
    assert sweeps <= 20


@pytest.mark.parametrize("n", [60, 300])
def test_syev_rank_deficient_gram(ttsn, n):
    # a Gram matrix of rank 10 padded to n: the null block must not stall Jacobi
    rng = np.random.default_rng(3)
    X = rng.standard_normal((10, n))
    G = X.T @ X
    lam, Vt, sweeps = ttsn.syev(G)
    lam = lam.cpu().numpy()
    ref = np.sort(np.linalg.eigvalsh(G))[::-1]
    assert np.abs(lam[:10] - ref[:10]).max() <= 1e-12 * ref[0]
    assert np.abs(lam[10:]).max() <= 1e-12 * ref[0]
    assert sweeps < 40


def test_syev_diagonal_and_degenerate(ttsn):
    G = np.diag([3.0, 1.0, 2.0, 2.0, 0.0])
    lam, Vt, sweeps = ttsn.syev(G)
    assert np.allclose(lam.cpu().numpy(), [3, 2, 2, 1, 0])
    G = np.ones((6, 6))
    lam, _, _ = ttsn.syev(G)
    assert np.allclose(lam.cpu().numpy(), [6, 0, 0, 0, 0, 0], atol=1e-14)


# n <= 384: one CTA; larger n: several CTAs with a grid barrier per pivot
@pytest.mark.parametrize("n,rank", [(1, 1), (51, 15), (61, 16), (200, 57), (600, 100), (897, 128)])
@pytest.mark.parametrize("spread", [1e-2, 1e-7])
def test_pchol_reconstructs_rank_deficient_gram(ttsn, n, rank, spread):
    """Pivoted Cholesky of G = B^T B with B (rank x n) of singular values from 1
    down to `spread`: W^T W reproduces G to the eps_mach max(diag G) floor at
    which the factorisation stops (pivots at the rounding-noise level above
    that floor may add rows beyond the true rank).  Columns whose
    residual rounds below zero must keep their later entries; dropping them
    leaves errors of sqrt(eps_mach) times the pivots' scale."""
    import torch

    rng = np.random.default_rng(n + rank)
    U, _ = np.linalg.qr(rng.standard_normal((rank, rank)))
    V, _ = np.linalg.qr(rng.standard_normal((n, rank)))
    S = np.geomspace(1.0, spread, rank)
    B = (U * S) @ V.T
    G = B.T @ B
    G = 0.5 * (G + G.T)
    for _ in range(3):
        W, k = ttsn.pchol(torch.tensor(G, device="cuda"))
        W = W.cpu().numpy()
        assert 1 <= k <= n
        # Cholesky backward error (k + 1) eps |W^T| |W| plus the neglected
        # Schur complement, whose entries are below the eps max(diag) floor
        assert np.abs(W.T @ W - G).max() <= 4 * (rank + 1) * np.finfo(float).eps * np.abs(np.diag(G)).max()
