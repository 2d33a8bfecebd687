"""Eigenpairs of positive semidefinite matrices by pivoted Cholesky and
one-sided Jacobi (tt_syev_psd), the eigensolver of the rounding's K = W G_A W^T
(App. A.2), against the two-sided Jacobi (tt_syev) and NumPy."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

EPS = np.finfo(float).eps


@pytest.fixture(scope="module")
def ttsn():
    assert torch.cuda.is_available()
    import paper_2503_18056_gb300 as m

    return m


def _graded(n, lo, seed, cond=10.0):
    """K = D A D with D = diag(geomspace(1, lo, n)) and A symmetric positive
    definite with unit diagonal and condition ~cond: its eigenvalues span
    1 .. ~lo^2 and are fixed to relative accuracy ~eps cond by the entries
    (Demmel & Veselic 1992), which both Jacobi forms attain."""
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = (Q * np.geomspace(1.0, 1.0 / cond, n)) @ Q.T
    s = 1.0 / np.sqrt(np.diag(A))
    A = s[:, None] * A * s[None, :]
    d = np.geomspace(1.0, lo, n)
    return d[:, None] * A * d[None, :]


@pytest.mark.parametrize("n,lo", [(2, 1e-3), (37, 1e-4), (200, 1e-6), (897, 1e-6)])
def test_psd_eigenpairs_match_two_sided_jacobi_to_relative_accuracy(ttsn, n, lo):
    K = _graded(n, lo, seed=n)
    lp, Vp, swp = ttsn.syev_psd(K)
    lt, Vt, swt = ttsn.syev(K)
    lp, Vp, lt = lp.cpu().numpy(), Vp.cpu().numpy(), lt.cpu().numpy()
    print("n %d: one-sided %d sweeps, two-sided %d sweeps" % (n, swp, swt))
    assert np.all(np.diff(lp) <= 0)
    # every eigenvalue to relative accuracy (both are relatively accurate; the
    # scaled matrix has condition ~10, so the bound is a few hundred eps n)
    assert np.max(np.abs(lp - lt) / lt) <= 100 * n * EPS
    # orthonormal eigenvectors and small residuals relative to each eigenvalue's scale
    assert np.abs(Vp @ Vp.T - np.eye(n)).max() <= 50 * np.sqrt(n) * EPS
    R = K @ Vp.T - Vp.T * lp[None, :]
    assert np.linalg.norm(R, axis=0).max() <= 100 * n * EPS * np.abs(K).max()
    # and the ordinary accuracy against NumPy
    ln = np.sort(np.linalg.eigvalsh(K))[::-1]
    assert np.abs(lp - ln).max() <= 100 * n * EPS * ln[0]


def test_psd_rank_deficient_matrix_returns_zero_tail(ttsn):
    rng = np.random.default_rng(3)
    n, r = 120, 40
    B = rng.standard_normal((r, n)) * np.geomspace(1.0, 1e-3, n)[None, :]
    K = B.T @ B
    lam, Vt, _ = ttsn.syev_psd(K)
    lam, Vt = lam.cpu().numpy(), Vt.cpu().numpy()
    k = int(np.sum(lam > 0))
    assert r <= k <= n
    assert np.all(lam[k:] == 0.0) and np.all(Vt[k:] == 0.0)
    Kr = (Vt[:k].T * lam[:k]) @ Vt[:k]
    assert np.abs(Kr - K).max() <= 1e3 * n * EPS * np.abs(K).max()
    ln = np.sort(np.linalg.eigvalsh(K))[::-1]
    assert np.abs(lam[:r] - ln[:r]).max() <= 100 * n * EPS * ln[0]


def test_psd_sweep_limit_is_reported(ttsn):
    from paper_2503_18056_gb300 import _native

    K = _graded(64, 1e-3, seed=9)
    lam, Vt, sw = ttsn.syev_psd(K, allow_unconverged=True, max_sweeps=1)
    assert sw == 1
    with pytest.raises(_native.TTError):
        ttsn.syev_psd(K, max_sweeps=1)
    lam, Vt, sw = ttsn.syev_psd(K)
    assert 1 < sw < 40


def test_psd_is_faster_than_two_sided_at_the_rounding_size(ttsn):
    # n = 897: the grown rank of the 128^3 workload at its rank cap
    K = torch.as_tensor(_graded(897, 1e-6, seed=11), device="cuda")
    ttsn.syev_psd(K)
    ttsn.syev(K)
    torch.cuda.synchronize()
    out = {}
    for name, fn in (("psd", ttsn.syev_psd), ("two_sided", ttsn.syev)):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        best = 1e30
        for _ in range(3):
            e0.record()
            fn(K)
            e1.record()
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1))
        out[name] = best
    print("n 897: one-sided %.1f ms, two-sided %.1f ms" % (out["psd"], out["two_sided"]))
    assert out["psd"] < out["two_sided"]
