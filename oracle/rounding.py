"""TT rounding, Algorithm 1 of App. A (oracle; test infrastructure).

Three truncation rules for Step "truncate" of Algorithm 1 (the randomized
one, ``round_randomized``, App. A.3, takes its Gaussian sketch as an input):

* ``round_ttsvd`` -- the traditional TT-SVD rounding of App. A.1
  (Oseledets 2011): QR orthogonalisation in the backward sweep, truncated SVD
  in the forward sweep.  The R factor of B is absorbed into the current core
  during the backward sweep (the standard arrangement), so it is never
  inverted; in exact arithmetic this is App. A.1's A' = Q_A U~,
  M_upd = (R_B^{-1} V~ S~)^T.
* ``round_gram`` -- the Gram-SVD rounding of App. A.2, Eq. gramfinal:
  G_A = A^T A, G_B = B^T B, eigendecompositions G = V S^2 V^T,
  M = S_A V_A^T V_B S_B, truncated SVD M ~ U~ S~ V~^T,
  A' = A V_A S_A^{-1} U~ and M_upd = (V_B S_B^{-1} V~ S~)^T.  The Gram matrices
  of B come from the backward sweep (App. A.2 footnote).

Tolerance (App. A, note on rank truncation): the error is balanced across the
d-1 bonds, delta = eps ||X||_F / sqrt(d-1), and bond k keeps the smallest rank
r >= 1 whose discarded singular values satisfy sum_{j>r} s_j^2 <= delta^2
(Oseledets 2011, Alg. 2).  ``forced`` ranks override the tolerance;
``max_rank`` caps it.  Gram eigenvalues lambda <= R * eps_mach * lambda_max are
discarded before S^{-1} is formed (the paper notes Gram-SVD singular values
carry only sqrt(eps_mach) relative precision, App. A.4 "Stability").
"""
import numpy as np

EPS_MACH = np.finfo(float).eps


def choose_rank(S, delta, max_rank=None, forced=None):
    """Smallest r >= 1 with sum_{j>r} S_j^2 <= delta^2 (S sorted descending)."""
    navail = len(S)
    if navail == 0:
        return 0
    if forced is not None:
        return int(max(1, min(forced, navail)))
    tail = np.concatenate([np.cumsum((S ** 2)[::-1])[::-1], [0.0]])  # tail[r] = sum_{j>=r}
    r = navail
    for cand in range(1, navail + 1):
        if tail[cand] <= delta * delta:
            r = cand
            break
    if max_rank is not None:
        r = min(r, int(max_rank))
    return r


def _forced_k(forced, k):
    return None if forced is None else forced[k]


def round_ttsvd(cores, eps=0.0, max_rank=None, forced=None):
    """Return (rounded cores, list of singular-value arrays per bond)."""
    d = len(cores)
    G = [np.array(c, float) for c in cores]
    # backward sweep: right-orthonormalise cores d..2
    for k in range(d - 1, 0, -1):
        r0, n, r1 = G[k].shape
        Q, R = np.linalg.qr(G[k].reshape(r0, n * r1).T)
        G[k] = Q.T.reshape(Q.shape[1], n, r1)
        G[k - 1] = np.tensordot(G[k - 1], R.T, axes=([2], [0]))
    nrm = float(np.linalg.norm(G[0]))
    delta = eps * nrm / np.sqrt(max(d - 1, 1))
    sig = []
    for k in range(d - 1):
        r0, n, r1 = G[k].shape
        A = G[k].reshape(r0 * n, r1)
        QA, RA = np.linalg.qr(A)
        U, S, Vt = np.linalg.svd(RA, full_matrices=False)
        sig.append(S)
        r = choose_rank(S, delta, max_rank, _forced_k(forced, k))
        G[k] = (QA @ U[:, :r]).reshape(r0, n, r)
        G[k + 1] = np.tensordot(S[:r, None] * Vt[:r], G[k + 1], axes=([1], [0]))
    return G, sig


def right_grams(cores):
    """Backward sweep of Algorithm 1 in Gram form: GB[k] = B_k^T B_k for bond k
    (between cores k and k+1, 0-based)."""
    d = len(cores)
    GB = [None] * (d - 1)
    last = cores[d - 1][:, :, 0]
    GB[d - 2] = last @ last.T
    for k in range(d - 3, -1, -1):
        # the two contractions of App. A.2's backward sweep:
        # W = G_{k+1} x_3 GB[k+1], then GB[k] = W x_{2,3} G_{k+1}
        C = cores[k + 1]
        W = np.tensordot(C, GB[k + 1], axes=([2], [0]))
        GB[k] = np.tensordot(W, C, axes=([1, 2], [1, 2]))
    return GB


def _eig_floored(Gm):
    lam, V = np.linalg.eigh(0.5 * (Gm + Gm.T))
    order = np.argsort(lam)[::-1]
    lam, V = lam[order], V[:, order]
    lmax = lam[0] if len(lam) else 0.0
    keep = lam > Gm.shape[0] * EPS_MACH * lmax
    if lmax <= 0.0:
        keep[:] = False
    return np.sqrt(lam[keep]), V[:, keep]


def round_gram(cores, eps=0.0, max_rank=None, forced=None):
    """Return (rounded cores, list of singular-value arrays of M per bond)."""
    d = len(cores)
    G = [np.array(c, float) for c in cores]
    GB = right_grams(G)
    delta = None
    sig = []
    for k in range(d - 1):
        r0, n, r1 = G[k].shape
        A = G[k].reshape(r0 * n, r1)
        SA, VA = _eig_floored(A.T @ A)
        SB, VB = _eig_floored(GB[k])
        if len(SA) == 0 or len(SB) == 0:  # zero tensor: keep a rank-1 zero TT
            G[k] = np.zeros((r0, n, 1))
            G[k + 1] = np.zeros((1,) + G[k + 1].shape[1:])
            sig.append(np.zeros(0))
            continue
        M = SA[:, None] * (VA.T @ VB) * SB[None, :]
        U, S, Vt = np.linalg.svd(M, full_matrices=False)
        sig.append(S)
        if delta is None:
            delta = eps * float(np.sqrt(np.sum(S ** 2))) / np.sqrt(max(d - 1, 1))
        r = choose_rank(S, delta, max_rank, _forced_k(forced, k))
        Aprime = A @ (VA / SA[None, :]) @ U[:, :r]
        Mupd = ((VB / SB[None, :]) @ Vt[:r].T * S[None, :r]).T
        G[k] = Aprime.reshape(r0, n, r)
        G[k + 1] = np.tensordot(Mupd, G[k + 1], axes=([1], [0]))
    return G, sig


def sketch_right(cores, omega):
    """Backward sweep of the randomized rounding (App. A.3, Eq. randprojection
    W = B^T Omega for every bond): W[k] (R_k x l_k) is the right part of bond k
    (cores k+1..d) contracted over all its modes with the random TT omega
    (cores of shape (l_{k-1}, n_k, l_k)), computed from the last core back."""
    d = len(cores)
    W = [None] * (d - 1)
    W[d - 2] = cores[d - 1][:, :, 0] @ omega[d - 1][:, :, 0].T
    for k in range(d - 2, 0, -1):
        T = np.tensordot(cores[k], W[k], axes=([2], [0]))          # (R_{k-1}, n_k, l_k)
        W[k - 1] = np.tensordot(T, omega[k], axes=([1, 2], [1, 2]))  # (R_{k-1}, l_{k-1})
    return W


def round_randomized(cores, omega):
    """Randomized rounding (App. A.3, Eq. randfinal): for each bond, left to
    right, X = A B^T is replaced by Q (Q^T A) B^T with Q an orthonormal basis of
    the sketch A W, W = B^T Omega from ``sketch_right``; A' = Q, M_upd = Q^T A.
    The output ranks are the sketch ranks l_k (capped by the bond's size)."""
    d = len(cores)
    G = [np.array(c, float) for c in cores]
    W = sketch_right(G, omega)
    for k in range(d - 1):
        r0, n, R = G[k].shape
        A = G[k].reshape(r0 * n, R)
        Y = A @ W[k]
        Q, _ = np.linalg.qr(Y)
        M = Q.T @ A
        G[k] = Q.reshape(r0, n, Q.shape[1])
        G[k + 1] = np.tensordot(M, G[k + 1], axes=([1], [0]))
    return G
