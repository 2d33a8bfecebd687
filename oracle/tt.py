"""Tensor-train arithmetic of Sec. 4.1 (oracle; test infrastructure).

A TT is a list of cores, core k an array of shape (r_{k-1}, n_k, r_k) with
r_0 = r_d = 1 (Sec. 4.1 / App. A notation).  Functions follow the paper's
definitions literally: addition concatenates the first core, block-diagonalises
the middle cores and stacks the last core (ranks add); the Hadamard product
takes Kronecker products of core slices (ranks multiply); integration over the
angular cores contracts them with the quadrature weights (Eq.
tt_energy_density).
"""
import numpy as np


def full(cores):
    """Expand a TT to the full array of shape (n_1, ..., n_d)."""
    out = cores[0]  # (1, n1, r1)
    for G in cores[1:]:
        out = np.tensordot(out, G, axes=([out.ndim - 1], [0]))
    return out.reshape(out.shape[1:-1])


def ranks(cores):
    return [G.shape[2] for G in cores[:-1]]


def add(A, B):
    """V = A + B in TT format (Sec. 4.1, Addition)."""
    d = len(A)
    assert len(B) == d
    if d == 1:
        return [A[0] + B[0]]
    out = []
    for k in range(d):
        a, b = A[k], B[k]
        n = a.shape[1]
        assert b.shape[1] == n
        if k == 0:
            out.append(np.concatenate([a, b], axis=2))
        elif k == d - 1:
            out.append(np.concatenate([a, b], axis=0))
        else:
            G = np.zeros((a.shape[0] + b.shape[0], n, a.shape[2] + b.shape[2]))
            G[: a.shape[0], :, : a.shape[2]] = a
            G[a.shape[0]:, :, a.shape[2]:] = b
            out.append(G)
    return out


def add_many(terms):
    out = terms[0]
    for t in terms[1:]:
        out = add(out, t)
    return out


def hadamard(A, B):
    """V = A * B elementwise in TT format (Sec. 4.1, Multiplication)."""
    out = []
    for a, b in zip(A, B):
        ra0, n, ra1 = a.shape
        rb0, _, rb1 = b.shape
        G = np.einsum("aib,cid->acibd", a, b).reshape(ra0 * rb0, n, ra1 * rb1)
        out.append(G)
    return out


def scale(A, alpha):
    """alpha * A (the scalar multiplies the first core)."""
    out = [G.copy() for G in A]
    out[0] = out[0] * alpha
    return out


def rank_one(vectors):
    """Rank-1 TT whose k-th core is the vector ``vectors[k]``."""
    return [np.asarray(v, float).reshape(1, -1, 1) for v in vectors]


def inner(A, B):
    """<A, B> by sequential contraction of core pairs."""
    W = np.ones((1, 1))
    for a, b in zip(A, B):
        W = np.einsum("ac,aib,cid->bd", W, a, b)
    return float(W[0, 0])


def norm(A):
    return float(np.sqrt(max(inner(A, A), 0.0)))


def energy_density_grouped(cores, w, v, c):
    """E_i = (1/c) X_i (sum_l Theta_l w_l)(sum_p Phi_p v_p), Eq. tt_energy_density,
    for the three-core layout (X, Theta, Phi)."""
    X, Th, Ph = cores
    phibar = np.einsum("bp,p->b", Ph[:, :, 0], v)
    thbar = np.einsum("alb,l,b->a", Th, w, phibar)
    return np.einsum("ia,a->i", X[0], thbar) / c
