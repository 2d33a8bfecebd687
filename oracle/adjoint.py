"""Boundary-escape energy and its exact gradient for the dense stepper
(oracle; test infrastructure).

Objective (the adjoint form's functional): the radiation energy that leaves
through the boundary faces, summed over the steps m = 1..M of a run,

    Q = sum_m sum_{faces f} sum_{cells i on f} sum_{lp} dt dA_f (n_lp . n_f)^+ I^m_{ilp} dOmega_lp,

with n_f the outward normal of face f (Sec. 3 normals, Sec. 4.5 boundaries) and
dA_f the face area (the product of the other axes' cell widths).  Q is linear
in each I^m.

The gradient dQ/dsigma_a is computed by reverse mode through the dense scheme
of Sec. 3 (``dense.DenseSN``), step by step in reverse:
  T' = T + (E* - E')/C_v, E' = (1/c) sum I' dOmega        (energy update)
  I' = s I* + e, s = 1/(1+k), e = s k B, B = c a_r T+^4/4pi (Eq. couple_a, sigma_s = 0)
  T+ from gamma a_r T+^4 + T+ = T + gamma E*, gamma = k/((1+k) C_v)  (Eq. couple_b;
      derivatives by the implicit-function theorem)
  E* = (1/c) sum I* dOmega,  I* = L I (the upwind operator of Eq. lhs / upwind;
      its transpose is applied by ``transport_T``)
  k = c dt sigma_a.
"""
import numpy as np

from . import angles
from .dense import PERIODIC, VACUUM, DenseSN


def face_weights(d: DenseSN):
    """W[i..., l, p] = sum over boundary faces f touching cell i of
    dt dA_f (n . n_f)^+ dOmega (the objective's weight, an array like I)."""
    n = d.n
    W = np.zeros(n + d.dOmega.shape)
    for a in range(d.ndim):
        if d.bc[a] == PERIODIC:
            continue  # no boundary in a periodic direction
        dA = float(np.prod([d.dx[b] for b in range(d.ndim) if b != a]))
        na = d.nvec[a]
        for side, sgn in ((-1, 1.0), (0, -1.0)):  # high face: +e_a, low face: -e_a
            sl = [slice(None)] * d.ndim
            sl[a] = side
            W[tuple(sl)] += d.dt * dA * np.maximum(sgn * na, 0.0) * d.dOmega
    return W


def transport_T(d: DenseSN, G):
    """Transpose of the upwind transport operator applied to an adjoint G."""
    out = G.copy()
    for a in range(d.ndim):
        na = d.nvec[a]
        nu = d.c * d.dt / d.dx[a]
        pos = np.where(na > 0.0, na, 0.0)
        neg = np.where(na < 0.0, na, 0.0)
        # forward: I*_i -= nu [pos (I_i - I_{i-1}) + neg (I_{i+1} - I_i)]
        # transpose: G_i -> -nu (pos - neg) G_i, G_{i-1} += nu pos G_i, G_{i+1} -= nu neg G_i
        out -= nu * (pos - neg) * G
        up = np.zeros_like(G)   # contribution to cell i-1 from G_i
        dn = np.zeros_like(G)   # contribution to cell i+1 from G_i
        N = d.n[a]
        src = [slice(None)] * G.ndim
        dst = [slice(None)] * G.ndim
        if d.bc[a] == PERIODIC:
            up = np.roll(nu * pos * G, -1, axis=a)
            dn = np.roll(-nu * neg * G, 1, axis=a)
        else:
            src[a], dst[a] = slice(1, N), slice(0, N - 1)
            up[tuple(dst)] = (nu * pos * G)[tuple(src)]
            src[a], dst[a] = slice(0, N - 1), slice(1, N)
            dn[tuple(dst)] = (-nu * neg * G)[tuple(src)]
        out += up + dn
    return out


def escape_energy_and_gradient(make, sigma_a, steps):
    """Run ``steps`` dense steps from a fresh problem ``make(sigma_a)`` and return
    (Q, dQ/dsigma_a) by reverse mode."""
    d = make(sigma_a)
    W = face_weights(d)
    c, a_r, dt = d.c, d.a_r, d.dt
    tape = []
    Q = 0.0
    for _ in range(steps):
        I0, T0 = d.I.copy(), d.T.copy()
        Istar = d.transport(I0)
        I1, T1, Td, Es = d.source(Istar)
        tape.append((Istar, T0, Td, Es, I1))
        d.I, d.T = I1, T1
        Q += float(np.sum(W * I1))
    k = c * dt * d.sigma_a
    s = 1.0 / (1.0 + k)
    gamma = k / ((1.0 + k) * d.cv)
    dO = d.dOmega
    gI = np.zeros_like(d.I)
    gT = np.zeros_like(d.T)
    gsig = np.zeros_like(d.sigma_a)
    for Istar, T0, Td, Es, I1 in reversed(tape):
        gI = gI + W
        # T' = T + (E* - E')/C_v
        gEs = gT / d.cv
        gE1 = -gT / d.cv
        gT0 = gT.copy()
        # E' = (1/c) sum I' dOmega
        gI = gI + (gE1 / c)[..., None, None] * dO
        # I' = s I* + e
        gs = np.sum(gI * Istar, axis=(-2, -1))
        ge = np.sum(gI, axis=(-2, -1))
        gIs = s[..., None, None] * gI
        # e = s k B, s = 1/(1+k), B = c a_r T+^4 / 4 pi
        B = c * a_r * Td ** 4 / (4 * np.pi)
        gB = ge * s * k
        gk = ge * s * s * B - gs * s * s
        gTd = gB * c * a_r * 4 * Td ** 3 / (4 * np.pi)
        # implicit: gamma a_r T+^4 + T+ = T + gamma E*
        fp = 4 * gamma * a_r * Td ** 3 + 1.0
        gT0 = gT0 + gTd / fp
        gEs = gEs + gTd * gamma / fp
        ggamma = gTd * (Es - a_r * Td ** 4) / fp
        gk = gk + ggamma / ((1.0 + k) ** 2 * d.cv)
        gsig += gk * c * dt
        # E* = (1/c) sum I* dOmega
        gIs = gIs + (gEs / c)[..., None, None] * dO
        gI = transport_T(d, gIs)
        gT = gT0
    return Q, gsig


def escape_energy(make, sigma_a, steps):
    d = make(sigma_a)
    W = face_weights(d)
    Q = 0.0
    for _ in range(steps):
        d.step()
        Q += float(np.sum(W * d.I))
    return Q
