"""Pins for the oracle's escape-energy gradient: central finite differences of
the dense scheme, the transpose identity of the transport operator, and the
objective's closed form for free streaming of one ordinate."""
import numpy as np
import pytest

from oracle import angles
from oracle.adjoint import escape_energy, escape_energy_and_gradient, face_weights, transport_T
from oracle.dense import PERIODIC, VACUUM, DenseSN


def _maker(n, nt, npf, bc, seed):
    rng = np.random.default_rng(seed)
    T0 = rng.uniform(0.3, 1.0, n)
    I0 = np.broadcast_to((rng.uniform(0.1, 0.5, n))[..., None, None], tuple(n) + (nt, npf)).copy()
    cv = rng.uniform(0.5, 2.0, n)
    dt = 0.4 / max(n)

    def make(sig):
        return DenseSN(n, [1.0] * len(n), nt, npf, 1.0, 1.0, dt, [bc] * len(n), sig, cv, T0, I0)
    return make, rng


@pytest.mark.parametrize("n,bc", [((7, 6), VACUUM), ((5, 4, 3), VACUUM), ((6, 5), PERIODIC)])
def test_transport_transpose_identity(n, bc):
    make, rng = _maker(n, 4, 8, bc, 1)
    d = make(np.ones(n))
    X = rng.standard_normal(tuple(n) + (4, 8))
    Y = rng.standard_normal(tuple(n) + (4, 8))
    assert abs(np.sum(Y * d.transport(X)) - np.sum(transport_T(d, Y) * X)) < 1e-12 * np.abs(X).sum()


@pytest.mark.parametrize("n", [(8, 7), (5, 4, 3)])
def test_gradient_matches_central_differences(n):
    make, rng = _maker(n, 4, 8, VACUUM, 2)
    sig = np.exp(rng.uniform(-1, 2, n))
    Q, g = escape_energy_and_gradient(make, sig, 4)
    assert abs(Q - escape_energy(make, sig, 4)) <= 1e-14 * abs(Q)
    cells = [tuple(rng.integers(0, m) for m in n) for _ in range(6)]
    for c in cells:
        h = 1e-6 * sig[c]
        sp, sm = sig.copy(), sig.copy()
        sp[c] += h
        sm[c] -= h
        fd = (escape_energy(make, sp, 4) - escape_energy(make, sm, 4)) / (2 * h)
        assert abs(fd - g[c]) <= 1e-6 * np.abs(g).max() + 1e-7 * abs(fd)


def test_escape_energy_of_free_streaming_closed_form():
    # sigma = 0, a_r = 0: one beam of one ordinate leaves through the high-x face
    # after walking; Q equals sum_m dt dA n_x I^m at the last cell (here the beam
    # sits in the last cell from the start, I^m = (1 - nu n_x)^m I^0 there).
    n, nt, npf = (4, 3), 2, 4
    g = angles.grid(nt, npf)
    nx, ny, _ = angles.normals(g)
    l, p = 1, 0  # mu > 0 and phi in (0, pi/2): n_x, n_y > 0
    dt = 0.1
    I0 = np.zeros(n + (nt, npf))
    I0[3, 2, l, p] = 1.0
    d = DenseSN(n, [1.0, 1.0], nt, npf, 1.0, 0.0, dt, [VACUUM, VACUUM], np.zeros(n), np.ones(n), np.ones(n), I0)
    W = face_weights(d)
    Q = 0.0
    for _ in range(3):
        d.step()
        Q += float(np.sum(W * d.I))
    # the corner cell (3,2) touches the high-x and high-y faces
    ax, ay = dt * 4 * nx[l, p], dt * 3 * ny[l, p]
    stay = 1 - ax - ay
    dO = 4 * np.pi / (nt * npf)
    ref = sum(stay ** m * dt * dO * ((1 / 3) * nx[l, p] + (1 / 4) * ny[l, p]) for m in range(1, 4))
    assert abs(Q - ref) <= 1e-15
