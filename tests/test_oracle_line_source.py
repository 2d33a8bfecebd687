"""Pins for the line source of Sec. 5.4: the oracle's analytic solution
(Green's function of the planar pulse convolved with the Gaussian) against
invariants, limits and a brute-force 2D convolution, and the dense stepper
against it."""
import numpy as np
import pytest

import workloads
from oracle.analytic import line_source_E, line_source_green
from oracle.dense import DenseSN


@pytest.mark.parametrize("t,omega", [(0.25, 0.03), (0.5, 0.03), (1.0, 0.03), (0.5, 0.1)])
def test_line_source_energy_is_U0(t, omega):
    """The Green's function carries unit energy (int_0^ct 2 pi r dr / (2 pi ct
    sqrt((ct)^2 - r^2)) = 1), so the convolution keeps the pulse's U0:
    2 pi int rho E(t, rho) d rho = U0."""
    x, w = np.polynomial.legendre.leggauss(32)
    edges = np.linspace(0.0, t + 14 * omega, 401)
    half = 0.5 * np.diff(edges)
    rho = (half[:, None] * (x + 1) + edges[:-1, None]).ravel()
    wr = (half[:, None] * w).ravel()
    U0 = 0.7
    tot = 2 * np.pi * np.sum(wr * rho * line_source_E(t, rho, omega, U0=U0))
    assert abs(tot - U0) <= 1e-9 * U0, tot


def test_line_source_at_t0_is_the_initial_gaussian():
    rho = np.linspace(0, 0.2, 9)
    g = 1.0 / (2 * np.pi * 0.03 ** 2) * np.exp(-rho ** 2 / (2 * 0.03 ** 2))
    for t in (0.0, 1e-9):
        assert np.abs(line_source_E(t, rho, 0.03) - g).max() <= 1e-12 * g.max()


def test_line_source_equals_brute_force_2d_convolution():
    """Independent route: integrate the Green's function against the plain
    2D Gaussian over the disc of radius ct in polar coordinates (r = ct sin a,
    psi), with no angular reduction to the Bessel function I_0."""
    t, om = 0.5, 0.08
    a, wa = np.polynomial.legendre.leggauss(400)
    a = 0.25 * np.pi * (a + 1)
    wa = 0.25 * np.pi * wa
    npsi = 720
    psi = (np.arange(npsi) + 0.5) * 2 * np.pi / npsi
    for rho in (0.0, 0.2, 0.47, 0.5, 0.53, 0.7):
        r = t * np.sin(a)[:, None]
        d2 = rho ** 2 + r ** 2 - 2 * rho * r * np.cos(psi)[None]
        G = np.exp(-d2 / (2 * om ** 2)) / (2 * np.pi * om ** 2)
        brute = np.sum((np.sin(a) * wa)[:, None] * G) / npsi
        got = line_source_E(t, rho, om)
        assert abs(got - brute) <= 1e-10 * max(brute, 1e-3), (rho, got, brute)


def test_line_source_narrow_pulse_tends_to_the_greens_function():
    """omega -> 0 away from the front: E -> U0 / (2 pi ct sqrt((ct)^2 -
    rho^2)), with an O(omega^2) correction."""
    rho = np.array([0.0, 0.3, 0.5, 0.7])
    green = line_source_green(1.0, rho)
    dev = [np.abs(line_source_E(1.0, rho, om) / green - 1).max() for om in (4e-3, 1e-3)]
    assert dev[0] <= 1e-4 and dev[1] <= 1e-5, dev
    assert 14 <= dev[0] / dev[1] <= 18, dev
    assert line_source_green(1.0, np.array([1.2]))[0] == 0.0


def _dense_line_source(m, nt, npf, omega=0.1, t=0.5):
    p = workloads.line_source(n=(m, m), n_theta=nt, n_phi=npf, omega=omega)
    E0 = p["Tr0"] ** 4
    I0 = (p["c"] * E0 / (4 * np.pi))[..., None, None] * np.ones((nt, npf))
    d = DenseSN(p["n"], p["L"], nt, npf, p["c"], p["a_r"], p["dt"], p["bc"], p["sigma_a"], p["cv"], p["T0"], I0)
    steps = int(round(t / p["dt"]))
    for _ in range(steps):
        d.step()
    E = d.energy_density()
    Ea = line_source_E(steps * p["dt"], p["radius"], omega)
    dV = float(np.prod([p["L"][a] / m for a in range(2)]))
    return np.abs(E - Ea).sum() / np.abs(Ea).sum(), E.sum() * dV, E0.sum() * dV


def test_line_source_dense_error_falls_with_ordinates_and_cells():
    """Sec. 5.4's line source on [-1.1, 1.1]^2 (pulse width 0.1, t = 0.5,
    CFL 0.4): the dense stepper's relative L1 error in E against the analytic
    solution falls as the ordinates are refined (ray effects: 2x4 -> 8x16)
    and as the cells are refined (spatial error of the upwind scheme:
    32^2 -> 64^2), and no energy leaves the domain before the front arrives."""
    e_coarse_ang, _, _ = _dense_line_source(64, 2, 4)
    e_64, tot, tot0 = _dense_line_source(64, 8, 16)
    e_32, _, _ = _dense_line_source(32, 8, 16)
    assert e_coarse_ang > 3 * e_64, (e_coarse_ang, e_64)
    assert e_32 > 1.4 * e_64, (e_32, e_64)
    assert e_64 < 0.2
    assert abs(tot - tot0) <= 1e-5 * tot0
