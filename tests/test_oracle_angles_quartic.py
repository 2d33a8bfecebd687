"""Pins for the oracle's angular grid (Sec. 3) and quartic (Sec. 3.2)."""
import numpy as np
import pytest
from scipy.optimize import brentq

from oracle import angles
from oracle.quartic import t_dagger


@pytest.mark.parametrize("nt,npf", [(2, 4), (8, 16), (32, 64), (7, 5)])
def test_solid_angles_sum_to_4pi(nt, npf):
    g = angles.grid(nt, npf)
    assert abs(angles.solid_angles(g).sum() - 4 * np.pi) < 1e-13


@pytest.mark.parametrize("nt,npf", [(8, 16), (32, 64)])
def test_normals_unit_and_first_moment_zero(nt, npf):
    g = angles.grid(nt, npf)
    nx, ny, nz = angles.normals(g)
    assert np.allclose(nx ** 2 + ny ** 2 + nz ** 2, 1.0, atol=1e-15)
    dO = angles.solid_angles(g)
    for n in (nx, ny, nz):
        assert abs((n * dO).sum()) < 1e-13
    # mu is the cell centre of a uniform split of [-1, 1]
    assert np.allclose(np.diff(g["mu"]), 2.0 / nt)
    assert abs(g["mu"][0] + 1 - 1.0 / nt) < 1e-15


def test_quartic_matches_independent_root_finder():
    rng = np.random.default_rng(3)
    Tm = rng.uniform(0.01, 2.0, 40)
    E = rng.uniform(0.0, 3.0, 40)
    k = np.exp(rng.uniform(-5, 10, 40))
    cv = rng.uniform(0.5, 8.0, 40)
    a_r = 1.3
    T = t_dagger(Tm, E, k, cv, a_r)
    for i in range(40):
        g = k[i] / ((1 + k[i]) * cv[i])
        rhs = Tm[i] + g * E[i]
        ref = brentq(lambda t: g * a_r * t ** 4 + t - rhs, 0.0, rhs + 1.0, xtol=1e-300, rtol=1e-15, maxiter=500)
        assert abs(T[i] - ref) <= 8e-15 * ref
        # residual relative to the size of the terms
        assert abs(g * a_r * T[i] ** 4 + T[i] - rhs) <= 1e-14 * rhs


def test_quartic_special_cases():
    # no absorption: T-dagger = T^m
    assert t_dagger(0.7, 5.0, 0.0, 1.0, 1.0) == 0.7
    # no emission constant: linear, T = T^m + gamma E
    k, cv = 3.0, 2.0
    assert abs(t_dagger(0.5, 2.0, k, cv, 0.0) - (0.5 + k / ((1 + k) * cv) * 2.0)) < 1e-15
    # equilibrium: E = a_r T^4 gives T-dagger = T
    for T in (0.1, 1.0, 3.0):
        assert abs(t_dagger(T, 1.7 * T ** 4, 10.0, 1.0, 1.7) - T) < 2e-15 * T


def test_quartic_stiff_limit_reaches_equilibrium():
    # kappa -> infinity: C_v T + a_r T^4 = C_v T^m + E* (paper Sec. 5.2 with c_v = 8)
    T = float(t_dagger(2.0, 1.0, 1e12, 8.0, 1.0))
    assert abs(8 * T + T ** 4 - 17.0) < 1e-9


@pytest.mark.parametrize("nt,npf", [(2, 4), (8, 16), (5, 7)])
def test_isotropic_intensity_gives_E_equal_4pi_I_over_c(nt, npf):
    """Sec. 4.1's quadrature of an isotropic intensity: E = 4 pi I / c exactly
    (the weights sum to 4 pi), in the dense form and the grouped TT form."""
    from oracle import tt
    from oracle.dense import DenseSN

    c = 2.5
    I = np.array([0.3, 1.7, 4.0])
    n = (3,)
    d = DenseSN(n, [1.0], nt, npf, c, 1.0, 0.1, [0], np.ones(n), np.ones(n), np.ones(n),
                I[:, None, None] * np.ones((nt, npf)))
    assert np.allclose(d.energy_density(), 4 * np.pi * I / c, rtol=1e-14, atol=0)
    g = angles.grid(nt, npf)
    cores = [I.reshape(1, 3, 1), np.ones((1, nt, 1)), np.ones((1, npf, 1))]
    E = tt.energy_density_grouped(cores, g["w"], g["v"], c)
    assert np.allclose(E, 4 * np.pi * I / c, rtol=1e-14, atol=0)
