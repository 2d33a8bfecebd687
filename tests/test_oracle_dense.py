"""Pins for the dense S_N oracle (Sec. 3) against closed forms."""
import json
import math
import os

import numpy as np
import pytest
from scipy.integrate import solve_ivp
from scipy.optimize import brentq

from oracle import angles
from oracle.dense import PERIODIC, VACUUM, DenseSN

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _dense(n, nt, npf, dt, bc, sigma_a=0.0, a_r=1.0, T0=1.0, I0=None, cv=1.0, L=None):
    L = L or [1.0] * len(n)
    shape = tuple(n)
    if I0 is None:
        I0 = np.zeros(shape + (nt, npf))
    return DenseSN(n, L, nt, npf, 1.0, a_r, dt, [bc] * len(n),
                   np.full(shape, sigma_a), np.full(shape, cv), np.full(shape, T0), I0)


def test_vacuum_streaming_matches_multinomial_closed_form():
    # one ordinate with n_x, n_y > 0 from a point source: the donor-cell upwind
    # scheme is I^{m} = sum multinomial(m; a, b, m-a-b) al^a be^b (1-al-be)^(m-a-b) I^0
    n, nt, npf, dt = (24, 24), 4, 8, 0.5 / 24
    I0 = np.zeros((24, 24, nt, npf))
    g = angles.grid(nt, npf)
    nx, ny, _ = angles.normals(g)
    l, p = 2, 1  # mu > 0? any ordinate with nx, ny > 0
    assert nx[l, p] > 0 and ny[l, p] > 0
    i0, j0 = 3, 4
    I0[i0, j0, l, p] = 1.0
    d = _dense(n, nt, npf, dt, VACUUM, sigma_a=0.0, a_r=0.0, I0=I0)
    m = 9
    for _ in range(m):
        d.step(with_source=False)
    al = dt * 24 * nx[l, p]
    be = dt * 24 * ny[l, p]
    ref = np.zeros((24, 24))
    for a in range(m + 1):
        for b in range(m + 1 - a):
            coef = math.factorial(m) / (math.factorial(a) * math.factorial(b) * math.factorial(m - a - b))
            ref[i0 + a, j0 + b] = coef * al ** a * be ** b * (1 - al - be) ** (m - a - b)
    assert np.abs(d.I[:, :, l, p] - ref).max() < 1e-15
    # every other ordinate stays zero
    mask = np.ones((nt, npf), bool)
    mask[l, p] = False
    assert np.abs(d.I[:, :, mask]).max() == 0.0


def test_vacuum_streaming_negative_direction_and_z():
    # 3D: an ordinate with n_x < 0, n_z < 0 moves to lower indices
    n, nt, npf, dt = (10, 6, 10), 4, 8, 0.3 / 10
    g = angles.grid(nt, npf)
    nx, ny, nz = angles.normals(g)
    l, p = 0, 3
    assert nx[l, p] < 0 and nz[l, p] < 0
    I0 = np.zeros(n + (nt, npf))
    I0[7, 3, 8, l, p] = 1.0
    d = _dense(n, nt, npf, dt, VACUUM, a_r=0.0, I0=I0)
    d.step(with_source=False)
    nux, nuy, nuz = dt * 10, dt * 6, dt * 10  # c dt / dx per axis
    ax, ay, az = -nux * nx[l, p], nuy * abs(ny[l, p]), -nuz * nz[l, p]
    out = d.I[..., l, p]
    assert abs(out[7, 3, 8] - (1 - ax - ay - az)) < 1e-15
    assert abs(out[6, 3, 8] - ax) < 1e-15
    assert abs(out[7, 3, 7] - az) < 1e-15
    yj = 4 if ny[l, p] > 0 else 2
    assert abs(out[7, yj, 8] - ay) < 1e-15


@pytest.mark.parametrize("n", [(16,), (12, 10), (6, 5, 4)])
def test_periodic_transport_conserves_each_ordinate(n):
    rng = np.random.default_rng(1)
    nt, npf = 4, 8
    I0 = rng.uniform(0, 1, tuple(n) + (nt, npf))
    d = _dense(n, nt, npf, 0.4 / max(n), PERIODIC, a_r=0.0, I0=I0)
    for _ in range(5):
        d.step(with_source=False)
    axes = tuple(range(len(n)))
    assert np.allclose(d.I.sum(axis=axes), I0.sum(axis=axes), rtol=1e-13, atol=0)


def test_periodic_streaming_moves_each_centroid_by_c_dt_n():
    """Donor-cell upwinding moves the first moment of every ordinate by
    exactly c dt n per step, and keeps its mass, while the support stays clear
    of the periodic seam: sum_i x_i I_{i-1} = sum_j (x_j + dx) I_j.  Catches
    a swapped axis, direction cosine or sign."""
    n, nt, npf = (40, 36), 4, 8
    rng = np.random.default_rng(5)
    I0 = np.zeros(n + (nt, npf))
    I0[17:23, 15:21] = rng.uniform(0.5, 1.5, (6, 6, nt, npf))
    dt = 0.01
    d = _dense(n, nt, npf, dt, PERIODIC, a_r=0.0, I0=I0)
    g = angles.grid(nt, npf)
    nx, ny = angles.normals(g)[:2]
    X, Y = np.meshgrid((np.arange(n[0]) + 0.5) / n[0], (np.arange(n[1]) + 0.5) / n[1], indexing="ij")

    def centroid(I):
        m = I.sum(axis=(0, 1))
        return m, np.einsum("ij,ijlp->lp", X, I) / m, np.einsum("ij,ijlp->lp", Y, I) / m

    m0, cx0, cy0 = centroid(I0)
    steps = 6
    for _ in range(steps):
        d.step(with_source=False)
    m1, cx1, cy1 = centroid(d.I)
    assert np.abs(m1 - m0).max() <= 1e-13 * m0.max()
    assert np.abs(cx1 - cx0 - steps * dt * nx).max() <= 1e-13
    assert np.abs(cy1 - cy0 - steps * dt * ny).max() <= 1e-13


def test_pure_absorption_decay_closed_form():
    # a_r = 0, uniform isotropic intensity, periodic: I^m = I^0 (1 + c dt sigma)^-m
    n, nt, npf = (8, 8), 4, 8
    sigma, dt, m = 3.0, 0.01, 20
    I0 = np.full(n + (nt, npf), 0.7)
    d = _dense(n, nt, npf, dt, PERIODIC, sigma_a=sigma, a_r=0.0, I0=I0, T0=0.5)
    for _ in range(m):
        d.step()
    ref = 0.7 * (1 + dt * sigma) ** (-m)
    assert np.abs(d.I - ref).max() < 1e-14
    # and the continuum limit exp(-c sigma t) is approached at first order in dt
    assert abs(ref - 0.7 * math.exp(-sigma * dt * m)) < 0.7 * sigma ** 2 * dt * (dt * m)


def test_equilibrium_is_a_fixed_point():
    n, nt, npf = (6, 5), 4, 6
    T = 0.8
    a_r, c = 1.0, 1.0
    I0 = np.full(n + (nt, npf), c * a_r * T ** 4 / (4 * np.pi))
    for bc in (PERIODIC,):
        d = _dense(n, nt, npf, 0.05, bc, sigma_a=7.0, a_r=a_r, I0=I0, T0=T)
        for _ in range(3):
            d.step()
        assert np.abs(d.I - I0).max() < 1e-15
        assert np.abs(d.T - T).max() < 1e-15


def test_dense_temperature_equals_t_dagger():
    # untruncated: the energy-conserving update reproduces T-dagger exactly
    rng = np.random.default_rng(5)
    n, nt, npf = (7, 6), 4, 8
    I0 = rng.uniform(0.0, 0.2, n + (nt, npf))
    d = DenseSN(n, [1, 1], nt, npf, 1.0, 1.0, 0.03, [VACUUM, PERIODIC],
                rng.uniform(0.1, 50, n), rng.uniform(0.5, 2, n), rng.uniform(0.2, 1, n), I0)
    Istar = d.transport(d.I)
    _, T_new, Td, _ = d.source(Istar)
    assert np.abs(T_new - Td).max() < 1e-14


def _relax_params():
    with open(os.path.join(GOLDEN, "thermal_relaxation.json")) as f:
        return json.load(f)


def test_thermal_relaxation_stiff_reaches_equilibrium_in_one_step():
    p = _relax_params()
    cv = p["rho"] * p["c_v"]
    T_eq = brentq(lambda t: cv * t + p["a_r"] * t ** 4 - (cv * p["T"] + p["a_r"] * p["T_r"] ** 4), 0, 10, xtol=1e-15)
    dt = p["t_lim"] / p["n_steps"]
    nt, npf = 4, 8
    I0 = np.full((p["n_cells"], nt, npf), p["c"] * p["a_r"] * p["T_r"] ** 4 / (4 * np.pi))
    d = DenseSN((p["n_cells"],), [p["n_cells"] * p["dx"]], nt, npf, p["c"], p["a_r"], dt, [PERIODIC],
                np.full(4, p["rho"] * p["kappa_a"][1]), np.full(4, cv), np.full(4, p["T"]), I0)
    d.step()
    # stiff (kappa = 1e6, c dt kappa = 1e4): one step lands at T_eq up to O(1/k)
    assert np.abs(d.T - T_eq).max() < 1e-3
    assert abs(T_eq - 1.4970877) < 1e-6
    E = d.energy_density()
    assert np.abs(E - p["a_r"] * T_eq ** 4).max() < 1e-2


def test_thermal_relaxation_translucent_follows_ode():
    p = _relax_params()
    cv = p["rho"] * p["c_v"]
    sig = p["rho"] * p["kappa_a"][0]
    dt = p["t_lim"] / p["n_steps"]
    nt, npf = 2, 4
    I0 = np.full((4, nt, npf), p["c"] * p["a_r"] * p["T_r"] ** 4 / (4 * np.pi))
    d = DenseSN((4,), [4.0], nt, npf, p["c"], p["a_r"], dt, [PERIODIC],
                np.full(4, sig), np.full(4, cv), np.full(4, p["T"]), I0)
    e0 = d.total_energy()
    for _ in range(p["n_steps"]):
        d.step()
    assert abs(d.total_energy() - e0) < 1e-13 * e0

    def rhs(t, y):
        T, E = y
        q = p["c"] * sig * (p["a_r"] * T ** 4 - E)
        return [-q / cv, q]

    sol = solve_ivp(rhs, (0, p["t_lim"]), [p["T"], p["a_r"] * p["T_r"] ** 4], rtol=1e-11, atol=1e-12)
    T_ode = sol.y[0, -1]
    # backward Euler is first order: error ~ dt * |dT/dt| ~ 1e-2 * O(0.1)
    assert abs(d.T[0] - T_ode) < 5e-3
    # isotropic and uniform: transport does nothing, every cell is identical
    assert np.ptp(d.T) == 0.0
