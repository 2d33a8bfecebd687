"""Pins for the Rusanov and HLL interface fluxes (Sec. 3.1, Sec. 4.3) in the
oracle: the dense definitions against their limits and invariants, and the
grouped TT stepper (every flux as 1 + 2 ndim rank-one-angular terms with
face-weighted stencils) against the dense stepper."""
import numpy as np
import pytest

import workloads
from oracle import tt
from oracle.dense import DenseSN
from oracle.ttstep import PERIODIC, VACUUM, TTSN


def _fields(n, seed, thick=False):
    f = workloads.random_fields(n, seed)
    if thick:
        # opacities spanning thin and thick cells so that both branches of the
        # HLL wave speeds (tau below and above the threshold) occur
        rng = np.random.default_rng(seed + 7)
        f["sigma_a"] = 10.0 ** rng.uniform(-2, 3, n)
    return f


def _pair(n, nt, npf, bc, seed, flux, **fk):
    nc = int(np.prod(n))
    cores = workloads.random_positive_tt([nc, nt, npf], [3, 2], seed)
    f = _fields(n, seed + 100, thick=(flux in ("hll", "rusanov_tau")))
    sigma_s = 0.5 * f["sigma_a"]
    dt = 0.3 * min(1.0 / m for m in n)
    args = dict(n=n, L=[1.0] * len(n), n_theta=nt, n_phi=npf, c=1.0, a_r=1.0, dt=dt,
                bc=[bc] * len(n), sigma_a=f["sigma_a"], cv=f["cv"], T0=f["T0"], sigma_s=sigma_s,
                flux=flux, **fk)
    ttsn = TTSN(cores=cores, rounding=None, **args)
    d = DenseSN(I0=tt.full(cores).reshape(tuple(n) + (nt, npf)), **args)
    return ttsn, d


FLUXES = [("rusanov", dict(rusanov_s=1.0)), ("rusanov", dict(rusanov_s=0.3)), ("rusanov", dict(rusanov_s=0.0)),
          ("hll", dict(hll_beta=1.0, hll_tau_threshold=1.0)), ("hll", dict(hll_beta=5.0, hll_tau_threshold=0.5)),
          ("rusanov_tau", dict(hll_beta=1.0)), ("rusanov_tau", dict(hll_beta=20.0))]


@pytest.mark.parametrize("n,bc", [((12,), VACUUM), ((8, 6), PERIODIC), ((8, 6), VACUUM),
                                  ((5, 4, 3), VACUUM)])
@pytest.mark.parametrize("flux,fk", FLUXES)
def test_untruncated_tt_step_equals_dense_step_all_fluxes(n, bc, flux, fk):
    ttsn, d = _pair(n, 4, 6, bc, seed=17, flux=flux, **fk)
    for _ in range(2):
        ttsn.step()
        d.step()
    F = ttsn.full()
    assert np.abs(F - d.I).max() <= 1e-12 * np.abs(d.I).max()
    assert np.abs(ttsn.T - d.T.reshape(-1)).max() <= 1e-12 * np.abs(d.T).max()
    k = 1 + 2 * len(n)
    assert tt.ranks(ttsn.cores)[0] == k * (k * 3 + 1) + 1


def _dense(n, flux, bc=VACUUM, sigma=1.0, **fk):
    nc = int(np.prod(n))
    I0 = workloads.random_positive_tt([nc, 4, 8], [2, 2], 3)
    return DenseSN(n, [1.0] * len(n), 4, 8, 1.0, 1.0, 0.2 / max(n), [bc] * len(n),
                   np.full(n, sigma), np.ones(n), np.ones(n), tt.full(I0).reshape(tuple(n) + (4, 8)),
                   flux=flux, **fk)


def test_hll_without_opacity_is_upwind():
    """tau -> 0 (no opacity): the HLL flux reduces to upwinding (Sec. 3.1)."""
    for bc in (VACUUM, PERIODIC):
        up = _dense((9, 7), "upwind", bc, sigma=0.0)
        hl = _dense((9, 7), "hll", bc, sigma=0.0)
        a, b = up.transport(up.I), hl.transport(hl.I)
        assert np.abs(a - b).max() <= 1e-15 * np.abs(a).max()


def test_hll_thick_limit_is_rusanov_with_speed_c_n_over_tau():
    """tau -> infinity: HLL equals the Rusanov flux with S+ = c |n_x| / tau_c
    (the series expansion stated after Eq. hll); exact once exp(-tau^2)
    underflows."""
    d = _dense((10,), "hll", VACUUM, sigma=1.0)
    tau = np.array([40.0, 55.0, 1e3])
    n = np.array([[0.3, -0.7, 0.9, -0.05]])
    S_R, S_L = d._hll_speeds(n, tau)
    UL, UR = 1.3, 0.4
    FL, FR = d.c * n * UL, d.c * n * UR
    F = (S_R * FL - S_L * FR + S_L * S_R * (UR - UL)) / (S_R - S_L)
    Splus = d.c * np.abs(n) / tau[:, None, None]
    rus = 0.5 * (FL + FR) - 0.5 * Splus * (UR - UL)
    assert np.abs(F - rus).max() <= 1e-15


def test_rusanov_with_unit_speed_is_upwind_for_unit_normals():
    """S+ = c and |n_x| = 1: Eq. rusanov_flux_toro gives F_L for n = 1 and F_R
    for n = -1, i.e. upwinding."""
    up = _dense((11,), "upwind", VACUUM)
    ru = _dense((11,), "rusanov", VACUUM, rusanov_s=1.0)
    sign = np.where(np.arange(8) < 4, 1.0, -1.0)
    for d in (up, ru):
        d.nvec = [np.broadcast_to(sign, (4, 8)).copy()]
    a, b = up.transport(up.I), ru.transport(ru.I)
    assert np.abs(a - b).max() <= 1e-15 * np.abs(a).max()


@pytest.mark.parametrize("flux,fk", FLUXES)
def test_periodic_transport_conserves_each_ordinate(flux, fk):
    """Fluxes telescope on a periodic grid: sum_i I_ilp is unchanged."""
    d = _dense((7, 6), flux, PERIODIC, sigma=2.0, **fk)
    d.sigma_a = 10.0 ** np.random.default_rng(2).uniform(-2, 2, (7, 6))
    out = d.transport(d.I)
    assert np.abs(out.sum(axis=(0, 1)) - d.I.sum(axis=(0, 1))).max() <= 1e-13 * np.abs(d.I).sum()


def test_rusanov_zero_speed_is_the_central_difference():
    """S+ = 0: the flux is the average of F_L and F_R, a central difference."""
    d = _dense((9,), "rusanov", PERIODIC, rusanov_s=0.0)
    out = d.transport(d.I)
    nu = d.c * d.dt / d.dx[0]
    ref = d.I - 0.5 * nu * d.nvec[0] * (np.roll(d.I, -1, axis=0) - np.roll(d.I, 1, axis=0))
    assert np.abs(out - ref).max() <= 1e-14 * np.abs(d.I).max()


@pytest.mark.parametrize("flux,fk", FLUXES[::2])
def test_energy_conserved_with_truncation_all_fluxes(flux, fk):
    n, nt, npf = (8, 7), 4, 8
    f = _fields(n, 33, thick=True)
    I0 = f["T0"] ** 4 / (4 * np.pi)
    t = TTSN(n, [1.0, 1.0], nt, npf, 1.0, 1.0, 0.04, [PERIODIC] * 2, f["sigma_a"].reshape(-1),
             f["cv"].reshape(-1), f["T0"].reshape(-1), TTSN.isotropic_cores(I0.reshape(-1), nt, npf),
             eps=1e-4, flux=flux, **fk)
    e0 = t.total_energy()
    for _ in range(4):
        t.step()
        assert abs(t.total_energy() - e0) <= 1e-13 * e0


def _gauss_E(p, t):
    """The analytic E(t, x, y) of the Gaussian-diffusion test (Sec. 5)."""
    xc = workloads.cell_centres(p["n"], p["L"])
    r2 = sum((x - c0) ** 2 for x, c0 in zip(xc, p["centre"]))
    s = 4.0 * p["D"] * (p["t0"] + t)
    return p["amp"] / (np.pi * s) * np.exp(-r2 / s)


def test_gaussian_diffusion_dense_follows_the_analytic_solution():
    """Pure isotropic scattering (rho kappa_s = 1e3) with the Rusanov flux at
    S+ = 0 diffuses a Gaussian pulse as E = A / (4 pi D (t0 + t))
    exp(-r^2 / (4 D (t0 + t))), D = c / (3 rho kappa_s) (Sec. 5).  On 32^2
    cells after 200 steps the stepper stays within 1e-2 of it while the
    solution itself moves by 5e-2 (a wrong diffusion coefficient, sign or
    scattering term would not)."""
    p = workloads.gaussian_diffusion(n=(32, 32))
    I0 = (p["c"] * p["a_r"] * p["Tr0"] ** 4 / (4 * np.pi))[..., None, None] * np.ones((p["n_theta"], p["n_phi"]))
    d = DenseSN(p["n"], p["L"], p["n_theta"], p["n_phi"], p["c"], p["a_r"], p["dt"], p["bc"], p["sigma_a"],
                p["cv"], p["T0"], I0, sigma_s=p["sigma_s"], flux="rusanov", rusanov_s=0.0)
    steps = 200
    for _ in range(steps):
        d.step()
    Ea, E0 = _gauss_E(p, steps * p["dt"]), _gauss_E(p, 0.0)
    err = np.linalg.norm(d.energy_density() - Ea) / np.linalg.norm(Ea)
    moved = np.linalg.norm(E0 - Ea) / np.linalg.norm(Ea)
    assert err <= 1e-2 and err <= 0.2 * moved, (err, moved)


def _hand_hll_face(n, tau, UL, UR, c=1.0, thr=1.0):
    """One face's HLL flux written out from Sec. 3.1's four-case table (wave
    speeds after Eq. hll), small-tau rows only (tau < thr):
    n >= 0: S_R = c n sqrt(1 - tau^2/2), S_L = -c n tau;
    n < 0:  S_R = -c n tau,              S_L = c n sqrt(1 - tau^2/2);
    then Eq. hll, F = (S_R F_L - S_L F_R + S_L S_R (U_R - U_L)) / (S_R - S_L)."""
    assert 0.0 < tau < thr
    if n >= 0.0:
        S_R, S_L = c * n * (1.0 - tau * tau / 2.0) ** 0.5, -c * n * tau
    else:
        S_R, S_L = -c * n * tau, c * n * (1.0 - tau * tau / 2.0) ** 0.5
    FL, FR = c * n * UL, c * n * UR
    return (S_R * FL - S_L * FR + S_L * S_R * (UR - UL)) / (S_R - S_L)


@pytest.mark.parametrize("beta,sigma", [(1.0, 3.0), (0.7, 5.0), (2.0, 0.25)])
def test_hll_small_tau_branch_against_the_table_by_hand(beta, sigma):
    """The small-tau rows of the wave-speed table (0 < tau_c < tau_threshold),
    which neither limit pins: a 1D row of 6 cells with uniform opacity has
    tau_c = beta sigma dx on every face (Eq. tauc, harmonic mean of equal
    values; the vacuum faces take the boundary cell's own opacity), and the
    dense transport must equal I_i - (dt/dx)(F_{i+1/2} - F_{i-1/2}) with each
    face's flux computed here by hand from the table, for ordinates of both
    signs (vacuum ghosts hold zero)."""
    N, L = 6, 1.0
    dx = L / N
    tau = beta * sigma * dx
    assert 0.0 < tau < 1.0
    rng = np.random.default_rng(3)
    normals = np.array([0.83, 0.21, -0.47, -0.95])
    I0 = rng.uniform(0.5, 2.0, (N, 1, 4))
    d = DenseSN((N,), [L], 1, 4, 1.0, 1.0, 0.3 * dx, [VACUUM], np.full(N, sigma), np.ones(N), np.ones(N), I0,
                flux="hll", hll_beta=beta, hll_tau_threshold=1.0)
    d.nvec = [normals.reshape(1, 4).copy()]
    out = d.transport(d.I)
    nu = d.dt / dx
    for p, n in enumerate(normals):
        U = np.concatenate([[0.0], I0[:, 0, p], [0.0]])  # ghost, cells, ghost
        F = [_hand_hll_face(n, tau, U[k], U[k + 1]) for k in range(N + 1)]
        want = [U[i + 1] - nu * (F[i + 1] - F[i]) for i in range(N)]
        assert np.abs(out[:, 0, p] - np.array(want)).max() <= 1e-14


def test_hll_small_tau_series_leaves_upwinding_at_third_order():
    """Series identity of the small-tau branch: with S_R = c n a, S_L = -c n b
    (n > 0) Eq. hll reduces to F = c n [U_L + b (1 - a)/(a + b) (U_R - U_L)];
    the table's a = sqrt(1 - tau^2/2), b = tau make the departure from
    upwinding (F - c n U_L) / (c n (U_R - U_L)) = tau^3/4 + O(tau^4), and the
    mirrored n < 0 case departs from c n U_R by -tau^3/4.  A wrong coefficient
    in either speed changes the tau^3 coefficient (b = tau/2 gives 1/8,
    sqrt(1 - tau^2) gives 1/2)."""
    d = _dense((10,), "hll", VACUUM, sigma=1.0)
    UL, UR = 1.7, 0.6
    for n in (0.4, -0.9):
        coef = []
        for tau in (2e-2, 1e-2, 5e-3):
            S_R, S_L = d._hll_speeds(np.array([[n]]), np.array([tau]))
            S_R, S_L = float(S_R.ravel()[0]), float(S_L.ravel()[0])
            FL, FR = d.c * n * UL, d.c * n * UR
            F = (S_R * FL - S_L * FR + S_L * S_R * (UR - UL)) / (S_R - S_L)
            up = FL if n >= 0 else FR
            coef.append((F - up) / (d.c * n * (UR - UL)) / tau ** 3)
        want = 0.25 if n > 0 else -0.25
        # O(tau) corrections shrink with tau
        assert abs(coef[-1] - want) < 2e-3 and abs(coef[-1] - want) < abs(coef[0] - want)


def test_rusanov_tau_on_thin_faces_is_upwind():
    """tau_c <= 1 on every face (here no opacity): S+ = c |n_x| and Eq.
    rusanov_flux_toro gives F_L for n_x > 0 and F_R for n_x < 0, upwinding."""
    for bc in (VACUUM, PERIODIC):
        up = _dense((9, 7), "upwind", bc, sigma=0.0)
        rt = _dense((9, 7), "rusanov_tau", bc, sigma=0.0)
        a, b = up.transport(up.I), rt.transport(rt.I)
        assert np.abs(a - b).max() <= 1e-15 * np.abs(a).max()


def test_rusanov_tau_on_thick_faces_is_the_hll_thick_limit():
    """tau_c >> 1 on every face: S+ = c |n_x| / tau_c is the speed of the
    series expansion of the HLL flux stated after Eq. hll, so the whole
    transport step equals the (independently pinned) HLL step once
    exp(-tau^2) underflows."""
    for n in ((10,), (6, 5)):
        hl = _dense(n, "hll", VACUUM, sigma=400.0, hll_beta=1.0, hll_tau_threshold=1.0)
        rt = _dense(n, "rusanov_tau", VACUUM, sigma=400.0, hll_beta=1.0)
        assert hl._face_tau(0).min() > 30.0
        a, b = hl.transport(hl.I), rt.transport(rt.I)
        assert np.abs(a - b).max() <= 1e-14 * np.abs(a).max()


def test_rusanov_tau_matches_uniform_rusanov_for_unit_normals():
    """Uniform tau_c = 3 and |n_x| = 1: the speed is c / 3 on every face, the
    Rusanov flux of Eq. rusanov_flux_toro with S+ = c / 3."""
    # dx = 1/12, beta = 1: tau = 2 dx / (2 / sigma) = dx sigma = 3 for sigma = 36
    rt = _dense((12,), "rusanov_tau", PERIODIC, sigma=36.0, hll_beta=1.0)
    ru = _dense((12,), "rusanov", PERIODIC, sigma=36.0, rusanov_s=1.0 / 3.0)
    assert np.allclose(rt._face_tau(0), 3.0, rtol=1e-14)
    sign = np.where(np.arange(8) < 4, 1.0, -1.0)
    for d in (rt, ru):
        d.nvec = [np.broadcast_to(sign, (4, 8)).copy()]
    a, b = rt.transport(rt.I), ru.transport(ru.I)
    assert np.abs(a - b).max() <= 1e-14 * np.abs(a).max()
