"""Rusanov and HLL interface fluxes (Sec. 3.1) on the GPU: the untruncated
step against the dense definitions (grouped and split layouts), rounded steps
against the oracle's TT stepper at its ranks, conservation, the precision
form, and the argument errors of the flux parameters."""
import ctypes

import numpy as np
import pytest
import torch

import workloads
from oracle import tt
from oracle.dense import DenseSN
from oracle.split import SplitTTSN
from oracle.ttstep import PERIODIC, VACUUM, TTSN as OracleTTSN

pytestmark = pytest.mark.gpu

FLUXES = [("rusanov", dict(rusanov_s=1.0)), ("rusanov", dict(rusanov_s=0.3)), ("rusanov", dict(rusanov_s=0.0)),
          ("hll", dict(hll_beta=1.0, hll_tau_threshold=1.0)), ("hll", dict(hll_beta=5.0, hll_tau_threshold=0.5)),
          ("rusanov_tau", dict(hll_beta=1.0)), ("rusanov_tau", dict(hll_beta=20.0))]


@pytest.fixture(scope="module")
def ttsn():
    assert torch.cuda.is_available()
    import paper_2503_18056_gb300 as m

    return m


def _args(n, nt, npf, bc, seed, uniform=False):
    f = workloads.random_fields(n, seed)
    rng = np.random.default_rng(seed + 7)
    sig = np.full(n, 3.0) if uniform else 10.0 ** rng.uniform(-2, 3, n)  # thin and thick cells
    return dict(n=n, L=[1.0] * len(n), n_theta=nt, n_phi=npf, c=1.0, a_r=1.0,
                dt=0.3 * min(1.0 / m for m in n), bc=[bc] * len(n), sigma_a=sig.reshape(-1),
                sigma_s=(0.5 * sig).reshape(-1), cv=f["cv"].reshape(-1), T0=f["T0"].reshape(-1))


def _dense(a, n, nt, npf, cores_full, flux, fk):
    return DenseSN(n, a["L"], nt, npf, a["c"], a["a_r"], a["dt"], a["bc"], a["sigma_a"].reshape(n),
                   a["cv"].reshape(n), a["T0"].reshape(n), cores_full, sigma_s=a["sigma_s"].reshape(n),
                   flux=flux, **fk)


@pytest.mark.parametrize("n,bc", [((13,), VACUUM), ((9, 7), PERIODIC), ((9, 7), VACUUM), ((6, 5, 4), VACUUM)])
@pytest.mark.parametrize("flux,fk", FLUXES)
def test_untruncated_step_equals_dense_all_fluxes(ttsn, n, bc, flux, fk):
    nt, npf = 4, 6
    a = _args(n, nt, npf, bc, 21)
    nc = int(np.prod(n))
    cores = workloads.random_positive_tt([nc, nt, npf], [3, 2], seed=22)
    d = _dense(a, n, nt, npf, tt.full(cores).reshape(tuple(n) + (nt, npf)), flux, fk)
    g = ttsn.TTSN(eps=0.0, flux=flux, **fk, **a)
    g.set_cores(cores)
    for _ in range(2):
        d.step()
        g.step(flags=ttsn.TT_STEP_NO_ROUND)
    F = g.full().cpu().numpy()
    assert np.abs(F - d.I).max() <= 1e-12 * np.abs(d.I).max()
    _, T, _ = g.energy()
    assert np.abs(T.cpu().numpy() - d.T.reshape(-1)).max() <= 1e-12 * np.abs(d.T).max()


@pytest.mark.parametrize("n,bc", [((9, 7), PERIODIC), ((6, 5, 4), VACUUM)])
@pytest.mark.parametrize("flux,fk", FLUXES[::2])
def test_untruncated_split_step_equals_dense_all_fluxes(ttsn, n, bc, flux, fk):
    nt, npf = 4, 6
    a = _args(n, nt, npf, bc, 23, uniform=True)
    cores = workloads.random_positive_tt(list(n) + [nt, npf], [3, 2, 2, 3][: len(n) + 1], seed=24)
    d = _dense(a, n, nt, npf, tt.full(cores), flux, fk)
    g = ttsn.TTSN(eps=0.0, flux=flux, layout=ttsn.TT_LAYOUT_SPLIT, **fk, **a)
    g.set_cores(cores)
    for _ in range(2):
        d.step()
        g.step(flags=ttsn.TT_STEP_NO_ROUND)
    F = g.full().cpu().numpy()
    assert np.abs(F - d.I).max() <= 1e-12 * np.abs(d.I).max()


@pytest.mark.parametrize("flux,fk", FLUXES[::2])
@pytest.mark.parametrize("bc", [PERIODIC, VACUUM])
def test_rounded_steps_match_oracle_at_its_ranks(ttsn, flux, fk, bc):
    n, nt, npf = (16, 12), 4, 8
    a = _args(n, nt, npf, bc, 25)
    I0 = a["c"] * a["a_r"] * a["T0"] ** 4 / (4 * np.pi)
    ref = OracleTTSN(n, a["L"], nt, npf, a["c"], a["a_r"], a["dt"], a["bc"], a["sigma_a"], a["cv"], a["T0"],
                     OracleTTSN.isotropic_cores(I0, nt, npf), sigma_s=a["sigma_s"], eps=1e-5,
                     rounding="ttsvd", flux=flux, **fk)
    g = ttsn.TTSN(eps=1e-5, flux=flux, **fk, **a)
    for _ in range(4):
        ref.step()
        info = g.step(forced=[r for rk in ref.last_ranks for r in rk])
        assert info["ranks"][1:-1] == tt.ranks(ref.cores)
    R = ref.full()
    assert np.linalg.norm(g.full().cpu().numpy() - R) <= 1e-10 * np.linalg.norm(R)
    _, T, _ = g.energy()
    assert np.abs(T.cpu().numpy() - ref.T).max() <= 1e-10 * np.abs(ref.T).max()


@pytest.mark.parametrize("flux,fk", FLUXES[::2])
def test_split_step_equals_grouped_oracle(ttsn, flux, fk):
    """The split layout from the 2D pulse's initial state equals the grouped
    oracle's untruncated steps (same tensor in both layouts)."""
    p = workloads.problem("small_2d", n=(16, 12), n_theta=4, n_phi=8, bc=VACUUM)
    I0 = p["c"] * p["a_r"] * p["Tr0"] ** 4 / (4 * np.pi)
    ref = OracleTTSN(p["n"], p["L"], p["n_theta"], p["n_phi"], p["c"], p["a_r"], p["dt"], p["bc"],
                     p["sigma_a"], p["cv"], p["T0"],
                     OracleTTSN.isotropic_cores(I0.reshape(-1), p["n_theta"], p["n_phi"]),
                     rounding=None, flux=flux, **fk)
    g = ttsn.TTSN.from_problem(p, layout=ttsn.TT_LAYOUT_SPLIT, flux=flux, eps=0.0, **fk)
    g.set_cores(SplitTTSN.isotropic_cores(I0, p["n_theta"], p["n_phi"]))
    for _ in range(2):
        ref.step()
        g.step(flags=ttsn.TT_STEP_NO_ROUND)
    R = ref.full()
    assert np.abs(g.full().cpu().numpy() - R).max() <= 1e-12 * np.abs(R).max()


@pytest.mark.parametrize("flux,fk", FLUXES[::2])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_energy_conserved_periodic_all_fluxes(ttsn, flux, fk, precision):
    n, nt, npf = (20, 18), 8, 16
    a = _args(n, nt, npf, PERIODIC, 27)
    prec = ttsn.TT_FP64 if precision == "fp64" else ttsn.TT_MIXED
    g = ttsn.TTSN(eps=1e-5, flux=flux, precision=prec, **fk, **a)
    _, _, t0 = g.energy()
    g.step(5)
    _, _, t1 = g.energy()
    assert abs(sum(t1) - sum(t0)) <= 1e-12 * sum(t0)


def test_hll_mixed_matches_fp64_at_fp64_ranks(ttsn):
    n, nt, npf = (48, 40), 8, 16
    a = _args(n, nt, npf, VACUUM, 29)
    g64 = ttsn.TTSN(eps=1e-5, flux="hll", hll_beta=2.0, **a)
    gmx = ttsn.TTSN(eps=1e-5, flux="hll", hll_beta=2.0, precision=ttsn.TT_MIXED, **a)
    for _ in range(8):
        info = g64.step()
        gmx.step(forced=info["ranks"][1:-1])
    E64, T64, _ = g64.energy()
    Em, Tm, _ = gmx.energy()
    assert float((Em - E64).abs().max() / E64.abs().max()) <= 1e-8
    assert float((Tm - T64).abs().max() / T64.abs().max()) <= 1e-8


@pytest.mark.parametrize("bad", [dict(flux=5), dict(flux="rusanov", rusanov_s=-0.1),
                                 dict(flux="hll", hll_beta=0.0), dict(flux="hll", hll_tau_threshold=1.5),
                                 dict(flux="hll", hll_tau_threshold=0.0), dict(flux="rusanov_tau", hll_beta=0.0),
                                 dict(flux="rusanov_tau", hll_beta=-1.0)])
def test_flux_parameter_errors(ttsn, bad):
    a = _args((6, 5), 4, 8, VACUUM, 31)
    with pytest.raises(ttsn.TTError) as e:
        ttsn.TTSN(**bad, **a)
    assert e.value.status == -1


def test_adjoint_tape_needs_upwinding(ttsn):
    a = _args((6, 5), 4, 8, VACUUM, 33)
    a["sigma_s"] = None
    g = ttsn.TTSN(flux="rusanov", **a)
    assert ttsn.lib.tt_tape_begin(g._h, ctypes.c_int(1)) == -6
    g.step()


def _gauss_E(p, t):
    """The analytic E(t, x, y) of the Gaussian-diffusion test (Sec. 5)."""
    xc = workloads.cell_centres(p["n"], p["L"])
    r2 = sum((x - c0) ** 2 for x, c0 in zip(xc, p["centre"]))
    s = 4.0 * p["D"] * (p["t0"] + t)
    return p["amp"] / (np.pi * s) * np.exp(-r2 / s)


def test_gaussian_diffusion_128_follows_the_analytic_solution(ttsn):
    """The paper's Gaussian-diffusion setup (128^2 cells on 5 x 5, rho kappa_s =
    1e3, Rusanov flux at S+ = 0) for 1024 steps (t0 = 200 -> 220): E stays
    within 5e-3 of the analytic solution while that moves by more than 25x as
    much from the initial state."""
    p = workloads.gaussian_diffusion()
    g = ttsn.TTSN.from_problem(p, flux="rusanov", rusanov_s=0.0)
    steps = 1024
    g.step(steps)
    E, _, _ = g.energy()
    Ea, E0 = _gauss_E(p, steps * p["dt"]).reshape(-1), _gauss_E(p, 0.0).reshape(-1)
    err = np.linalg.norm(E.cpu().numpy() - Ea) / np.linalg.norm(Ea)
    moved = np.linalg.norm(E0 - Ea) / np.linalg.norm(Ea)
    assert err <= 5e-3 and err <= moved / 25, (err, moved)


def test_gaussian_diffusion_32_matches_the_dense_oracle(ttsn):
    p = workloads.gaussian_diffusion(n=(32, 32), eps=1e-9)
    I0 = (p["c"] * p["a_r"] * p["Tr0"] ** 4 / (4 * np.pi))[..., None, None] * np.ones((p["n_theta"], p["n_phi"]))
    d = DenseSN(p["n"], p["L"], p["n_theta"], p["n_phi"], p["c"], p["a_r"], p["dt"], p["bc"], p["sigma_a"],
                p["cv"], p["T0"], I0, sigma_s=p["sigma_s"], flux="rusanov", rusanov_s=0.0)
    g = ttsn.TTSN.from_problem(p, flux="rusanov", rusanov_s=0.0)
    for _ in range(200):
        d.step()
    g.step(200)
    E, _, _ = g.energy()
    Ed = d.energy_density().reshape(-1)
    # 200 roundings at eps = 1e-9 (each within eps of the tensor, Gram-SVD
    # resolution ~1e-8 of the largest singular value)
    assert np.abs(E.cpu().numpy() - Ed).max() <= 1e-6 * np.abs(Ed).max()


@pytest.mark.parametrize("layout", ["grouped", "split"])
@pytest.mark.parametrize("n,bc", [((9, 7), [2, 2]), ((6, 5, 4), [2, 1, 0])])
@pytest.mark.parametrize("flux,fk", [("upwind", {}), ("hll", dict(hll_beta=2.0, hll_tau_threshold=1.0)),
                                     ("rusanov_tau", dict(hll_beta=20.0))])
def test_outflow_faces_untruncated_step_equals_dense(ttsn, layout, n, bc, flux, fk):
    """Outflow faces (ghost cells copy the boundary cell, Sec. 4.5)."""
    nt, npf = 4, 6
    a = _args(n, nt, npf, 0, 35, uniform=(layout == "split"))
    a["bc"] = bc
    if layout == "split":
        cores = workloads.random_positive_tt(list(n) + [nt, npf], [3, 2, 2, 3][: len(n) + 1], seed=36)
        full = tt.full(cores)
    else:
        cores = workloads.random_positive_tt([int(np.prod(n)), nt, npf], [3, 2], seed=36)
        full = tt.full(cores).reshape(tuple(n) + (nt, npf))
    d = _dense(a, n, nt, npf, full, flux, fk)
    g = ttsn.TTSN(eps=0.0, flux=flux, layout=ttsn.TT_LAYOUT_SPLIT if layout == "split" else 0, **fk, **a)
    g.set_cores(cores)
    for _ in range(2):
        d.step()
        g.step(flags=ttsn.TT_STEP_NO_ROUND)
    F = g.full().cpu().numpy()
    assert np.abs(F - d.I).max() <= 1e-12 * np.abs(d.I).max()
