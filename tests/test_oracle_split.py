"""Pins for the oracle's split-space stepper (one core per spatial axis, then
theta and phi; Sec. 4.1 TT arithmetic, Sec. 4.3-4.5 step) against the dense
S_N stepper, closed forms and invariants."""
import numpy as np
import pytest

import workloads
from oracle import tt
from oracle.dense import DenseSN
from oracle.split import PERIODIC, VACUUM, SplitTTSN, field_tt, spatial_full
from oracle.ttstep import TTSN


@pytest.mark.parametrize("n", [(9,), (7, 5), (4, 5, 3)])
def test_field_tt_reproduces_the_field(n):
    rng = np.random.default_rng(1)
    F = rng.standard_normal(n)
    cores = field_tt(F)
    assert len(cores) == len(n)
    assert np.abs(tt.full(cores) - F).max() <= 1e-13 * np.abs(F).max()
    # a separable field has rank one at every bond
    vecs = [rng.uniform(0.5, 1.5, m) for m in n]
    G = vecs[0]
    for v in vecs[1:]:
        G = np.multiply.outer(G, v)
    assert tt.ranks(field_tt(G))[: len(n) - 1] == [1] * (len(n) - 1)


def test_spatial_full_contracts_the_right_bond():
    rng = np.random.default_rng(2)
    cores = [rng.standard_normal((1, 4, 2)), rng.standard_normal((2, 3, 3)),
             rng.standard_normal((3, 5, 2))]  # last bond (rank 2) stays open
    u = np.array([0.3, -1.2])
    ref = np.einsum("ia,ajb,bkc,c->ijk", cores[0][0], cores[1], cores[2], u)
    assert np.allclose(spatial_full(cores, u), ref, rtol=1e-13, atol=1e-14)


def _split_pair(n, nt, npf, bc, seed, uniform=True, ranks=None):
    f = workloads.random_fields(n, seed + 100)
    if uniform:
        sigma_a = np.full(n, float(f["sigma_a"].reshape(-1)[0]))
    else:
        sigma_a = f["sigma_a"]
    d = len(n) + 2
    ranks = ranks or [2] * (d - 1)
    cores = workloads.random_positive_tt(list(n) + [nt, npf], ranks, seed)
    dt = 0.4 * min(1.0 / m for m in n)
    args = dict(n=n, L=[1.0] * len(n), n_theta=nt, n_phi=npf, c=1.0, a_r=1.0, dt=dt,
                bc=[bc] * len(n), cv=f["cv"], T0=f["T0"])
    sp = SplitTTSN(cores=cores, rounding=None, sigma_a=sigma_a, **args)
    dn = DenseSN(I0=tt.full(cores), sigma_a=sigma_a, **args)
    return sp, dn


@pytest.mark.parametrize("n,bc", [((12,), VACUUM), ((8, 6), PERIODIC), ((8, 6), VACUUM),
                                  ((5, 4, 3), PERIODIC), ((5, 4, 3), VACUUM)])
@pytest.mark.parametrize("uniform", [True, False])
def test_untruncated_split_step_equals_dense_step(n, bc, uniform):
    sp, dn = _split_pair(n, 4, 6, bc, seed=11, uniform=uniform)
    for _ in range(2):
        sp.step()
        dn.step()
    F = sp.full()
    assert np.abs(F - dn.I).max() <= 1e-12 * np.abs(dn.I).max()
    assert np.abs(sp.T - dn.T).max() <= 1e-12 * np.abs(dn.T).max()


def test_untruncated_split_transport_ranks():
    """Transport alone multiplies every bond by 1 + 2 ndim (Sec. 4.1 addition)."""
    sp, _ = _split_pair((5, 4), 4, 6, PERIODIC, seed=3, ranks=[2, 3, 2])
    out = sp.transport(sp.cores)
    assert tt.ranks(out) == [10, 15, 10]


def test_split_and_grouped_steps_agree_untruncated():
    """The two layouts hold the same tensor: one step of each from the same
    intensity gives the same result (both equal the dense step)."""
    n, nt, npf = (6, 5), 4, 6
    sp, dn = _split_pair(n, nt, npf, VACUUM, seed=5)
    F0 = sp.full()
    gt = tt_three(F0.reshape(30, nt, npf))
    g = TTSN(n, [1.0, 1.0], nt, npf, 1.0, 1.0, sp.dt, [VACUUM] * 2, sp.sigma_a.reshape(-1),
             sp.cv.reshape(-1), sp.T.reshape(-1), gt, rounding=None)
    sp.step()
    g.step()
    assert np.abs(sp.full() - g.full()).max() <= 1e-12 * np.abs(g.full()).max()


def tt_three(F):
    """Exact three-core TT of F (N_c, n_theta, n_phi) by two SVDs."""
    nc, nt, npf = F.shape
    U, S, Vt = np.linalg.svd(F.reshape(nc, nt * npf), full_matrices=False)
    r1 = len(S)
    X = U.reshape(1, nc, r1)
    R = (S[:, None] * Vt).reshape(r1 * nt, npf)
    U2, S2, Vt2 = np.linalg.svd(R, full_matrices=False)
    return [X, U2.reshape(r1, nt, len(S2)), (S2[:, None] * Vt2).reshape(len(S2), npf, 1)]


def test_equilibrium_is_a_fixed_point_split():
    n, nt, npf = (6, 4), 4, 8
    T = np.full(n, 0.7)
    I0 = 0.7 ** 4 / (4 * np.pi)
    cores = SplitTTSN.isotropic_cores(np.full(n, I0), nt, npf)
    sp = SplitTTSN(n, [1.0, 1.0], nt, npf, 1.0, 1.0, 0.05, [PERIODIC] * 2, 3.0, np.ones(n), T,
                   cores, eps=1e-10)
    for _ in range(3):
        sp.step()
    assert np.abs(sp.full() - I0).max() <= 1e-14
    assert np.abs(sp.T - 0.7).max() <= 1e-14
    assert tt.ranks(sp.cores) == [1, 1, 1]


@pytest.mark.parametrize("rounds", [1, 2])
def test_periodic_energy_conserved_with_truncation_split(rounds):
    """One rounding per step: sum (E + C_v T) dV is conserved to round-off (the
    temperature update absorbs the source stage and the rounding).  With the
    post-transport rounding as well, that first rounding's change of E is not
    absorbed, so the total moves by at most eps of the energy per step."""
    n, nt, npf = (8, 7), 4, 8
    f = workloads.random_fields(n, 21)
    cores = SplitTTSN.isotropic_cores(f["T0"] ** 4 / (4 * np.pi), nt, npf)
    eps = 1e-3
    sp = SplitTTSN(n, [1.0, 1.0], nt, npf, 1.0, 1.0, 0.05, [PERIODIC] * 2, 2.0, f["cv"], f["T0"],
                   cores, eps=eps, rounds_per_step=rounds)
    e0 = sp.total_energy()
    for m in range(1, 6):
        sp.step()
        tol = 1e-13 if rounds == 1 else m * eps
        assert abs(sp.total_energy() - e0) <= tol * e0


def test_small_2d_workload_split_stays_near_dense():
    """The 2D 32 x 32, 8 x 16 Gaussian-pulse problem in the split layout at
    eps = 1e-8: after 10 steps the TT stays within the rounding error of the
    dense stepper (each TT-SVD rounding moves the tensor by at most eps ||X||;
    the Gram-SVD rounding resolves only ~sqrt(eps_mach) of sigma_max, App. A.4,
    so the bound is checked with TT-SVD)."""
    p = workloads.problem("small_2d")
    I0 = p["c"] * p["a_r"] * p["Tr0"] ** 4 / (4 * np.pi)
    cores = SplitTTSN.isotropic_cores(I0, p["n_theta"], p["n_phi"])
    assert tt.ranks(cores)[0] <= 5  # T = bg + g(x) g(y): T^4 has rank <= 5
    sp = SplitTTSN(p["n"], p["L"], p["n_theta"], p["n_phi"], p["c"], p["a_r"], p["dt"], p["bc"],
                   1.0, p["cv"], p["T0"], cores, eps=p["eps"], rounding="ttsvd")
    dn = DenseSN(p["n"], p["L"], p["n_theta"], p["n_phi"], p["c"], p["a_r"], p["dt"], p["bc"],
                 p["sigma_a"], p["cv"], p["T0"], tt.full(cores))
    for _ in range(p["steps"]):
        sp.step()
        dn.step()
    F = sp.full()
    assert np.linalg.norm(F - dn.I) <= 10 * p["eps"] * np.linalg.norm(dn.I)
    assert np.abs(sp.T - dn.T).max() <= 1e-7 * np.abs(dn.T).max()
