"""Pins for the oracle's TT arithmetic (Sec. 4.1) and TT stepper (Sec. 4.3-4.5)."""
import numpy as np
import pytest

import workloads
from oracle import angles, tt
from oracle.dense import DenseSN
from oracle.ttstep import PERIODIC, VACUUM, TTSN


def test_addition_hadamard_inner_match_full():
    A = workloads.random_tt([3, 4, 5, 2], [2, 3, 2], seed=1)
    B = workloads.random_tt([3, 4, 5, 2], [1, 2, 3], seed=2)
    FA, FB = tt.full(A), tt.full(B)
    S = tt.add(A, B)
    assert tt.ranks(S) == [3, 5, 5]
    assert np.allclose(tt.full(S), FA + FB, atol=1e-13)
    H = tt.hadamard(A, B)
    assert tt.ranks(H) == [2, 6, 6]
    assert np.allclose(tt.full(H), FA * FB, atol=1e-12)
    assert abs(tt.inner(A, B) - (FA * FB).sum()) < 1e-11
    assert abs(tt.norm(A) - np.linalg.norm(FA)) < 1e-12


def test_energy_density_grouped_matches_dense_sum():
    g = angles.grid(4, 6)
    cores = workloads.random_tt([10, 4, 6], [3, 2], seed=3)
    F = tt.full(cores)
    E = tt.energy_density_grouped(cores, g["w"], g["v"], 2.0)
    ref = np.einsum("ilp,lp->i", F, angles.solid_angles(g)) / 2.0
    assert np.allclose(E, ref, rtol=1e-13, atol=1e-14)


def _pair(n, nt, npf, bc, seed, ranks=(3, 2), with_fields=True):
    nc = int(np.prod(n))
    cores = workloads.random_positive_tt([nc, nt, npf], list(ranks), seed)
    f = workloads.random_fields(n, seed + 100)
    dt = 0.4 * min(1.0 / m for m in n)
    args = dict(n=n, L=[1.0] * len(n), n_theta=nt, n_phi=npf, c=1.0, a_r=1.0, dt=dt,
                bc=[bc] * len(n), sigma_a=f["sigma_a"], cv=f["cv"], T0=f["T0"])
    ttsn = TTSN(cores=cores, rounding=None, **args)
    d = DenseSN(I0=tt.full(cores).reshape(tuple(n) + (nt, npf)), **args)
    return ttsn, d


@pytest.mark.parametrize("n,bc", [((12,), VACUUM), ((8, 6), PERIODIC), ((8, 6), VACUUM),
                                  ((5, 4, 3), PERIODIC), ((5, 4, 3), VACUUM)])
def test_untruncated_tt_step_equals_dense_step(n, bc):
    ttsn, d = _pair(n, 4, 6, bc, seed=7)
    for _ in range(2):
        ttsn.step()
        d.step()
    F = ttsn.full()
    scale = np.abs(d.I).max()
    assert np.abs(F - d.I).max() <= 1e-12 * scale
    assert np.abs(ttsn.T - d.T.reshape(-1)).max() <= 1e-12
    # ranks grew as (1 + 2 ndim) r + 1 per step (transport terms plus emission)
    r1 = tt.ranks(ttsn.cores)[0]
    k = 1 + 2 * len(n)
    assert r1 == k * (k * 3 + 1) + 1


def test_transport_only_equals_dense_transport():
    ttsn, d = _pair((9, 7), 4, 8, VACUUM, seed=11)
    Istar = d.transport(d.I)
    cur = ttsn.transport(ttsn.cores)
    assert np.abs(tt.full(cur).reshape(Istar.shape) - Istar).max() <= 1e-14 * np.abs(Istar).max()


def test_periodic_energy_conserved_with_truncation():
    p = workloads.problem("small_2d", n=(16, 16), n_theta=4, n_phi=8)
    I0 = p["c"] * p["a_r"] * p["Tr0"] ** 4 / (4 * np.pi)
    for rounding in ("gram", "ttsvd"):
        s = TTSN(p["n"], p["L"], p["n_theta"], p["n_phi"], p["c"], p["a_r"], p["dt"], p["bc"],
                 p["sigma_a"], p["cv"], p["T0"], TTSN.isotropic_cores(I0.reshape(-1), 4, 8),
                 eps=1e-3, rounding=rounding)
        e0 = s.total_energy()
        for _ in range(4):
            s.step()
        assert abs(s.total_energy() - e0) <= 1e-13 * e0
        assert max(tt.ranks(s.cores)) < 50  # rounding did truncate


def test_isotropic_uniform_problem_keeps_rank_one():
    # Sec. 5.2: the relaxation problem keeps ranks (1, 1)
    n = (4,)
    I0 = np.full(4, 1.0 / (4 * np.pi))
    s = TTSN(n, [4.0], 8, 16, 1.0, 1.0, 0.01, [PERIODIC], np.full(4, 1.0), np.full(4, 8.0),
             np.full(4, 2.0), TTSN.isotropic_cores(I0, 8, 16), eps=1e-8, rounding="gram")
    for _ in range(5):
        s.step()
    assert tt.ranks(s.cores) == [1, 1]


def test_equilibrium_fixed_point_tt():
    n = (6, 5)
    T = 0.9
    I0 = np.full(30, T ** 4 / (4 * np.pi))
    s = TTSN(n, [1, 1], 4, 8, 1.0, 1.0, 0.05, [PERIODIC] * 2, np.full(30, 3.0), np.ones(30),
             np.full(30, T), TTSN.isotropic_cores(I0, 4, 8), eps=1e-10, rounding="gram")
    s.step()
    assert np.abs(s.full() - T ** 4 / (4 * np.pi)).max() < 1e-15
    assert np.abs(s.T - T).max() < 1e-14
