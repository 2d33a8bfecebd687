"""Pins for the oracle's fixed external sources (I* = L I + c dt S): the
one-step closed form from a cold, transparent start, the energy balance with
sources on a periodic domain (the source's integrated power is the only
change of sum(E + C_v T)), and the untruncated TT step against the dense one."""
import numpy as np
import pytest

import workloads
from oracle import angles
from oracle.dense import DenseSN
from oracle.ttstep import PERIODIC, VACUUM, TTSN


def _sources(n, nt, npf, seed, count=2):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        x = rng.uniform(0.0, 1.0, n) * (rng.uniform(size=n) < 0.3)
        out.append((x, rng.uniform(0.0, 2.0, nt), rng.uniform(0.0, 2.0, npf)))
    return out


def test_one_step_from_cold_transparent_start_is_c_dt_S():
    n, nt, npf = (6, 5), 4, 8
    src = _sources(n, nt, npf, 0)
    z = np.zeros(n)
    d = DenseSN(n, [1.0, 1.0], nt, npf, 2.0, 1.0, 0.03, [VACUUM, VACUUM], z, np.ones(n), z,
                np.zeros(n + (nt, npf)), sources=src)
    d.step()
    S = sum(x[..., None, None] * np.outer(th, ph) for x, th, ph in src)
    np.testing.assert_allclose(d.I, 2.0 * 0.03 * S, rtol=1e-15, atol=0)
    assert np.all(d.T == 0.0)


@pytest.mark.parametrize("kind", ["dense", "tt"])
def test_energy_balance_with_sources_periodic(kind):
    """sum(E + C_v T) dV grows by dt sum_k (sum_i x_k[i] dV) q_k per step,
    q_k = sum_lp theta_k[l] phi_k[p] dOmega_lp, through transport, source
    stage and rounding (periodic: streaming moves energy, never out)."""
    n, nt, npf = (9, 7), 4, 8
    f = workloads.random_fields(n, 5)
    src = _sources(n, nt, npf, 1)
    g = angles.grid(nt, npf)
    dO = angles.solid_angles(g)
    dt = 0.4 / 9
    dV = 1.0 / (9 * 7)
    power = sum(float(np.sum(x)) * dV * float(th @ dO @ ph) for x, th, ph in src)
    I0 = workloads.random_positive_tt([63, nt, npf], [3, 2], 6)
    args = dict(n=n, L=[1.0, 1.0], n_theta=nt, n_phi=npf, c=1.0, a_r=1.0, dt=dt,
                bc=[PERIODIC, PERIODIC], sigma_a=f["sigma_a"], cv=f["cv"], T0=f["T0"],
                sources=src)
    if kind == "dense":
        from oracle import tt
        s = DenseSN(I0=tt.full(I0).reshape(n + (nt, npf)), **args)
    else:
        s = TTSN(cores=I0, eps=1e-6, rounding="ttsvd", **args)
    e0 = s.total_energy()
    for m in range(1, 5):
        s.step()
        assert abs(s.total_energy() - (e0 + m * dt * power)) <= 1e-12 * (e0 + m * dt * power)


@pytest.mark.parametrize("n,bc", [((7, 6), VACUUM), ((5, 4, 3), PERIODIC)])
def test_untruncated_tt_step_with_sources_equals_dense(n, bc):
    from oracle import tt
    nt, npf = 4, 6
    nc = int(np.prod(n))
    cores = workloads.random_positive_tt([nc, nt, npf], [2, 3], 11)
    f = workloads.random_fields(n, 12)
    src = _sources(n, nt, npf, 13)
    args = dict(n=n, L=[1.0] * len(n), n_theta=nt, n_phi=npf, c=1.0, a_r=1.0,
                dt=0.4 * min(1.0 / m for m in n), bc=[bc] * len(n), sigma_a=f["sigma_a"],
                cv=f["cv"], T0=f["T0"], sources=src)
    ttsn = TTSN(cores=cores, rounding=None, **args)
    dense = DenseSN(I0=tt.full(cores).reshape(n + (nt, npf)), **args)
    for _ in range(2):
        ttsn.step()
        dense.step()
        scale = np.abs(dense.I).max()
        assert np.abs(ttsn.full() - dense.I).max() <= 1e-12 * scale
        assert np.abs(ttsn.T - dense.T.reshape(-1)).max() <= 1e-12 * np.abs(dense.T).max()


def test_crossing_beams_workload_shape():
    p = workloads.crossing_beams(n=(32, 32), n_theta=16, n_phi=32)
    (x1, th1, ph1), (x2, th2, ph2) = p["sources"]
    assert x1.sum() == 16 and x2.sum() == 8
    assert x1[0:4, 14:18].all() and x2[14:18, 0:4].all()
    # theta window: mu within sin(10 deg) of 0; phi windows around 0 and 90 deg
    mu = -1 + (np.arange(16) + 0.5) / 8
    assert np.array_equal(th1 > 0, np.abs(mu) <= np.sin(np.radians(10)) + 1e-12)
    phi = (np.arange(32) + 0.5) * 360 / 32
    assert set(np.flatnonzero(ph1)) == {p_ for p_ in range(32) if min(phi[p_], 360 - phi[p_]) <= 10}
    assert set(np.flatnonzero(ph2)) == {p_ for p_ in range(32) if abs(phi[p_] - 90) <= 10}
