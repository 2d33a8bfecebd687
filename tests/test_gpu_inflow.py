"""Inflow faces on the GPU (tt_set_inflow: a rank-one Dirichlet ghost
intensity on a vacuum face, Sec. 4.5) and the hohlraum problem of Sec. 5.1."""
import numpy as np
import pytest
import torch

import workloads
from oracle import tt
from oracle.analytic import hohlraum_J
from oracle.dense import DenseSN
from oracle.ttstep import PERIODIC, VACUUM, TTSN as OracleTTSN

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ttsn():
    assert torch.cuda.is_available()
    import paper_2503_18056_gb300 as m

    return m


def _inflow(n, nt, npf, seed):
    rng = np.random.default_rng(seed)
    return {(0, 0): (rng.uniform(0.5, 1.5, n), rng.uniform(0.5, 1.5, nt), rng.uniform(0.5, 1.5, npf)),
            (len(n) - 1, 1): (rng.uniform(0.5, 1.5, n), np.ones(nt), rng.uniform(0.5, 1.5, npf))}


@pytest.mark.parametrize("n", [(13,), (9, 7), (6, 5, 4)])
@pytest.mark.parametrize("flux,fk", [("upwind", {}), ("rusanov", dict(rusanov_s=0.5)),
                                     ("hll", dict(hll_beta=2.0, hll_tau_threshold=1.0))])
def test_untruncated_step_with_inflow_equals_dense(ttsn, n, flux, fk):
    nt, npf = 4, 6
    f = workloads.random_fields(n, 51)
    nc = int(np.prod(n))
    cores = workloads.random_positive_tt([nc, nt, npf], [3, 2], 52)
    inflow = _inflow(n, nt, npf, 53)
    a = dict(n=n, L=[1.0] * len(n), n_theta=nt, n_phi=npf, c=1.0, a_r=1.0, dt=0.3 * min(1.0 / m for m in n),
             bc=[VACUUM] * len(n), sigma_a=f["sigma_a"].reshape(-1), cv=f["cv"].reshape(-1),
             T0=f["T0"].reshape(-1))
    d = DenseSN(I0=tt.full(cores).reshape(tuple(n) + (nt, npf)), flux=flux, inflow=inflow, **fk,
                **{k: (v.reshape(n) if isinstance(v, np.ndarray) else v) for k, v in a.items()})
    g = ttsn.TTSN(eps=0.0, flux=flux, **fk, **a)
    g.set_cores(cores)
    for (axis, side), (gf, th, ph) in inflow.items():
        g.set_inflow(axis, side, gf, th, ph)
    for _ in range(2):
        d.step()
        g.step(flags=ttsn.TT_STEP_NO_ROUND)
    F = g.full().cpu().numpy()
    assert np.abs(F - d.I).max() <= 1e-12 * np.abs(d.I).max()
    _, T, _ = g.energy()
    assert np.abs(T.cpu().numpy() - d.T.reshape(-1)).max() <= 1e-12 * np.abs(d.T).max()


def test_hohlraum_rounded_steps_match_oracle_at_its_ranks(ttsn):
    p = workloads.hohlraum(n=(32, 32), n_theta=8, n_phi=16, eps=1e-4)
    ref = OracleTTSN(p["n"], p["L"], p["n_theta"], p["n_phi"], p["c"], p["a_r"], p["dt"], p["bc"],
                     p["sigma_a"], p["cv"], p["T0"],
                     OracleTTSN.isotropic_cores(np.zeros(32 * 32), p["n_theta"], p["n_phi"]),
                     eps=p["eps"], rounding="ttsvd", inflow=p["inflow"])
    g = ttsn.TTSN.from_problem(p)
    for _ in range(12):
        ref.step()
        info = g.step(forced=[r for rk in ref.last_ranks for r in rk])
        assert info["ranks"][1:-1] == tt.ranks(ref.cores)
    R = ref.full()
    assert np.linalg.norm(g.full().cpu().numpy() - R) <= 1e-10 * np.linalg.norm(R)


def test_hohlraum_256_follows_the_analytic_solution(ttsn):
    """Sec. 5.1 at dx = 1/128 (256^2 on [0, 2]^2), 32 x 64 ordinates, eps 1e-4,
    upwinding, to t = 0.75: the L1 error of J over the causally disconnected
    subset [0, 1)^2 (dense oracle on 64^2: 9e-3 at 8 x 16, 7.4e-3 at 16 x 32)."""
    p = workloads.hohlraum()
    g = ttsn.TTSN.from_problem(p)
    steps = int(round(p["t_lim"] / p["dt"]))
    info = g.step(steps)
    E, _, _ = g.energy()
    xc = workloads.cell_centres(p["n"], p["L"])
    J = p["c"] * E.cpu().numpy().reshape(p["n"]) / (4 * np.pi)
    Ja = hohlraum_J(steps * p["dt"], xc[0], xc[1], p["c"])
    sub = (xc[0] < 1.0) & (xc[1] < 1.0)
    err = float(np.mean(np.abs(J - Ja)[sub]))
    print("hohlraum 256^2 32x64: L1 %.4e ranks %s" % (err, info["ranks"]))
    assert err < 6e-3, err


def test_inflow_argument_errors(ttsn):
    p = workloads.problem("small_2d", n=(6, 5), n_theta=4, n_phi=8, bc=PERIODIC)
    g = ttsn.TTSN.from_problem(p)
    with pytest.raises(ttsn.TTError) as e:
        g.set_inflow(0, 0, np.ones(30), np.ones(4), np.ones(8))  # periodic axis
    assert e.value.status == -1
    q = workloads.problem("small_2d", n=(6, 5), n_theta=4, n_phi=8, bc=VACUUM)
    g = ttsn.TTSN.from_problem(q)
    with pytest.raises(ttsn.TTError):
        g.set_inflow(2, 0, np.ones(30), np.ones(4), np.ones(8))  # no such axis
    src = [(np.ones(30), np.ones(4), np.ones(8))] * 15
    g.set_sources(src)
    with pytest.raises(ttsn.TTError):
        g.set_inflow(0, 0, np.ones(30), np.ones(4), np.ones(8))  # 15 + 2 terms > 16
    g.set_sources(src[:4])
    g.set_inflow(0, 0, np.ones(30), np.ones(4), np.ones(8))
    g.step()
    g.set_inflow(0, 0)  # removed
    g.step()
    s = ttsn.TTSN.from_problem(workloads.problem("small_2d", n=(6, 5), n_theta=4, n_phi=8, bc=VACUUM),
                               layout=ttsn.TT_LAYOUT_SPLIT)
    with pytest.raises(ttsn.TTError) as e:
        s.set_inflow(0, 0, np.ones(30), np.ones(4), np.ones(8))
    assert e.value.status == -6
