"""The line source of Sec. 5.4 on the GPU: a Gaussian pulse of radiation
streaming through an empty vacuum domain, where the rank grows step after
step (the paper's hard case for the TT format)."""
import numpy as np
import pytest
import torch

import workloads
from oracle.analytic import line_source_E
from oracle.dense import DenseSN

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ttsn():
    assert torch.cuda.is_available()
    import paper_2503_18056_gb300 as m

    return m


def test_line_source_rounded_run_stays_within_the_rounding_bound_of_dense(ttsn):
    """64^2 cells on [-1.1, 1.1]^2, 16 x 32 ordinates, pulse width 0.1,
    eps 1e-4, to t = 0.5 (36 steps).  With no material the source stage is
    the identity, the upwind update of each ordinate is a convex combination
    of cell values at this CFL (so a contraction in the Frobenius norm), and
    each rounding moves the tensor by at most eps times its norm; hence
    ||I_TT - I_dense||_F <= steps * eps * ||I_0||_F after `steps` steps.  The
    TT run's E stays as close to the analytic solution as the dense run's."""
    nt, npf = 16, 32
    p = workloads.line_source(n=(64, 64), n_theta=nt, n_phi=npf, omega=0.1, eps=1e-4)
    E0 = p["Tr0"] ** 4
    I0 = (p["c"] * E0 / (4 * np.pi))[..., None, None] * np.ones((nt, npf))
    d = DenseSN(p["n"], p["L"], nt, npf, p["c"], p["a_r"], p["dt"], p["bc"], p["sigma_a"], p["cv"], p["T0"],
                I0.copy())
    g = ttsn.TTSN.from_problem(p)
    steps = int(round(0.5 / p["dt"]))
    ranks = []
    for _ in range(steps):
        d.step()
        ranks.append(g.step()["ranks"][1:-1])
    diff = np.linalg.norm(g.full().cpu().numpy() - d.I)
    bound = steps * p["eps"] * np.linalg.norm(I0)
    assert diff <= bound, (diff, bound)
    assert ranks[-1][0] > ranks[0][0]  # the rank grows as the ring spreads
    E, T, _ = g.energy()
    E = E.cpu().numpy().reshape(p["n"])
    Ea = line_source_E(steps * p["dt"], p["radius"], 0.1)
    err_tt = np.abs(E - Ea).sum() / np.abs(Ea).sum()
    err_dense = np.abs(d.energy_density() - Ea).sum() / np.abs(Ea).sum()
    assert abs(err_tt - err_dense) <= 1e-3, (err_tt, err_dense)
    # rounding moves radiation energy into T (C_v dT = E* - E^{m+1}); the
    # total of E + C_v T equals the dense run's up to what each run leaks
    # through the faces
    dV = float(np.prod([p["L"][a] / p["n"][a] for a in range(2)]))
    tot = (E.sum() + (p["cv"].reshape(-1) * T.cpu().numpy()).sum()) * dV
    tot_d = (d.energy_density().sum() + (p["cv"] * d.T).sum()) * dV
    assert abs(tot - tot_d) <= 1e-6 * abs(tot_d)
