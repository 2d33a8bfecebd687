"""Pins for outflow faces (Sec. 4.5: ghost cells copy the boundary cell) in
the oracle's dense, grouped-TT and split-TT steppers."""
import numpy as np
import pytest

import workloads
from oracle import angles, tt
from oracle.dense import OUTFLOW, DenseSN
from oracle.split import SplitTTSN
from oracle.ttstep import TTSN


def _args(n, nt, npf, bc, seed, flux="upwind", **fk):
    f = workloads.random_fields(n, seed)
    return dict(n=n, L=[1.0] * len(n), n_theta=nt, n_phi=npf, c=1.0, a_r=1.0,
                dt=0.3 * min(1.0 / m for m in n), bc=bc, sigma_a=f["sigma_a"], cv=f["cv"], T0=f["T0"],
                flux=flux, **fk)


@pytest.mark.parametrize("n,bc", [((12,), [OUTFLOW]), ((8, 6), [OUTFLOW, OUTFLOW]), ((8, 6), [OUTFLOW, 0]),
                                  ((5, 4, 3), [OUTFLOW, 1, OUTFLOW])])
@pytest.mark.parametrize("flux,fk", [("upwind", {}), ("rusanov", dict(rusanov_s=0.5)),
                                     ("hll", dict(hll_beta=2.0, hll_tau_threshold=1.0))])
def test_untruncated_grouped_step_with_outflow_equals_dense(n, bc, flux, fk):
    nt, npf = 4, 6
    a = _args(n, nt, npf, bc, 5, flux, **fk)
    nc = int(np.prod(n))
    cores = workloads.random_positive_tt([nc, nt, npf], [3, 2], 6)
    t = TTSN(cores=cores, rounding=None, **a)
    d = DenseSN(I0=tt.full(cores).reshape(tuple(n) + (nt, npf)), **a)
    for _ in range(2):
        t.step()
        d.step()
    assert np.abs(t.full() - d.I).max() <= 1e-12 * np.abs(d.I).max()


@pytest.mark.parametrize("n,bc", [((8, 6), [OUTFLOW, OUTFLOW]), ((5, 4, 3), [OUTFLOW, 1, 0])])
def test_untruncated_split_step_with_outflow_equals_dense(n, bc):
    nt, npf = 4, 6
    a = _args(n, nt, npf, bc, 7)
    a["sigma_a"] = np.full(n, 2.0)
    a.pop("flux")
    cores = workloads.random_positive_tt(list(n) + [nt, npf], [3, 2, 2, 3][: len(n) + 1], 8)
    s = SplitTTSN(cores=cores, rounding=None, **a)
    d = DenseSN(I0=tt.full(cores), **a)
    for _ in range(2):
        s.step()
        d.step()
    assert np.abs(s.full() - d.I).max() <= 1e-12 * np.abs(d.I).max()


@pytest.mark.parametrize("flux,fk", [("upwind", {}), ("rusanov", dict(rusanov_s=1.0)), ("hll", dict(hll_beta=1.0))])
def test_uniform_field_is_a_fixed_point_of_outflow_transport(flux, fk):
    """With zero-gradient faces a uniform (angle-dependent) intensity has no
    net flux through any face, so transport leaves it unchanged; vacuum faces
    would drain it."""
    n, nt, npf = (7, 5), 4, 8
    rng = np.random.default_rng(3)
    ang = rng.uniform(0.5, 1.5, (nt, npf))
    I0 = np.broadcast_to(ang, n + (nt, npf)).copy()
    d = DenseSN(n, [1.0, 1.0], nt, npf, 1.0, 1.0, 0.05, [OUTFLOW, OUTFLOW], np.full(n, 3.0), np.ones(n),
                np.ones(n), I0, flux=flux, **fk)
    assert np.abs(d.transport(d.I) - I0).max() <= 1e-15 * I0.max()
    dv = DenseSN(n, [1.0, 1.0], nt, npf, 1.0, 1.0, 0.05, [1, 1], np.full(n, 3.0), np.ones(n),
                 np.ones(n), I0, flux=flux, **fk)
    assert np.abs(dv.transport(dv.I) - I0).max() > 1e-3


def test_outflow_energy_change_is_the_face_flux():
    """Upwind transport with outflow faces: sum_i E_i dV changes by exactly
    -dt sum_faces dA sum_lp (n . n_out) I_boundary dOmega (c = 1), the net
    energy through the faces (the discrete conservative update telescopes;
    outgoing ordinates leave with the boundary value and incoming ones bring
    the copied ghost value, the same boundary value)."""
    n, nt, npf = (9, 6), 4, 8
    rng = np.random.default_rng(4)
    I0 = rng.uniform(0.1, 1.0, n + (nt, npf))
    d = DenseSN(n, [1.0, 1.0], nt, npf, 1.0, 1.0, 0.03, [OUTFLOW, OUTFLOW], np.ones(n), np.ones(n),
                np.ones(n), I0)
    g = angles.grid(nt, npf)
    dO = angles.solid_angles(g)
    nx, ny = angles.normals(g)[:2]
    dx, dy = d.dx
    E0 = d.energy_density(I0).sum() * dx * dy
    E1 = d.energy_density(d.transport(I0)).sum() * dx * dy
    # faces: x = 0 (n_out = -x), x = 1 (+x), y = 0 (-y), y = 1 (+y)
    out = 0.0
    out += np.einsum("jlp,lp->", I0[-1], nx * dO) * dy - np.einsum("jlp,lp->", I0[0], nx * dO) * dy
    out += np.einsum("ilp,lp->", I0[:, -1], ny * dO) * dx - np.einsum("ilp,lp->", I0[:, 0], ny * dO) * dx
    assert abs((E1 - E0) - (-d.dt * out)) <= 1e-13 * E0
