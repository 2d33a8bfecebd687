"""The split-space layout on the GPU (one core per spatial axis, then theta
and phi; Sec. 4.1 / Sec. 7): the untruncated step equal to the dense step,
rounded steps at the oracle's ranks against the oracle's split stepper, the
2D 32 x 32, 8 x 16, 4-core workload, conservation, the precision form,
creation, and the argument errors of the layout."""
import ctypes

import numpy as np
import pytest
import torch

import workloads
from oracle import tt
from oracle.dense import DenseSN
from oracle.split import PERIODIC, VACUUM, SplitTTSN

pytestmark = pytest.mark.gpu

EPS_MACH = np.finfo(float).eps


@pytest.fixture(scope="module")
def ttsn():
    assert torch.cuda.is_available()
    import paper_2503_18056_gb300 as m

    return m


def _args(n, nt, npf, bc, seed):
    f = workloads.random_fields(n, seed)
    nc = int(np.prod(n))
    return dict(n=n, L=[1.0] * len(n), n_theta=nt, n_phi=npf, c=1.0, a_r=1.0,
                dt=0.4 * min(1.0 / m for m in n), bc=[bc] * len(n),
                sigma_a=np.full(nc, float(f["sigma_a"].reshape(-1)[3])), cv=f["cv"].reshape(-1),
                T0=f["T0"].reshape(-1))


def _emission_ranks(n):
    nd = len(n)
    er = [1] * (nd + 3)
    if nd >= 2:
        er[1] = n[0]
    if nd == 3:
        er[2] = n[2]
    return er


@pytest.mark.parametrize("n,bc", [((13,), VACUUM), ((9, 7), PERIODIC), ((9, 7), VACUUM),
                                  ((5, 4, 6), PERIODIC), ((6, 5, 4), VACUUM)])
@pytest.mark.parametrize("source", [False, True])
def test_untruncated_split_step_equals_dense(ttsn, n, bc, source):
    nt, npf = 4, 6
    a = _args(n, nt, npf, bc, seed=31)
    d = len(n) + 2
    r0 = [3, 2, 2, 3][: d - 1]
    cores = workloads.random_positive_tt(list(n) + [nt, npf], r0, seed=32)
    dn = DenseSN(n, a["L"], nt, npf, a["c"], a["a_r"], a["dt"], a["bc"],
                 a["sigma_a"].reshape(n), a["cv"].reshape(n), a["T0"].reshape(n), tt.full(cores))
    g = ttsn.TTSN(eps=0.0, layout=ttsn.TT_LAYOUT_SPLIT, **a)
    g.set_cores(cores)
    flags = ttsn.TT_STEP_NO_ROUND | (0 if source else ttsn.TT_STEP_NO_SOURCE)
    for _ in range(2):
        dn.step(with_source=source)
        info = g.step(flags=flags)
    F = g.full().cpu().numpy()
    assert np.abs(F - dn.I).max() <= 1e-12 * np.abs(dn.I).max()
    # ranks: every bond grows as K r (+ the emission term's rank), K = 1 + 2 ndim
    K = 1 + 2 * len(n)
    er = _emission_ranks(n)
    want = [1] + [K * (K * r + (er[k + 1] if source else 0)) + (er[k + 1] if source else 0)
                  for k, r in enumerate(r0)] + [1]
    assert info["ranks"] == want
    _, T, _ = g.energy()
    assert np.abs(T.cpu().numpy() - dn.T.reshape(-1)).max() <= 1e-12 * np.abs(dn.T).max()


def _split_pair(ttsn, p, rounding="ttsvd", **kw):
    """The oracle's split stepper from the isotropic initial intensity (TT-SVD
    of the field) and a GPU handle holding the same initial cores."""
    I0 = p["c"] * p["a_r"] * p["Tr0"] ** 4 / (4 * np.pi)
    cores = SplitTTSN.isotropic_cores(I0, p["n_theta"], p["n_phi"])
    ref = SplitTTSN(p["n"], p["L"], p["n_theta"], p["n_phi"], p["c"], p["a_r"], p["dt"], p["bc"],
                    p["sigma_a"], p["cv"], p["T0"], cores, eps=p["eps"],
                    max_rank=p.get("max_rank"), rounding=rounding, **kw)
    g = ttsn.TTSN.from_problem(p, layout=ttsn.TT_LAYOUT_SPLIT, **kw)
    g.set_cores(cores)
    return ref, g


def _forced(ref):
    return [r for rk in ref.last_ranks for r in rk]


@pytest.mark.parametrize("rounds", [1, 2])
@pytest.mark.parametrize("bc", [PERIODIC, VACUUM])
def test_split_step_matches_oracle_at_oracle_ranks(ttsn, rounds, bc):
    p = workloads.problem("small_2d", n=(16, 12), n_theta=4, n_phi=8, eps=1e-5, bc=bc)
    ref, g = _split_pair(ttsn, p, rounds_per_step=rounds)
    for _ in range(4):
        ref.step()
        info = g.step(forced=_forced(ref))
        assert info["ranks"][1:-1] == tt.ranks(ref.cores)
    F = g.full().cpu().numpy()
    R = ref.full()
    assert np.linalg.norm(F - R) <= 1e-10 * np.linalg.norm(R)
    E, T, _ = g.energy()
    # T inherits the TT's difference through E^{m+1} (T += (E* - E^{m+1}) / C_v)
    assert np.abs(T.cpu().numpy() - ref.T.reshape(-1)).max() <= 1e-10 * np.abs(ref.T).max()
    Eref = ref.energy_density().reshape(-1)
    assert np.abs(E.cpu().numpy() - Eref).max() <= 1e-10 * np.abs(Eref).max()


def test_split_3d_matches_oracle_at_oracle_ranks(ttsn):
    # eps = 1e-4: with delta = eps ||X|| / sqrt(d - 1) the cuts keep singular
    # values down to ~eps / 2 of the largest; the Gram-SVD resolves a kept
    # component of size sigma to ~eps_mach sigma_max / sigma (App. A.4), so at
    # eps = 1e-5 (kept values ~5e-6 sigma_max) each rounding alone may differ
    # from TT-SVD by ~4e-11 over 4 bonds (a numpy model of the same one-sided
    # rounding shows 6e-11 after 3 steps); at 1e-4 that is 10x smaller
    p = workloads.problem("small_2d", n=(8, 7, 6), n_theta=4, n_phi=8, eps=1e-4, bc=VACUUM,
                          sigma_a=np.full((8, 7, 6), 2.0))
    ref, g = _split_pair(ttsn, p)
    for _ in range(3):
        _step_at_gap_ranks(ref, g, p["eps"])
    R = ref.full()
    assert np.linalg.norm(g.full().cpu().numpy() - R) <= 1e-10 * np.linalg.norm(R)
    # T += (E* - E^{m+1}) / C_v: each step adds the E difference (within the
    # TT's 1e-10) divided by C_v
    _, T, _ = g.energy()
    Emax = np.abs(ref.energy_density()).max()
    assert np.abs(T.cpu().numpy() - ref.T.reshape(-1)).max() <= 3 * 1e-10 * Emax / ref.cv.min()


@pytest.mark.parametrize("eps", [1e-8, 1e-6])
def test_small_2d_split_workload_ten_steps(ttsn, eps):
    """2D 32 x 32 cells, 8 x 16 ordinates, 4 cores (x, y, theta, phi), sigma_a = 1,
    Gaussian T pulse, periodic, CFL 0.5, 10 steps, eps = 1e-8 (and 1e-6), at the
    ranks the oracle's TT-SVD picks.  At eps = 1e-8 the cuts lie at the Gram-SVD
    resolution (Gram eigenvalues carry errors ~ eps_mach lambda_max, App. A.4),
    so each rounding may differ from the exact truncation by up to
    2 sqrt(d-1) sqrt(eps^2 + R eps_mach) ||X||; that sum is the yardstick."""
    p = workloads.problem("small_2d", eps=eps)
    ref, g = _split_pair(ttsn, p)
    _, _, tot0 = g.energy()
    budget = 0.0
    for _ in range(p["steps"]):
        ref.step()
        info = g.step(forced=_forced(ref))
        R = max(info["grown"])
        budget += 2 * np.sqrt(3) * np.sqrt(p["eps"] ** 2 + R * EPS_MACH)
    F = g.full().cpu().numpy()
    Rf = ref.full()
    err = np.linalg.norm(F - Rf) / np.linalg.norm(Rf)
    assert err < budget, (err, budget)
    _, T, tot = g.energy()
    assert np.abs(T.cpu().numpy() - ref.T.reshape(-1)).max() < budget * np.abs(ref.T).max()
    assert abs(sum(tot) - sum(tot0)) <= 1e-12 * sum(tot0)


def _gap_ranks(grown, eps, ratio=1.05):
    """Ranks for the rounding of `grown`: bond by bond, the TT-SVD rank at eps
    moved up to the next clear gap (sigma_{r-1} / sigma_r >= ratio) of that
    bond's singular values given the cuts already chosen before it (moving a
    cut changes the later bonds' spectra).  The pulse's x <-> y and
    phi -> -phi symmetries give pairs of equal singular values; a cut inside a
    pair has no unique answer and makes the truncation ill-conditioned."""
    from oracle.rounding import round_ttsvd

    d = len(grown)
    ranks = []
    for k in range(d - 1):
        Z, sig = round_ttsvd(grown, eps=eps, forced=ranks + [None] * (d - 1 - k))
        S, r = sig[k], tt.ranks(Z)[k]
        while r < len(S) and S[r] > 0 and S[r - 1] / S[r] < ratio:
            r += 1
        ranks.append(r)
    return ranks


def _step_at_gap_ranks(ref, g, eps):
    grown, _, _ = ref.source(ref.transport(ref.cores))
    forced = _gap_ranks(grown, eps)
    ref.step(forced=forced)
    info = g.step(forced=forced)
    assert info["ranks"][1:-1] == tt.ranks(ref.cores)


@pytest.mark.parametrize("eps", [1e-3, 1e-4])
def test_small_2d_split_workload_at_resolvable_tolerance(ttsn, eps):
    """The same 4-core workload with every cut at a clear gap: every kept
    singular value is resolved by the Gram-SVD, parity 1e-10."""
    p = workloads.problem("small_2d", eps=eps)
    ref, g = _split_pair(ttsn, p)
    for _ in range(p["steps"]):
        _step_at_gap_ranks(ref, g, p["eps"])
    F = g.full().cpu().numpy()
    Rf = ref.full()
    assert np.linalg.norm(F - Rf) <= 1e-10 * np.linalg.norm(Rf)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_split_energy_conserved_periodic_free_ranks(ttsn, precision):
    p = workloads.problem("small_2d", n=(24, 20), n_theta=8, n_phi=16, eps=1e-4)
    prec = ttsn.TT_FP64 if precision == "fp64" else ttsn.TT_MIXED
    g = ttsn.TTSN.from_problem(p, layout=ttsn.TT_LAYOUT_SPLIT, precision=prec)
    _, _, t0 = g.energy()
    g.step(5)
    _, _, t1 = g.energy()
    assert abs(sum(t1) - sum(t0)) <= 1e-12 * sum(t0)


def test_split_mixed_matches_fp64_at_fp64_ranks(ttsn):
    n = (32, 32, 32)
    p = workloads.problem("small_2d", n=n, n_theta=8, n_phi=16, eps=1e-5, bc=VACUUM,
                          sigma_a=np.full(n, 5.0))
    g64 = ttsn.TTSN.from_problem(p, layout=ttsn.TT_LAYOUT_SPLIT)
    gmx = ttsn.TTSN.from_problem(p, layout=ttsn.TT_LAYOUT_SPLIT, precision=ttsn.TT_MIXED)
    assert g64.ranks() == gmx.ranks()
    for _ in range(6):
        info = g64.step()
        gmx.step(forced=info["ranks"][1:-1])
    E64, T64, _ = g64.energy()
    Em, Tm, _ = gmx.energy()
    assert float((Em - E64).abs().max() / E64.abs().max()) <= 1e-8
    assert float((Tm - T64).abs().max() / T64.abs().max()) <= 1e-8


def test_split_creation_holds_the_initial_field(ttsn):
    """tt_create in the split layout: d = ndim + 2 cores, the isotropic initial
    intensity held to the tolerance (the Gaussian pulse's T^4 has spatial rank
    at most 5: T = bg + g(x) g(y))."""
    p = workloads.problem("small_2d")
    g = ttsn.TTSN.from_problem(p, layout=ttsn.TT_LAYOUT_SPLIT)
    d, n = g.dims()
    assert d == 4 and n == [32, 32, 8, 16]
    r = g.ranks()
    assert r[0] == 1 and r[-1] == 1 and r[1] <= 5 and r[2:] == [1, 1, 1]
    I0 = p["c"] * p["a_r"] * p["Tr0"] ** 4 / (4 * np.pi)
    F = g.full().cpu().numpy()
    full0 = np.broadcast_to(I0[..., None, None], F.shape)
    # rounded to eps = 1e-8 (the background's T^4 term sits near that level)
    assert np.linalg.norm(F - full0) <= 2 * p["eps"] * np.linalg.norm(full0)


def test_split_argument_errors(ttsn):
    p = workloads.problem("small_2d", n=(6, 5), n_theta=4, n_phi=8)
    p2 = dict(p)
    p2["sigma_a"] = np.linspace(1.0, 2.0, 30).reshape(6, 5)
    with pytest.raises(ttsn.TTError) as e:
        ttsn.TTSN.from_problem(p2, layout=ttsn.TT_LAYOUT_SPLIT)
    assert e.value.status == -1
    with pytest.raises(ttsn.TTError) as e:
        ttsn.TTSN.from_problem(p, layout=2)
    assert e.value.status == -1
    g = ttsn.TTSN.from_problem(p, layout=ttsn.TT_LAYOUT_SPLIT)
    with pytest.raises(ttsn.TTError) as e:
        g.set_sources([(np.ones(30), np.ones(4), np.ones(8))])
    assert e.value.status == -6
    assert ttsn.lib.tt_tape_begin(g._h, ctypes.c_int(1)) == -6
    g.step()  # the handle stays usable
