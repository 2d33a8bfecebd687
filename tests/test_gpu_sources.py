"""Fixed external sources on the GPU (I* = L I + c dt S, each source one more
rank-one term): the untruncated step against the dense oracle, the rounded
step against the oracle's TT-SVD stepper at its ranks, the energy balance on a
periodic domain, the precision form against FP64, and the crossing-beam
workload at full size (256^2 cells, 64 x 128 ordinates)."""
import numpy as np
import pytest
import torch

import workloads
from oracle import angles, tt
from oracle.dense import DenseSN
from oracle.ttstep import PERIODIC, VACUUM, TTSN as OracleTTSN

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ttsn():
    assert torch.cuda.is_available()
    import paper_2503_18056_gb300 as m

    return m


def _sources(n, nt, npf, seed, count=2):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        x = rng.uniform(0.0, 1.0, n) * (rng.uniform(size=n) < 0.3)
        out.append((x, rng.uniform(0.0, 2.0, nt), rng.uniform(0.0, 2.0, npf)))
    return out


def _args(n, nt, npf, bc, seed):
    f = workloads.random_fields(n, seed)
    return dict(n=n, L=[1.0] * len(n), n_theta=nt, n_phi=npf, c=1.0, a_r=1.0,
                dt=0.4 * min(1.0 / m for m in n), bc=[bc] * len(n),
                sigma_a=f["sigma_a"].reshape(-1), cv=f["cv"].reshape(-1), T0=f["T0"].reshape(-1))


@pytest.mark.parametrize("n,bc", [((9, 7), VACUUM), ((5, 4, 6), PERIODIC), ((13,), VACUUM)])
@pytest.mark.parametrize("count", [1, 3])
def test_untruncated_step_with_sources_equals_dense(ttsn, n, bc, count):
    nt, npf = 4, 6
    a = _args(n, nt, npf, bc, 31)
    src = _sources(n, nt, npf, 32, count)
    nc = int(np.prod(n))
    cores = workloads.random_positive_tt([nc, nt, npf], [3, 2], seed=33)
    d = DenseSN(n, a["L"], nt, npf, a["c"], a["a_r"], a["dt"], a["bc"],
                a["sigma_a"].reshape(n), a["cv"].reshape(n), a["T0"].reshape(n),
                tt.full(cores).reshape(tuple(n) + (nt, npf)), sources=src)
    g = ttsn.TTSN(eps=0.0, **a)
    g.set_cores(cores)
    g.set_sources([(x.reshape(-1), th, ph) for x, th, ph in src])
    for _ in range(2):
        d.step()
        info = g.step(flags=ttsn.TT_STEP_NO_ROUND)
    k = 1 + 2 * len(n)
    assert info["ranks"][1] == k * (k * 3 + count + 1) + count + 1
    F = g.full().cpu().numpy()
    assert np.abs(F - d.I).max() <= 1e-12 * np.abs(d.I).max()
    _, T, _ = g.energy()
    assert np.abs(T.cpu().numpy() - d.T.reshape(-1)).max() <= 1e-12 * np.abs(d.T).max()


@pytest.mark.parametrize("rounds", [1, 2])
def test_rounded_step_with_sources_matches_oracle_at_its_ranks(ttsn, rounds):
    # eps = 1e-4: the Gram-SVD resolves a retained component of size sigma to
    # about eps_mach (sigma_max / sigma)^2 of itself (App. A.4), so cuts near
    # 1e-5 sigma_max leave ~2e-11 per bond and step against TT-SVD (measured
    # 1.3e-10 after 6 steps at eps = 1e-5); at 1e-4 that is 100x smaller.
    p = workloads.crossing_beams(n=(24, 20), n_theta=8, n_phi=16, eps=1e-4, max_rank=0)
    I0 = p["c"] * p["a_r"] * p["Tr0"] ** 4 / (4 * np.pi)
    ref = OracleTTSN(p["n"], p["L"], p["n_theta"], p["n_phi"], p["c"], p["a_r"], p["dt"], p["bc"],
                     p["sigma_a"], p["cv"], p["T0"],
                     OracleTTSN.isotropic_cores(I0.reshape(-1), p["n_theta"], p["n_phi"]),
                     eps=p["eps"], rounding="ttsvd", rounds_per_step=rounds, sources=p["sources"])
    g = ttsn.TTSN.from_problem(p, rounds_per_step=rounds, max_rank=0)
    for _ in range(6):
        ref.step()
        info = g.step(forced=[r for rk in ref.last_ranks for r in rk])
        assert info["ranks"][1:-1] == tt.ranks(ref.cores)
    F = g.full().cpu().numpy()
    R = ref.full()
    assert np.linalg.norm(F - R) <= 1e-10 * np.linalg.norm(R)
    _, T, _ = g.energy()
    assert np.abs(T.cpu().numpy() - ref.T).max() <= 1e-10 * np.abs(ref.T).max()


def _power(p, sources):
    g = angles.grid(p["n_theta"], p["n_phi"])
    dO = angles.solid_angles(g)
    dV = float(np.prod([p["L"][a] / p["n"][a] for a in range(len(p["n"]))]))
    return sum(float(np.sum(x)) * dV * float(th @ dO @ ph) for x, th, ph in sources)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_energy_balance_with_sources_periodic(ttsn, precision):
    n, nt, npf = (20, 18), 8, 16
    a = _args(n, nt, npf, PERIODIC, 41)
    src = _sources(n, nt, npf, 42)
    prec = ttsn.TT_FP64 if precision == "fp64" else ttsn.TT_MIXED
    g = ttsn.TTSN(eps=1e-6, precision=prec, **a)
    g.set_sources([(x.reshape(-1), th, ph) for x, th, ph in src])
    power = _power(dict(n=n, L=a["L"], n_theta=nt, n_phi=npf), src)
    _, _, tot0 = g.energy()  # totals are volume integrals (sum dV)
    e0 = sum(tot0)
    for m in range(1, 6):
        g.step()
        _, _, tot = g.energy()
        want = e0 + m * a["dt"] * power
        assert abs(sum(tot) - want) <= 1e-12 * want


def test_mixed_matches_fp64_with_sources_at_fp64_ranks(ttsn):
    p = workloads.crossing_beams(n=(64, 64), n_theta=16, n_phi=32, max_rank=32)
    g64 = ttsn.TTSN.from_problem(p)
    gmx = ttsn.TTSN.from_problem(p, precision=ttsn.TT_MIXED)
    for _ in range(40):
        info = g64.step()
        gmx.step(forced=info["ranks"][1:-1])
    E64, T64, _ = g64.energy()
    Em, Tm, _ = gmx.energy()
    # The bound is the precision form's stated error target, 1e-6 relative to
    # the FP64 run at equal ranks.  A tighter a-priori bound does not follow
    # from the split's per-term error (<= 8 2^-48 m of the column scales,
    # pinned in test_gpu_mixed): propagated through a Gram-SVD truncation it
    # acts like a larger unit roundoff, and the Gram resolution argument
    # (sqrt of the relative Gram error per bond and step) gives ~1e-5 over
    # these 40 steps, looser than the target.  Measured 2e-13 (E) and
    # 2e-12 (T, which sits near its 1e-3 background).
    dE = float((Em - E64).abs().max() / E64.abs().max())
    dT = float((Tm - T64).abs().max() / T64.abs().max())
    print("precision form vs FP64 with sources, 40 steps: E %.1e, T %.1e" % (dE, dT))
    assert dE <= 1e-6 and dT <= 1e-6


@pytest.fixture(scope="module")
def beams_full(ttsn):
    """The crossing-beam workload at full size: 60 FP64 steps, then the same
    steps in the precision form at the FP64 ranks.  Periodic instead of
    vacuum: within 60 steps no beam comes near a face, and without the faces
    the energy balance is exact (with vacuum faces the truncation's noise at
    the boundary leaves the box, ~1e-5 of the added energy)."""
    p = workloads.crossing_beams()
    p["bc"] = [PERIODIC, PERIODIC]
    g64 = ttsn.TTSN.from_problem(p)
    gmx = ttsn.TTSN.from_problem(p, precision=ttsn.TT_MIXED)
    _, _, tot0 = g64.energy()
    ranks = []
    for _ in range(60):
        info = g64.step()
        ranks.append(info["ranks"][1:-1])
        gmx.step(forced=ranks[-1])
    return p, g64, gmx, tot0, ranks


def test_crossing_beams_full_size_energy_balance(ttsn, beams_full):
    """sum(E + C_v T) dV grows by the sources' power times the elapsed time."""
    p, g64, gmx, tot0, ranks = beams_full
    added = 60 * p["dt"] * _power(p, p["sources"])
    for g in (g64, gmx):
        _, _, tot = g.energy()
        assert abs((sum(tot) - sum(tot0)) - added) <= 1e-9 * added
    assert max(max(r) for r in ranks) <= p["max_rank"]


def test_crossing_beams_full_size_mixed_error(ttsn, beams_full):
    """The precision form stays within 1e-6 (stated bound) of FP64 in E and T."""
    p, g64, gmx, tot0, ranks = beams_full
    E64, T64, _ = g64.energy()
    Em, Tm, _ = gmx.energy()
    assert float((Em - E64).abs().max() / E64.abs().max()) <= 1e-6
    assert float((Tm - T64).abs().max() / T64.abs().max()) <= 1e-6
