"""GPU TT-S_N step (tt_sn_step) against the FP64 oracle: untruncated step equal
to the dense step, full step at the oracle's ranks, conservation, and sampled
outputs of the 3D 128^3 workload in the launch configuration the bench uses."""
import numpy as np
import pytest

import workloads
from oracle import tt
from oracle.dense import DenseSN
from oracle.rounding import round_ttsvd
from oracle.ttstep import PERIODIC, VACUUM, TTSN as OracleTTSN

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ttsn():
    import torch

    assert torch.cuda.is_available()
    import paper_2503_18056_gb300 as m

    return m


def _args(n, nt, npf, bc, seed):
    f = workloads.random_fields(n, seed)
    dt = 0.4 * min(1.0 / m for m in n)
    return dict(n=n, L=[1.0] * len(n), n_theta=nt, n_phi=npf, c=1.0, a_r=1.0, dt=dt,
                bc=[bc] * len(n), sigma_a=f["sigma_a"].reshape(-1), cv=f["cv"].reshape(-1),
                T0=f["T0"].reshape(-1))


@pytest.mark.parametrize("n,bc", [((13,), VACUUM), ((9, 7), PERIODIC), ((9, 7), VACUUM),
                                  ((5, 4, 6), PERIODIC), ((6, 5, 4), VACUUM)])
@pytest.mark.parametrize("source", [False, True])
def test_untruncated_step_equals_dense(ttsn, n, bc, source):
    nt, npf = 4, 6
    a = _args(n, nt, npf, bc, seed=21)
    nc = int(np.prod(n))
    cores = workloads.random_positive_tt([nc, nt, npf], [3, 2], seed=22)
    d = DenseSN(n, a["L"], nt, npf, a["c"], a["a_r"], a["dt"], a["bc"],
                a["sigma_a"].reshape(n), a["cv"].reshape(n), a["T0"].reshape(n),
                tt.full(cores).reshape(tuple(n) + (nt, npf)))
    g = ttsn.TTSN(eps=0.0, **a)
    g.set_cores(cores)
    flags = ttsn.TT_STEP_NO_ROUND | (0 if source else ttsn.TT_STEP_NO_SOURCE)
    for _ in range(2):
        d.step(with_source=source)
        info = g.step(flags=flags)
    F = g.full().cpu().numpy()
    assert np.abs(F - d.I).max() <= 1e-12 * np.abs(d.I).max()
    k = 1 + 2 * len(n)
    s = 1 if source else 0
    assert info["ranks"][1] == k * (k * 3 + s) + s
    _, T, _ = g.energy()
    assert np.abs(T.cpu().numpy() - d.T.reshape(-1)).max() <= 1e-12


def _oracle(p, rounding="ttsvd", **kw):
    # The rounded tensor at given ranks has a plain definition, the sequential
    # truncated SVD of the unfoldings (TT-SVD, App. A.1), which the Gram-SVD
    # truncation of App. A.2 reaches in exact arithmetic; the oracle's TT-SVD is
    # the parity reference, its rank choices are replayed on the GPU.
    I0 = p["c"] * p["a_r"] * p["Tr0"] ** 4 / (4 * np.pi)
    return OracleTTSN(p["n"], p["L"], p["n_theta"], p["n_phi"], p["c"], p["a_r"], p["dt"], p["bc"],
                      p["sigma_a"], p["cv"], p["T0"],
                      OracleTTSN.isotropic_cores(I0.reshape(-1), p["n_theta"], p["n_phi"]),
                      eps=p["eps"], max_rank=p.get("max_rank"), rounding=rounding, **kw)


def _forced(ref):
    return [r for rk in ref.last_ranks for r in rk]


@pytest.mark.parametrize("rounds", [1, 2])
@pytest.mark.parametrize("bc", [PERIODIC, VACUUM])
def test_step_matches_oracle_at_oracle_ranks(ttsn, rounds, bc):
    p = workloads.problem("small_2d", n=(16, 12), n_theta=4, n_phi=8, eps=1e-5, bc=bc)
    ref = _oracle(p, rounds_per_step=rounds)
    g = ttsn.TTSN.from_problem(p, rounds_per_step=rounds)
    for _ in range(4):
        ref.step()
        info = g.step(forced=_forced(ref))
        assert info["ranks"][1:-1] == tt.ranks(ref.cores)
    F = g.full().cpu().numpy()
    R = ref.full()
    assert np.linalg.norm(F - R) <= 1e-10 * np.linalg.norm(R)
    E, T, _ = g.energy()
    assert np.abs(T.cpu().numpy() - ref.T).max() <= 1e-12
    assert np.abs(E.cpu().numpy() - ref.energy_density()).max() <= 1e-10 * np.abs(ref.energy_density()).max()


EPS_MACH = np.finfo(float).eps


@pytest.mark.parametrize("eps", [1e-8, 1e-6])
def test_small_2d_workload_ten_steps(ttsn, eps):
    # 2D 32x32, 8x16 ordinates, periodic, eps = 1e-8 (and 1e-6), 10 steps; the
    # oracle's TT-SVD picks the ranks.  The cut then lies at (or near) the Gram-SVD
    # resolution:
    # Gram eigenvalues carry absolute errors ~ eps_mach lambda_max (App. A.4), so
    # singular values are resolved only to sqrt(R eps_mach) sigma_max per bond
    # (R the grown rank).  Each step may therefore differ from the exact
    # truncation by up to 2 sqrt(d-1) sqrt(eps^2 + R eps_mach) ||X||, and the
    # upwind step is L2-contractive at this CFL, so differences add up.
    p = workloads.problem("small_2d", eps=eps)
    ref = _oracle(p)
    g = ttsn.TTSN.from_problem(p)
    _, _, tot0 = g.energy()
    budget = 0.0
    for _ in range(p["steps"]):
        ref.step()
        info = g.step(forced=_forced(ref))
        R = max(info["grown"])
        budget += 2 * np.sqrt(2) * np.sqrt(p["eps"] ** 2 + R * EPS_MACH)
    F = g.full().cpu().numpy()
    Rf = ref.full()
    err = np.linalg.norm(F - Rf) / np.linalg.norm(Rf)
    assert err < budget, (err, budget)
    _, T, tot = g.energy()
    assert np.abs(T.cpu().numpy() - ref.T).max() < budget * np.abs(ref.T).max()
    # periodic: total energy conserved through transport, source and rounding
    assert abs(sum(tot) - sum(tot0)) <= 1e-12 * sum(tot0)
    print("small_2d eps %.0e 10 steps: rel. difference to the TT-SVD oracle %.2e (yardstick %.2e)" % (eps, err, budget))


def _gap_ranks(sig, ranks, ratio=1.05):
    # the pulse problem is symmetric (x <-> y, phi -> -phi), so singular values
    # come in exactly equal pairs; a cut inside a pair has no unique answer.
    # Move each cut up to the next index with a clear gap.
    out = []
    for S, r in zip(sig, ranks):
        while r < len(S) and S[r] > 0 and S[r - 1] / S[r] < ratio:
            r += 1
        out.append(r)
    return out


def _resolution_bound(sig, ranks):
    """Derived per-step bound of the Gram-SVD truncation against TT-SVD at the
    given cuts (App. A.4: Gram eigenvalues carry absolute errors ~ eps_mach
    lambda_max).  A kept component with singular value sigma_r then carries a
    relative error eps_mach sigma_1^2 / sigma_r^2, and its mixing with the
    first discarded one (relative gap 1 - (sigma_{r+1}/sigma_r)^2) moves the
    rounded tensor by about eps_mach (sigma_1 / sigma_r) / gap relative to
    ||X||; 4 covers the Gram's own accumulation constant.  Summed over the
    bonds."""
    b = 0.0
    for S, r in zip(sig, ranks):
        r = min(r, len(S))
        gap = 1.0 - (S[r] / S[r - 1]) ** 2 if r < len(S) else 1.0
        b += 4.0 * EPS_MACH * (S[0] / S[r - 1]) / gap
    return b


@pytest.mark.parametrize("eps", [1e-4, 1e-5, 1e-6, 1e-8])
def test_small_2d_workload_cuts_at_gaps(ttsn, eps):
    # The 32x32 workload with every cut moved to the next clear gap of the
    # oracle's singular values, which separates the two sources of difference
    # seen at free cuts: cuts inside the symmetric pairs, and the Gram
    # resolution.  The resolution bound (above) grows with sigma_1 / sigma_cut;
    # summed over the 10 steps it is 2.5e-10 (eps = 1e-4), 1.3e-9 (1e-5) and
    # 8.3e-9 (1e-6), and the test asserts the larger of it and 1e-10.  Measured:
    # 1e-13 .. 2e-11, 5e-13 .. 8e-13 and 9e-13 .. 5e-10; the last varies with
    # the trajectory, because one step of this run (step 7, cut at
    # sigma ~ 7e-7 sigma_1) moves by 5e-10 from the oracle's own state with
    # every revision of the eigensolver.  At the stated eps = 1e-8 the cut
    # (sigma ~ 1e-8 sigma_1) lies at the resolution itself and the pivoted
    # Cholesky of G_B can resolve fewer directions than the oracle keeps (rank
    # 53 against 54 at one bond): the free-cut budget applies (measured
    # 4e-8 .. 7e-8).
    p = workloads.problem("small_2d", eps=eps)
    ref = _oracle(p)
    g = ttsn.TTSN.from_problem(p)
    bound = 0.0
    for _ in range(p["steps"]):
        grown, _, _ = ref.source(ref.transport(ref.cores))
        Z, sig = round_ttsvd(grown, eps=p["eps"])
        forced = _gap_ranks(sig, tt.ranks(Z))
        ref.step(forced=forced)
        info = g.step(forced=forced)
        if eps >= 1e-6:
            assert info["ranks"][1:-1] == tt.ranks(ref.cores)
        else:
            # below the resolution a forced rank can exceed the directions the
            # right Gram resolves (its pivoted Cholesky stops at eps_mach of
            # the largest pivot); the GPU then keeps those it resolves
            assert all(a <= b for a, b in zip(info["ranks"][1:-1], tt.ranks(ref.cores)))
        if eps >= 1e-6:
            bound += _resolution_bound(sig, forced)
        else:
            bound += 2 * np.sqrt(2) * np.sqrt(p["eps"] ** 2 + max(info["grown"]) * EPS_MACH)
    F = g.full().cpu().numpy()
    Rf = ref.full()
    err = np.linalg.norm(F - Rf) / np.linalg.norm(Rf)
    print("small_2d eps %.0e, cuts at gaps: rel. difference to the TT-SVD oracle %.2e (bound %.2e)"
          % (eps, err, bound))
    assert err <= max(1e-10, bound), (err, bound)


def test_energy_conserved_periodic_free_ranks(ttsn):
    p = workloads.problem("small_2d", n=(24, 24), n_theta=8, n_phi=16, eps=1e-4)
    g = ttsn.TTSN.from_problem(p)
    _, _, t0 = g.energy()
    g.step(5)
    _, _, t1 = g.energy()
    assert abs(sum(t1) - sum(t0)) <= 1e-12 * sum(t0)


def test_equilibrium_fixed_point(ttsn):
    n = (10, 8)
    nc = 80
    T = 0.9
    g = ttsn.TTSN(n=n, L=[1, 1], n_theta=4, n_phi=8, sigma_a=np.full(nc, 5.0), cv=np.ones(nc),
                  T0=np.full(nc, T), Tr0=np.full(nc, T), dt=0.02, bc=PERIODIC, eps=1e-10)
    info = g.step(3)
    assert info["ranks"] == [1, 1, 1, 1]
    assert np.abs(g.full().cpu().numpy() - T ** 4 / (4 * np.pi)).max() < 1e-15
    _, TT, _ = g.energy()
    assert np.abs(TT.cpu().numpy() - T).max() < 1e-14


def test_blob_3d_full_size_sampled(ttsn):
    # 3D 128^3 cells, 32x64 ordinates, vacuum, eps = 1e-6: the first two steps
    # at full size, compared with the oracle on sampled cells and in the totals
    p = workloads.problem("blob_3d")
    ref = _oracle(p)
    g = ttsn.TTSN.from_problem(p)
    for _ in range(2):
        ref.step()
        info = g.step(forced=_forced(ref))
    assert info["ranks"][1:-1] == tt.ranks(ref.cores)
    E, T, tot = g.energy()
    E, T = E.cpu().numpy(), T.cpu().numpy()
    Er = ref.energy_density()
    rng = np.random.default_rng(0)
    idx = np.concatenate([rng.integers(0, E.size, 4096), np.argsort(Er)[-256:]])
    assert np.abs(E[idx] - Er[idx]).max() <= 1e-10 * np.abs(Er).max()
    assert np.abs(T[idx] - ref.T[idx]).max() <= 1e-12
    dV = 1.0 / E.size
    assert abs(tot[0] - Er.sum() * dV) <= 1e-10 * Er.sum() * dV


def test_state_through_host_memory(ttsn):
    # set_cores / set_T read float64 CPU tensors (pinned or pageable) straight
    # from host memory and cores(into=...) writes into caller buffers: the
    # steps that follow are bit for bit those from the device-held state
    import torch

    p = workloads.problem("small_2d", n=(16, 12), n_theta=4, n_phi=8, eps=1e-6)
    g = ttsn.TTSN.from_problem(p)
    g.step(3)
    dev = [c.clone() for c in g.cores()]
    T = g.energy()[1].clone()
    pinned = [torch.empty(c.numel() + 5, dtype=torch.float64).pin_memory() for c in dev]
    host = g.cores(into=pinned)
    for h, d in zip(host, dev):
        assert h.device.type == "cpu" and h.shape == d.shape and torch.equal(h, d.cpu())
    with pytest.raises(ValueError):
        g.cores(into=[torch.empty(1, dtype=torch.float64)] * len(dev))
    runs = []
    for cores, temp in ((dev, T), (host, T.cpu().pin_memory()), ([d.cpu() for d in dev], T.cpu())):
        h = ttsn.TTSN.from_problem(p)
        h.set_cores(cores)
        h.set_T(temp)
        h.step(2)
        runs.append((h.full().cpu(), h.energy()[1].cpu()))
    for F, Tn in runs[1:]:
        assert torch.equal(F, runs[0][0]) and torch.equal(Tn, runs[0][1])
