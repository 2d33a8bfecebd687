"""Edge cases of the C-ABI on the GPU: empty and one-element inputs of the
kernel-level calls, and the argument errors the calls return instead of
faulting (invalid problem descriptions, forced ranks, source counts, short
output buffers)."""
import ctypes

import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ttsn():
    assert torch.cuda.is_available()
    import paper_2503_18056_gb300 as m

    return m


def _empty(shape):
    return torch.empty(shape, dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("which", ["gram", "gram_mixed"])
def test_gram_of_an_empty_matrix_is_zero(ttsn, which):
    """m = 0 rows: G = A^T A is the n x n zero matrix (A may be a null pointer)."""
    for n in (1, 5, 130):
        G = getattr(ttsn, which)(_empty((0, n)))
        torch.cuda.synchronize()
        assert G.shape == (n, n) and float(G.abs().max()) == 0.0


@pytest.mark.parametrize("which", ["gram", "gram_mixed"])
def test_gram_of_one_element(ttsn, which):
    for v in (3.0, -2.5e-100, 7.0e150):
        G = getattr(ttsn, which)(torch.tensor([[v]], dtype=torch.float64, device="cuda"))
        assert abs(float(G[0, 0]) - v * v) <= 1e-13 * v * v


def test_gemm_nt_mixed_empty_contraction_is_zero(ttsn):
    A, B = _empty((37, 0)), _empty((5, 0))
    C = ttsn.gemm_nt_mixed(A, B)
    torch.cuda.synchronize()
    assert C.shape == (37, 5) and float(C.abs().max()) == 0.0


def test_dgemm_empty_contraction_is_zero(ttsn):
    C = ttsn.dgemm(_empty((9, 0)), _empty((0, 4)))
    torch.cuda.synchronize()
    assert C.shape == (9, 4) and float(C.abs().max()) == 0.0


def test_syev_of_one_by_one(ttsn):
    lam, Vt, sweeps = ttsn.syev(torch.tensor([[4.5]], dtype=torch.float64, device="cuda"))
    assert float(lam[0]) == 4.5 and abs(float(Vt[0, 0])) == 1.0


@pytest.mark.parametrize("bad", [dict(n_theta=0), dict(n_phi=0), dict(c=0.0), dict(eps=-1.0),
                                 dict(rounds_per_step=3), dict(precision=7), dict(bc=5),
                                 dict(L=[0.0, 1.0])])
def test_invalid_problem_description_is_an_argument_error(ttsn, bad):
    p = workloads.problem("small_2d", n=(6, 5), n_theta=4, n_phi=8)
    with pytest.raises(ttsn.TTError) as e:
        ttsn.TTSN.from_problem(p, **bad)
    assert e.value.status == -1, e.value


def test_forced_rank_below_one_is_an_argument_error(ttsn):
    p = workloads.problem("small_2d", n=(6, 5), n_theta=4, n_phi=8)
    tt = ttsn.TTSN.from_problem(p)
    with pytest.raises(ttsn.TTError):
        tt.step(forced=[0, 1])
    with pytest.raises(ttsn.TTError):
        tt.round(forced=[1, 0])
    tt.step()  # the handle stays usable


def test_too_many_sources_is_an_argument_error(ttsn):
    p = workloads.problem("small_2d", n=(6, 5), n_theta=4, n_phi=8)
    tt = ttsn.TTSN.from_problem(p)
    src = [(np.ones(30), np.ones(4), np.ones(8))] * 17
    with pytest.raises(ttsn.TTError):
        tt.set_sources(src)
    tt.set_sources(src[:16])
    tt.step()


def test_to_full_with_a_short_buffer_is_refused(ttsn):
    p = workloads.problem("small_2d", n=(6, 5), n_theta=4, n_phi=8)
    tt = ttsn.TTSN.from_problem(p)
    short = _empty(6 * 5 * 4 * 8 - 1)
    st = ttsn.lib.tt_to_full(tt._h, ctypes.c_void_p(short.data_ptr()), short.numel())
    assert st == -7  # TT_ERR_TOO_LARGE: the buffer is too small, nothing written
    assert tt.full().shape == (6, 5, 4, 8)


def test_bounded_wait_runs_out_and_the_context_stays_usable(ttsn):
    """Failure detection without a GPU fault: a grid-barrier wait that can
    never complete gives up after its iteration limit, the kernel returns and
    the call reports TT_ERR_TIMEOUT; the next calls on the device succeed."""
    import time

    t0 = time.perf_counter()
    st = ttsn.lib.tt_wait_probe(None)
    elapsed = time.perf_counter() - t0
    assert st == -5, st  # TT_ERR_TIMEOUT
    assert elapsed < 30.0
    p = workloads.problem("small_2d", n=(6, 5), n_theta=4, n_phi=8)
    tt_ = ttsn.TTSN.from_problem(p)
    tt_.step(2)
    tt_.sync()
    G = ttsn.gram(torch.ones((10, 3), dtype=torch.float64, device="cuda"))
    assert float(G[0, 0]) == 10.0


def test_checkpoint_and_resume_continue_bit_for_bit(ttsn, tmp_path):
    """state_dict / load_state_dict (cores and T through tt_get_core,
    tt_set_cores, tt_set_T), saved with torch.save: a handle resumed from the
    checkpoint takes the same next steps as the original."""
    p = workloads.problem("small_2d", n=(16, 12), n_theta=4, n_phi=8, eps=1e-6)
    a = ttsn.TTSN.from_problem(p)
    a.step(3)
    path = tmp_path / "ckpt.pt"
    torch.save(a.state_dict(), path)
    a.step(2)
    b = ttsn.TTSN.from_problem(p)
    b.load_state_dict(torch.load(path))
    b.step(2)
    assert a.ranks() == b.ranks()
    assert torch.equal(a.full(), b.full())
    assert torch.equal(a.energy()[1], b.energy()[1])


def test_mismatched_state_is_refused_before_any_copy(ttsn):
    """load_state_dict / set_cores check the core count and every shape against
    the handle's grid before the library copies anything: a state from another
    grid, a short list or a misshaped core is a ValueError and the handle's
    state is unchanged."""
    p = workloads.problem("small_2d", n=(16, 12), n_theta=4, n_phi=8, eps=1e-6)
    a = ttsn.TTSN.from_problem(p)
    a.step(2)
    full0 = a.full().clone()
    good = a.state_dict()
    other = ttsn.TTSN.from_problem(workloads.problem("small_2d", n=(8, 8), n_theta=4, n_phi=8, eps=1e-6))
    other.step(1)
    cores = good["cores"]
    bad_states = [
        other.state_dict()["cores"],                      # another grid
        cores[:-1],                                       # a core short
        cores + [cores[-1]],                              # a core too many
        [cores[0][..., :-1]] + cores[1:],                 # r_1 disagrees with the next core
        [cores[0]] + [cores[1][:, :-1]] + cores[2:],      # wrong n_theta
        [c.reshape(-1) for c in cores],                   # not 3-dimensional
        cores[:-1] + [torch.cat([cores[-1], cores[-1]], dim=2)],  # last rank not 1
    ]
    for bad in bad_states:
        with pytest.raises(ValueError):
            a.set_cores(bad)
        with pytest.raises(ValueError):
            a.load_state_dict({"cores": bad, "T": good["T"]})
    assert torch.equal(a.full(), full0)
    a.load_state_dict(good)
    assert torch.equal(a.full(), full0)


def test_run_log_records_each_step(ttsn, tmp_path):
    """TTSN.run: one JSON line per step with the step's ranks (as step()
    reports them), t = step dt, the compression factor of those ranks, and
    total energy conserved on a periodic grid."""
    import json

    p = workloads.problem("small_2d", n=(16, 12), n_theta=4, n_phi=8, eps=1e-6)
    a = ttsn.TTSN.from_problem(p)
    b = ttsn.TTSN.from_problem(p)
    path = tmp_path / "run.jsonl"
    recs = a.run(3, log=str(path))
    lines = [json.loads(x) for x in path.read_text().splitlines()]
    assert lines == recs and [r["step"] for r in recs] == [1, 2, 3]
    for r in recs:
        info = b.step()
        assert r["ranks"] == info["ranks"] and r["discarded"] == info["discarded"]
        assert r["t"] == r["step"] * p["dt"] and r["ms"] > 0
        assert r["compression"] == ttsn.compression_factor([16 * 12, 4, 8], info["ranks"])
    e0 = recs[0]["E_total"]
    assert all(abs(r["E_total"] - e0) <= 1e-12 * e0 for r in recs)
    assert a.compression() == recs[-1]["compression"]


@pytest.mark.parametrize("where", ["T", "theta_core"])
def test_non_finite_state_is_reported_and_a_checkpoint_restores(ttsn, where):
    """Failure detection without a device fault: a NaN planted on the host in
    the temperature (it reaches the emission column of the spatial core, so
    the left Gram and its eigenvalues) or in the theta core (it reaches a
    right Gram, so the pivoted Cholesky) makes the step return
    TT_ERR_NONFINITE instead of rounding to the zero tensor; reloading a
    checkpoint restores a handle that then steps exactly like an untouched
    twin."""
    p = workloads.problem("small_2d", n=(16, 12), n_theta=4, n_phi=8, eps=1e-6)
    a = ttsn.TTSN.from_problem(p)
    b = ttsn.TTSN.from_problem(p)
    a.step(2)
    b.step(2)
    ckpt = a.state_dict()
    if where == "T":
        T = ckpt["T"].clone()
        T[7] = float("nan")
        a.set_T(T)
    else:
        cores = [c.clone() for c in ckpt["cores"]]
        cores[1][0, 1, 0] = float("inf")
        a.set_cores(cores)
    with pytest.raises(ttsn.TTError) as e:
        a.step()
    assert e.value.status == -8
    a.load_state_dict(ckpt)
    a.step(2)
    b.step(2)
    assert torch.equal(a.full(), b.full())
    assert torch.equal(a.energy()[1], b.energy()[1])


@pytest.mark.parametrize("n", [40, 500])
def test_pchol_of_a_non_finite_diagonal_is_reported(ttsn, n):
    """One CTA (n <= 384) and the cooperative multi-CTA kernel both stop before
    factorising when the diagonal holds NaN or Inf."""
    rng = np.random.default_rng(n)
    X = rng.standard_normal((n + 3, n))
    G = X.T @ X
    for bad in (float("nan"), float("inf")):
        H = G.copy()
        H[n // 2, n // 2] = bad
        with pytest.raises(ttsn.TTError) as e:
            ttsn.pchol(torch.tensor(H, device="cuda"))
        assert e.value.status == -8
    W, k = ttsn.pchol(torch.tensor(G, device="cuda"))
    assert k == n


def test_sweep_limit_reached_is_reported_and_the_handle_stays_usable(ttsn):
    """The eigensolver's sweep limit as a failure the host can make happen: a
    limit of one sweep on a matrix that needs several returns
    TT_ERR_NOT_CONVERGED (kernel level and inside a step), nothing faults, and
    with the default limit back the same handle steps on normally."""
    rng = np.random.default_rng(3)
    B = rng.standard_normal((96, 96))
    G = torch.as_tensor(B @ B.T, device="cuda")
    with pytest.raises(ttsn.TTError) as e:
        ttsn.syev(G, max_sweeps=1)
    assert e.value.status == -4
    lam, Vt, sweeps = ttsn.syev(G)
    assert 1 < sweeps <= 40
    with pytest.raises(ttsn.TTError):
        ttsn.syev(G, max_sweeps=0)
    p = workloads.problem("small_2d", n=(16, 12), n_theta=4, n_phi=8, eps=1e-6)
    g = ttsn.TTSN.from_problem(p)
    g.step(3)
    g.set_max_sweeps(1)
    with pytest.raises(ttsn.TTError) as e:
        g.step()
    assert e.value.status == -4
    with pytest.raises(ttsn.TTError):
        g.set_max_sweeps(41)
    g.set_max_sweeps(40)
    # the failed step left a valid (less accurate) state; stepping resumes
    info = g.step()
    assert info["ranks"][0] == 1 and info["sweeps"] > 1
    assert torch.isfinite(g.full()).all()
