"""Adjoint form on the GPU: the escape-energy objective and its gradient with
respect to sigma_a (reverse sweep with the rounding's factors frozen),
checked against the dense oracle's exact gradient, central finite differences
of the GPU forward at the taped ranks, checkpointed replays and the autograd
wrapper."""
import numpy as np
import pytest
import torch

from oracle.adjoint import escape_energy, escape_energy_and_gradient
from oracle.dense import DenseSN
from workloads import gaussian_pulse, gaussian_random_field, grf_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ttsn():
    assert torch.cuda.is_available()
    import paper_2503_18056_gb300 as m

    return m


def _problem(n=(12, 12), n_theta=4, n_phi=8, steps=6, eps=1e-10, seed=0):
    """A small random-field problem whose radiation reaches the vacuum boundary
    within the run (hot background, wide pulse)."""
    p = grf_problem(n=n, n_theta=n_theta, n_phi=n_phi, steps=steps, eps=eps, seed=seed)
    T0 = gaussian_pulse(p["n"], p["L"], 1.0, 0.2, 0.3)
    p["T0"], p["Tr0"] = T0, T0.copy()
    return p


def _make_dense(p):
    def make(sig):
        I0 = p["c"] * p["a_r"] * p["Tr0"] ** 4 / (4 * np.pi)
        I0 = np.broadcast_to(I0[..., None, None], p["n"] + (p["n_theta"], p["n_phi"]))
        return DenseSN(p["n"], p["L"], p["n_theta"], p["n_phi"], p["c"], p["a_r"], p["dt"],
                       p["bc"], sig, p["cv"], p["T0"], I0)
    return make


def _taped_run(tt_mod, p, sigma=None, every=1, forced=None, infos=None):
    """Run p's steps with the tape on; returns (handle, per-step output ranks).
    infos (a list, optional) receives each step's rounding diagnostics."""
    kw = tt_mod.TTSN.problem_kwargs(p)
    if sigma is not None:
        kw["sigma_a"] = sigma
    tt = tt_mod.TTSN(**kw)
    tt.tape_begin(every)
    ranks = []
    for m in range(p["steps"]):
        info = tt.step(1, forced=None if forced is None else forced[m])
        ranks.append(list(info["ranks"][1:3]))
        if infos is not None:
            infos.append(info)
    return tt, ranks


def test_escape_energy_matches_dense_oracle(ttsn):
    p = _problem()
    tt, _ = _taped_run(ttsn, p)
    q_gpu, m = tt.escape_energy()
    q_ref = escape_energy(_make_dense(p), p["sigma_a"], p["steps"])
    assert m == p["steps"]
    assert abs(q_gpu - q_ref) <= 1e-9 * abs(q_ref)


@pytest.mark.parametrize("n,bc", [((12, 12), None), ((10, 14), "mixed"), ((6, 5, 7), None)])
def test_gradient_matches_dense_oracle(ttsn, n, bc):
    """Below resolution (eps = 1e-10) the truncated directions carry nothing, so
    the frozen-factor gradient is the dense scheme's exact gradient."""
    p = _problem(n=n, steps=5)
    if bc == "mixed":  # periodic in x: faces only in y
        p["bc"] = [ttsn.TT_BC_PERIODIC, ttsn.TT_BC_VACUUM]
    tt, _ = _taped_run(ttsn, p)
    q_gpu, g_gpu = tt.escape_gradient()
    q_ref, g_ref = escape_energy_and_gradient(_make_dense(p), p["sigma_a"], p["steps"])
    g_ref = g_ref.reshape(-1)
    scale = np.abs(g_ref).max()
    assert scale > 0
    assert abs(q_gpu - q_ref) <= 1e-9 * abs(q_ref)
    np.testing.assert_allclose(g_gpu.cpu().numpy(), g_ref, rtol=0, atol=1e-8 * scale)


def test_gradient_central_fd_at_taped_ranks(ttsn):
    """Central differences of the GPU forward (ranks forced to the taped ones)
    on 16 seeded cells.  h = 1e-4 sigma_i: below that the forward's rounding
    noise (about 1e-13 of Q) over 2h dominates the difference."""
    p = _problem(eps=1e-6)
    tt, ranks = _taped_run(ttsn, p)
    _, g = tt.escape_gradient()
    g = g.cpu().numpy()
    scale = np.abs(g).max()
    sig = p["sigma_a"].reshape(-1)
    rng = np.random.default_rng(7)
    nx, ny = p["n"]
    edge = [0 * ny + 5, (nx - 1) * ny + 3]  # two boundary cells
    cells = list(rng.choice(sig.size, 14, replace=False)) + edge
    for i in cells:
        h = 1e-4 * sig[i]
        qs = []
        for sgn in (1.0, -1.0):
            s2 = sig.copy()
            s2[i] += sgn * h
            t2, _ = _taped_run(ttsn, p, sigma=s2, forced=ranks)
            qs.append(t2.escape_energy()[0])
        fd = (qs[0] - qs[1]) / (2 * h)
        assert abs(fd - g[i]) <= 2e-5 * scale, (i, fd, g[i], scale)


@pytest.mark.parametrize("every", [2, 4, 6])
def test_checkpointed_replay_matches_full_tape(ttsn, every):
    p = _problem(eps=1e-6)
    tt1, _ = _taped_run(ttsn, p, every=1)
    q1, g1 = tt1.escape_gradient()
    tt2, _ = _taped_run(ttsn, p, every=every)
    q2, g2 = tt2.escape_gradient()
    assert q1 == q2
    scale = float(g1.abs().max())
    assert float((g1 - g2).abs().max()) <= 1e-13 * scale


def test_state_after_adjoint_is_the_last_step(ttsn):
    p = _problem(eps=1e-6)
    tt, ranks = _taped_run(ttsn, p, every=3)
    full0 = tt.full().clone()
    _, T0, _ = tt.energy()
    tt.escape_gradient()
    assert tt.ranks()[1:3] == ranks[-1]
    assert torch.equal(tt.full(), full0)
    _, T1, _ = tt.energy()
    assert torch.equal(T0, T1)
    tt.step(1)  # the handle keeps stepping after the reverse sweep


def test_autograd_function(ttsn):
    p = _problem(eps=1e-6)
    kw = ttsn.TTSN.problem_kwargs(p)
    sig = torch.tensor(kw.pop("sigma_a"), dtype=torch.float64, device="cuda", requires_grad=True)
    q = ttsn.escape_energy(sig, kw, p["steps"], 2)
    (g,) = torch.autograd.grad(2.0 * q, sig)
    tt, _ = _taped_run(ttsn, p)
    q_ref, g_ref = tt.escape_gradient()
    assert float(q.detach()) == q_ref
    assert float((g - 2.0 * g_ref).abs().max()) <= 1e-13 * float(g_ref.abs().max())


def test_autograd_with_sigma_on_the_grid_shape(ttsn):
    """sigma_a given with the grid's shape (n_x, n_y): the gradient comes back
    in that shape, and a second backward through the released tape is a clear
    RuntimeError."""
    p = _problem(eps=1e-6)
    kw = ttsn.TTSN.problem_kwargs(p)
    flat = np.asarray(kw.pop("sigma_a"), dtype=np.float64).reshape(-1)
    sig = torch.tensor(flat.reshape(p["n"]), dtype=torch.float64, device="cuda", requires_grad=True)
    q = ttsn.escape_energy(sig, kw, p["steps"], 2)
    (g,) = torch.autograd.grad(q, sig, retain_graph=True)
    assert g.shape == sig.shape
    tt, _ = _taped_run(ttsn, p)
    _, g_ref = tt.escape_gradient()
    assert float((g.reshape(-1) - g_ref).abs().max()) <= 1e-13 * float(g_ref.abs().max())
    with pytest.raises(RuntimeError, match="released"):
        torch.autograd.grad(q, sig)


def test_tape_argument_and_state_errors(ttsn):
    p = _problem(eps=1e-6, steps=2)
    tt = ttsn.TTSN.from_problem(p)
    with pytest.raises(ttsn.TTError):
        tt.tape_begin(0)
    with pytest.raises(ttsn.TTError):
        tt.escape_gradient()  # nothing taped
    tt.set_precision(ttsn.TT_MIXED)
    with pytest.raises(ttsn.TTError):
        tt.tape_begin(1)
    tt.set_precision(ttsn.TT_FP64)
    tt.tape_begin(1)
    tt.step(1)
    tt.set_T(p["T0"].reshape(-1))  # a state change outside a step ends the tape
    with pytest.raises(ttsn.TTError):
        tt.escape_gradient()


@pytest.fixture(scope="module")
def full_size(ttsn):
    """The 128^2 x (32 x 64), 20-step, eps 1e-6 random-field run, taped with
    checkpoints every 5 steps: (problem, taped ranks, Q, gradient)."""
    p = grf_problem()
    infos = []
    tt, ranks = _taped_run(ttsn, p, every=5, infos=infos)
    q, g = tt.escape_gradient()
    # first-order size of what the frozen factors leave out, relative to the
    # derivative: 2 sum over roundings of (discarded tail) / ||X||
    model = 2.0 * sum(sum(i["discarded"]) / i["norm"] for i in infos)
    return p, ranks, q, g.cpu().numpy(), model


def _q_at(ttsn, p, sigma, ranks):
    t2, _ = _taped_run(ttsn, p, sigma=sigma, forced=ranks)
    return t2.escape_energy()[0]


def test_full_size_directional_derivative(ttsn, full_size):
    """<g, v> against a central difference of the rounded forward map along a
    smooth direction v at the taped ranks, within a bound made of three
    derived parts:
    - model: the gradient holds each rounding's factors fixed.  For a
      truncation A -> U_r U_r^T A perturbed by dA = D A (sigma_a scales rows)
      the true derivative differs from the frozen-factor one, to first order,
      by P_U dA V_perp V_perp^T + U_r U_r^T dA^T-terms acting on the
      discarded part, each at most ||D|| ||A_disc||; relative to the
      derivative that is 2 (discarded tail) / ||X|| per rounding, summed over
      the taped roundings (from the run's own step diagnostics);
    - noise: the forward's round-off, measured as the largest change of Q
      under perturbations 1e-12 .. 1e-11 v whose true effect is negligible,
      enters the difference as noise / h;
    - truncation: the O(h^2) error, estimated by |fd(h) - fd(2h)|."""
    p, ranks, q, g, model = full_size
    assert np.isfinite(g).all() and q > 0
    sig = p["sigma_a"].reshape(-1)
    v = sig * gaussian_random_field(p["n"], seed=3).reshape(-1)
    dd = float(g @ v)
    q0 = _q_at(ttsn, p, sig, ranks)
    noise = max(abs(_q_at(ttsn, p, sig + eta * v, ranks) - q0 - eta * dd) for eta in (1e-12, 3e-12, 1e-11))

    def fd(h):
        return (_q_at(ttsn, p, sig + h * v, ranks) - _q_at(ttsn, p, sig - h * v, ranks)) / (2 * h)

    h = 1e-4
    f1, f2 = fd(h), fd(2 * h)
    bound = model * abs(dd) + noise / h + abs(f1 - f2)
    print("directional derivative: |fd - dd| / |dd| = %.2e; bound %.2e (model %.2e, noise %.2e, "
          "truncation %.2e)" % (abs(f1 - dd) / abs(dd), bound / abs(dd), model, noise / h / abs(dd),
                                abs(f1 - f2) / abs(dd)))
    assert abs(f1 - dd) <= bound, (f1, dd, bound)


def test_full_size_central_fd_on_16_cells(ttsn, full_size):
    """Central differences on 16 cells: the 8 largest |g| and 8 seeded ones
    among the cells with |g| >= 1% of the largest.  Elsewhere the difference of
    the rounded map is dominated by the rotation of the retained subspaces,
    which the frozen factors leave out (about 1e-3 of max |g| at eps = 1e-6).
    h = 1e-3 sigma_i: a one-cell change moves Q by about 1e-8 of itself per
    1e-4, where the forward's own noise (a few 1e-12 of Q) is already visible."""
    p, ranks, q, g, _ = full_size
    sig = p["sigma_a"].reshape(-1)
    scale = np.abs(g).max()
    rng = np.random.default_rng(1)
    top = np.argsort(-np.abs(g))[:8]
    resolved = np.setdiff1d(np.flatnonzero(np.abs(g) >= 1e-2 * scale), top)
    cells = list(top) + list(rng.choice(resolved, 8, replace=False))
    for i in cells:
        h = 1e-3 * sig[i]
        sp, sm = sig.copy(), sig.copy()
        sp[i] += h
        sm[i] -= h
        fd = (_q_at(ttsn, p, sp, ranks) - _q_at(ttsn, p, sm, ranks)) / (2 * h)
        assert abs(fd - g[i]) <= 5e-4 * scale, (i, fd, g[i], scale)
