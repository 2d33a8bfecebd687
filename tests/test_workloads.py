"""The seeded input generators against the setups they state (Sec. 5 test
problems and the synthetic recipes): sizes, time steps, normalisations and
field statistics."""
import numpy as np
import pytest

import workloads


def test_blob_3d_recipe():
    p = workloads.problem("blob_3d", n=(32, 32, 32))
    assert p["n_theta"] == 32 and p["n_phi"] == 64 and p["eps"] == 1e-6 and p["max_rank"] == 128
    assert set(np.unique(p["sigma_a"])) <= {1e2, 1e-2} and (p["sigma_a"] == 1e2).any()
    assert set(np.unique(p["T0"])) == {1.0, 1e-3}
    assert p["bc"] == [workloads.VACUUM] * 3 and p["dt"] == pytest.approx(0.5 / 32)
    full = workloads.problem("blob_3d")
    assert full["n"] == (128, 128, 128) and full["steps"] == 100


def test_small_2d_recipe():
    p = workloads.problem("small_2d")
    assert p["n"] == (32, 32) and p["n_theta"] == 8 and p["n_phi"] == 16 and p["eps"] == 1e-8
    assert p["dt"] == pytest.approx(0.5 / 32) and p["bc"] == [workloads.PERIODIC] * 2
    assert 0.95 < p["T0"].max() <= 1.01 and p["T0"].min() >= 0.01  # peak 1 on 0.01, centre between cells


def test_line_source_recipe_carries_U0_and_reaches_t1_in_568_steps():
    """Sec. 5.4: [-1.1, 1.1]^2 at 500^2, pulse width 0.03 (6.8 cells), CFL 0.4."""
    p = workloads.line_source()
    dV = (2.2 / 500) ** 2
    assert (p["Tr0"] ** 4).sum() * dV == pytest.approx(1.0, rel=1e-9)
    assert int(round(p["t_lim"] / p["dt"])) == 568 and p["dt"] == pytest.approx(0.4 * 2.2 / 500)
    assert not p["sigma_a"].any() and p["bc"] == [workloads.VACUUM] * 2
    i, j = np.unravel_index(np.argmax(p["Tr0"]), p["n"])
    assert abs(p["radius"][i, j]) < 2.2 / 500


def test_hohlraum_recipe():
    """Sec. 5.1: [0, 2]^2, unit isotropic inflow on x = 0 and y = 0, empty."""
    p = workloads.hohlraum()
    assert p["n"] == (256, 256) and p["L"] == (2.0, 2.0) and int(round(p["t_lim"] / p["dt"])) == 192
    assert sorted(p["inflow"]) == [(0, 0), (1, 0)] and not p["Tr0"].any() and not p["sigma_a"].any()
    for g, th, ph in p["inflow"].values():
        assert (g == 1).all() and (th == 1).all() and (ph == 1).all()


def test_gaussian_diffusion_recipe_carries_A():
    """Sec. 5: E(0) = A / (4 pi D t0) exp(-r^2 / (4 D t0)), D = c / (3 sigma_s)."""
    p = workloads.gaussian_diffusion()
    dV = (5.0 / 128) ** 2
    assert (p["Tr0"] ** 4).sum() * dV == pytest.approx(p["amp"], rel=1e-6)
    assert p["D"] == pytest.approx(1.0 / 3e3) and not p["sigma_a"].any()


def test_grf_field_statistics_and_batch_ranges():
    g = workloads.gaussian_random_field((128, 128), seed=0, corr=0.1)
    assert abs(g.mean()) < 1e-12 and g.std() == pytest.approx(1.0)
    # smooth: neighbouring cells correlate strongly at corr length 0.1 = 12.8 cells
    assert np.corrcoef(g[:-1].ravel(), g[1:].ravel())[0, 1] > 0.9
    probs = workloads.batch_problems()
    assert len(probs) == 64
    assert {p["n"][0] for p in probs} <= {64, 128, 256} and {p["eps"] for p in probs} <= {1e-4, 1e-6}
    assert all(8 <= p["max_rank"] <= 96 and 1e-2 <= p["sigma_a"].flat[0] <= 1e2 for p in probs)
    again = workloads.batch_problems()
    assert all(np.array_equal(a["T0"], b["T0"]) for a, b in zip(probs, again))  # seeded
