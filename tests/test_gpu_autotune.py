"""The products' autotuner (tt_autotune): it measures a split of K for every
(tile-count, depth) bucket, installs the table for host-driven and captured
steps alike, stores and reloads it, and a product computed under any table
stays within FP64 rounding of the exact product."""
import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ttsn():
    assert torch.cuda.is_available()
    import paper_2503_18056_gb300 as m

    yield m
    m.load_autotune([0] * 176)  # later tests run with the built-in rule


def test_autotune_measures_stores_and_reloads(ttsn, tmp_path):
    path = tmp_path / "splits.json"
    table = ttsn.autotune(path=str(path))
    assert len(table) == 176 and all(0 <= x <= 64 for x in table)
    for tb in range(8):  # every measured bucket holds a power-of-two split
        for kb in range(6, 15):
            x = table[tb * 22 + kb]
            assert x >= 1 and (x & (x - 1)) == 0 and x <= max(1, (1 << kb) // 32)
    assert ttsn.autotune_table() == table
    ttsn.load_autotune([0] * 176)
    assert ttsn.autotune_table() == [0] * 176
    ttsn.load_autotune(str(path))
    assert ttsn.autotune_table() == table
    with pytest.raises(ttsn.TTError):
        ttsn.load_autotune([65] * 176)
    with pytest.raises(ttsn.TTError):
        ttsn.load_autotune([1] * 10)


@pytest.mark.parametrize("split", [1, 4, 64])
def test_products_under_any_table_stay_exact_to_rounding(ttsn, split):
    ttsn.load_autotune([split] * 176)
    rng = np.random.default_rng(split)
    for M, N, K in ((70, 90, 3000), (300, 64, 700), (5, 7, 20000)):
        A, B = rng.standard_normal((M, K)), rng.standard_normal((K, N))
        C = ttsn.dgemm(A, B).cpu().numpy()
        ref = A @ B
        bound = 2 * K * np.finfo(float).eps * (np.abs(A) @ np.abs(B))
        assert np.all(np.abs(C - ref) <= bound)
    ttsn.load_autotune([0] * 176)


def test_captured_steps_follow_the_installed_table(ttsn):
    ttsn.load_autotune([2] * 176)
    p = workloads.problem("small_2d", n=(16, 12), n_theta=4, n_phi=8, eps=1e-6)
    p["max_rank"] = 24
    a = ttsn.TTSN.from_problem(p)
    b = ttsn.TTSN.from_problem(p)
    b.set_graph(True)
    a.step(5)
    b.step(5)
    assert torch.equal(a.full(), b.full())
    ttsn.load_autotune([0] * 176)
