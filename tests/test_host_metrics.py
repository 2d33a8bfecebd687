"""Host-side metrics of the binding (no GPU): the compression factor of
Sec. 5.1 against the paper's printed hohlraum figures, and the run-log record."""
import json
import math
import os

import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2503_18056_gb300 as m

    return m


def test_compression_factor_reproduces_the_hohlraum_figures(pkg):
    """Sec. 5.1 prints C ~ 5e5 at ranks (1, 1) and C ~ 3e3 at the final ranks
    (141, 61) for 512^2 cells and 512 x 1024 ordinates (one significant
    figure each)."""
    with open(os.path.join(GOLDEN, "hohlraum_compression.json")) as f:
        g = json.load(f)
    dims = [g["Nx"] * g["Ny"], g["Ntheta"], g["Nphi"]]
    r1, r2 = g["ranks_final"]
    c_final = pkg.compression_factor(dims, [1, r1, r2, 1])
    c_init = pkg.compression_factor(dims, [1, 1, 1, 1])
    for c, printed in ((c_final, g["C_final_approx"]), (c_init, g["C_initial_approx"])):
        scale = 10 ** math.floor(math.log10(c))
        assert round(c / scale) * scale == printed, c  # 3318 -> 3e3, 5.2e5 -> 5e5


def test_compression_factor_of_a_rank_one_split_tt(pkg):
    """Five cores of a rank-one TT store the sum of the mode sizes."""
    dims = [128, 128, 128, 32, 64]
    assert pkg.compression_factor(dims, [1] * 6) == 128 ** 3 * 32 * 64 / (3 * 128 + 32 + 64)


def test_step_record_fields(pkg):
    info = {"ranks": [1, 5, 3, 1], "grown": [1, 26, 16, 1], "discarded": [1e-9, 2e-9], "norm": 3.0,
            "capped": False, "sweeps": 7}
    rec = pkg.step_record(4, 0.125, info, (2.0, 0.5), [100, 8, 16], ms=1.5)
    assert rec["step"] == 4 and rec["t"] == 0.125 and rec["ranks"] == [1, 5, 3, 1]
    assert rec["compression"] == 100 * 8 * 16 / (5 * 100 + 5 * 3 * 8 + 3 * 16)
    assert rec["E_total"] == 2.5 and rec["ms"] == 1.5
    json.dumps(rec)  # serialisable as one JSON line
    assert "ms" not in pkg.step_record(1, 0.0, info, (1.0, 1.0), [100, 8, 16])
