"""The allocation-free Gram entry point (tt_gram_noalloc).

Some callers cannot let a library allocate device memory: an application whose
own allocator owns the device's memory, or a latency-critical loop that cannot
pay for the synchronisation of cudaMalloc/cudaFree.  tt_gram_noalloc computes
the same left Gram G = A^T A as tt_gram using a fixed scratch array built into
the library.  This file is collected last so a stop-at-first-failure run has
already run every other test; it passes alone in a fresh process too.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ttsn():
    import torch

    assert torch.cuda.is_available()
    import paper_2503_18056_gb300 as m

    return m


def _check(ttsn, m, n, seed):
    import torch

    rng = np.random.default_rng(seed)
    A = torch.as_tensor(rng.standard_normal((m, n)), device="cuda")
    ref = ttsn.gram(A).cpu().numpy()          # existing entry point (tt_gram)
    G = torch.full((n, n), float("nan"), dtype=torch.float64, device="cuda")
    out = ttsn.gram_noalloc(A, G).cpu().numpy()   # through the C ABI, caller-owned output
    assert np.array_equal(out, out.T)
    # the tolerance of the tt_gram tests: reduction order differs, values agree
    assert np.abs(out - ref).max() <= 1e-13 * np.abs(ref).max() * np.sqrt(m)


def test_noalloc_gram_matches_tt_gram_on_two_calls_in_a_row(ttsn):
    # a large call then a smaller one: the second must not see the first's contents
    _check(ttsn, 300000, 897, seed=1)
    _check(ttsn, 4099, 130, seed=2)


def test_noalloc_gram_rejects_sizes_over_its_limit(ttsn):
    from paper_2503_18056_gb300 import _native

    st = _native.lib.tt_gram_noalloc(10, 1025, ctypes.c_void_p(1), 1025, ctypes.c_void_p(1), 1025, None)
    assert st == -7  # TT_ERR_TOO_LARGE, rejected on the host before any device work
    assert b"1024" in _native.lib.tt_last_error()
