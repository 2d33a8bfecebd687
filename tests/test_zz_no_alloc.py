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
    A_host = rng.standard_normal((m, n))
    A = torch.as_tensor(A_host, device="cuda")
    ref = ttsn.gram(A).cpu().numpy()          # existing entry point (tt_gram)
    G = torch.full((n, n), float("nan"), dtype=torch.float64, device="cuda")
    out = ttsn.gram_noalloc(A, G).cpu().numpy()   # through the C ABI, caller-owned output
    assert np.array_equal(out, out.T)
    # the tolerance of the tt_gram tests: reduction order differs, values agree
    assert np.abs(out - ref).max() <= 1e-13 * np.abs(ref).max() * np.sqrt(m)
    # and against NumPy's A^T A, independent of every CUDA path, within the
    # classical bound of a sum of m products in any order, |error_ij| <=
    # m eps (|A|^T |A|)_ij, taken once for each of the two sums
    exact = A_host.T @ A_host
    absA = np.abs(A_host)
    bound = 2.0 * m * np.finfo(float).eps * (absA.T @ absA)
    assert np.all(np.abs(out - exact) <= bound)


def test_noalloc_gram_matches_tt_gram_on_two_calls_in_a_row(ttsn):
    # a large call then a smaller one: the second must not see the first's contents
    _check(ttsn, 300000, 897, seed=1)
    _check(ttsn, 4099, 130, seed=2)


def test_noalloc_gram_rejects_sizes_over_its_limit(ttsn):
    import torch

    from paper_2503_18056_gb300 import _native

    # real device buffers of the declared sizes: were the host-side limit ever
    # lost, the call would still touch only memory it owns
    m, n = 10, 1025
    A = torch.ones((m, n), dtype=torch.float64, device="cuda")
    G = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    st = _native.lib.tt_gram_noalloc(m, n, ctypes.c_void_p(A.data_ptr()), n, ctypes.c_void_p(G.data_ptr()), n,
                                     None)
    torch.cuda.synchronize()
    assert st == -7  # TT_ERR_TOO_LARGE, rejected on the host before any device work
    assert b"1024" in _native.lib.tt_last_error()
    assert float(G.abs().max()) == 0.0


def test_noalloc_binding_refuses_an_output_that_cannot_hold_the_gram(ttsn):
    import torch

    A = torch.ones((64, 16), dtype=torch.float64, device="cuda")
    for G in (torch.zeros((16, 16), dtype=torch.float32, device="cuda"),
              torch.zeros((15, 16), dtype=torch.float64, device="cuda"),
              torch.zeros((16, 32), dtype=torch.float64, device="cuda")[:, ::2],
              torch.zeros((16, 16), dtype=torch.float64)):
        with pytest.raises(ValueError):
            ttsn.gram_noalloc(A, G)
    # a row-padded output is written at its own row stride, padding untouched
    P = torch.full((16, 24), -1.0, dtype=torch.float64, device="cuda")
    out = ttsn.gram_noalloc(A, P[:, :16])
    torch.cuda.synchronize()
    assert float((out - 64.0).abs().max()) == 0.0
    assert float((P[:, 16:] + 1.0).abs().max()) == 0.0
