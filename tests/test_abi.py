"""CPU checks of the C-ABI library: it loads and exports every declared symbol."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ttsn.h")).read()
    return sorted(set(re.findall(r"^\s*(?:tt_status|const char\*|void|unsigned long long)\s+(tt_\w+)\s*\(", src, re.M)))


def test_header_declarations_found():
    names = _declared()
    assert "tt_sn_step" in names and "tt_round" in names and len(names) >= 15


def test_library_builds_loads_and_exports_all_symbols():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2503_18056_gb300 import _native

    missing = [n for n in _declared() if not hasattr(_native.lib, n)]
    assert missing == []
    assert sorted(_native.EXPORTED) == _declared()


def test_error_message_without_gpu_is_reported_not_raised():
    # a call with an invalid argument returns TT_ERR_ARG without touching the GPU
    import ctypes

    from paper_2503_18056_gb300 import _native

    h = ctypes.c_void_p()
    st = _native.lib.tt_create_tt(0, None, None, None, ctypes.byref(h))
    assert st == -1
    assert b"null" in _native.lib.tt_last_error() or b"range" in _native.lib.tt_last_error()


_KEEP = []


def _valid_desc(_native):
    import ctypes

    d = _native.ProblemDesc()
    d.ndim = 2
    d.n[0], d.n[1], d.n[2] = 8, 6, 1
    d.L[0] = d.L[1] = d.L[2] = 1.0
    d.n_theta, d.n_phi = 4, 8
    d.c, d.a_r, d.cfl, d.dt = 1.0, 1.0, 0.5, 0.0
    # a real buffer of N_c doubles (host memory; no device here): every case
    # below is refused before any field is read, and were a check ever lost
    # the call would read only memory that exists
    field = (ctypes.c_double * (8 * 6))()
    _KEEP.append(field)
    d.sigma_a = d.cv = d.T0 = ctypes.cast(field, ctypes.c_void_p)
    d.eps, d.max_rank, d.rounds_per_step, d.precision = 1e-6, 0, 1, 0
    d.layout, d.flux = 0, 0
    return d


BAD_DESCS = [
    ("ndim", lambda d: setattr(d, "ndim", 0)), ("ndim", lambda d: setattr(d, "ndim", 4)),
    ("n[a]", lambda d: d.n.__setitem__(1, 0)), ("L[a]", lambda d: d.L.__setitem__(0, 0.0)),
    ("bc", lambda d: d.bc.__setitem__(1, 7)), ("n_theta", lambda d: setattr(d, "n_theta", 0)),
    ("n_theta", lambda d: setattr(d, "n_phi", 0)), ("c > 0", lambda d: setattr(d, "c", 0.0)),
    ("a_r", lambda d: setattr(d, "a_r", -1.0)), ("cfl", lambda d: setattr(d, "cfl", 0.0)),
    ("sigma_a", lambda d: setattr(d, "sigma_a", None)), ("eps", lambda d: setattr(d, "eps", -1.0)),
    ("rounds_per_step", lambda d: setattr(d, "rounds_per_step", 3)),
    ("precision", lambda d: setattr(d, "precision", 2)), ("layout", lambda d: setattr(d, "layout", 5)),
    ("flux", lambda d: setattr(d, "flux", 9)),
    ("Rusanov", lambda d: (setattr(d, "flux", 1), d.flux_param.__setitem__(0, -1.0))),
    ("HLL", lambda d: (setattr(d, "flux", 2), d.flux_param.__setitem__(0, 0.0), d.flux_param.__setitem__(1, 1.0))),
    ("HLL", lambda d: (setattr(d, "flux", 2), d.flux_param.__setitem__(0, 1.0), d.flux_param.__setitem__(1, 2.0))),
]


def test_invalid_problem_descriptions_are_refused_on_the_host():
    """tt_create validates the whole description before touching the device:
    every malformed field is TT_ERR_ARG with a message naming it (no GPU
    needed), and an oversized grid is TT_ERR_TOO_LARGE."""
    import ctypes

    from paper_2503_18056_gb300 import _native

    lib = _native.lib
    for word, spoil in BAD_DESCS:
        d = _valid_desc(_native)
        spoil(d)
        h = ctypes.c_void_p()
        st = lib.tt_create(ctypes.byref(d), None, ctypes.byref(h))
        assert st == -1, (word, st)
        assert h.value is None
        assert word.encode() in lib.tt_last_error(), (word, lib.tt_last_error())
    d = _valid_desc(_native)
    d.n[0], d.n[1] = 65536, 65536
    assert lib.tt_create(ctypes.byref(d), None, ctypes.byref(ctypes.c_void_p())) == -7
    assert lib.tt_create(None, None, ctypes.byref(ctypes.c_void_p())) == -1
    bad_alloc = _native.Allocator()
    d = _valid_desc(_native)
    assert lib.tt_create_ex(ctypes.byref(d), None, ctypes.byref(bad_alloc), ctypes.byref(ctypes.c_void_p())) == -1
    assert b"allocator" in lib.tt_last_error()


def test_null_handle_and_bad_sizes_are_refused_on_the_host():
    """Every handle call refuses a null handle with TT_ERR_ARG, and the
    kernel-level calls refuse negative sizes, null operands and short leading
    dimensions before any device work (no GPU needed)."""
    import ctypes

    from paper_2503_18056_gb300 import _native

    lib = _native.lib
    null = ctypes.c_void_p()
    buf = (ctypes.c_int * 8)()
    calls = [
        lambda: lib.tt_sn_step(null, 1, None), lambda: lib.tt_sn_step_ex(null, 1, 0, None, None),
        lambda: lib.tt_round(null, 1e-6, 0, None, None), lambda: lib.tt_energy(null, None, None, None),
        lambda: lib.tt_to_full(null, None, 0), lambda: lib.tt_get_ranks(null, buf, 8),
        lambda: lib.tt_get_dims(null, buf, buf), lambda: lib.tt_set_T(null, None),
        lambda: lib.tt_sync(null), lambda: lib.tt_set_precision(null, 0),
        lambda: lib.tt_set_rounding(null, 0), lambda: lib.tt_profile(null, 1),
        lambda: lib.tt_tape_begin(null, 1), lambda: lib.tt_tape_clear(null),
    ]
    for i, call in enumerate(calls):
        assert call() == -1, i
        assert b"null" in lib.tt_last_error(), (i, lib.tt_last_error())
    # a real 64-double buffer, larger than any size below: each call is refused
    # before touching it, and a lost check would still stay inside it
    xbuf = (ctypes.c_double * 64)()
    x = ctypes.cast(xbuf, ctypes.c_void_p)
    assert lib.tt_gram(-1, 4, x, 4, x, 4, None) == -1
    assert lib.tt_gram(8, 4, None, 4, x, 4, None) == -1
    assert lib.tt_gram(8, 4, x, 3, x, 4, None) == -1 and b"leading" in lib.tt_last_error()
    assert lib.tt_gram(8, 0, None, 0, None, 0, None) == 0  # nothing to do
    assert lib.tt_dgemm(0, 0, -1, 2, 2, 1.0, x, 2, x, 2, 0.0, x, 2, None) == -1
    assert lib.tt_dgemm(0, 0, 2, 2, 2, 1.0, None, 2, x, 2, 0.0, x, 2, None) == -1
    assert lib.tt_syev(-3, x, 3, x, x, 3, None, None) == -1
    assert lib.tt_pchol(-1, x, 4, x, None, None) == -1
    assert lib.tt_pchol(4, x, 3, x, None, None) == -1 and b"leading" in lib.tt_last_error()
    assert lib.tt_pchol(0, None, 0, None, None, None) == 0


def test_autotune_table_arguments_are_checked_on_the_host():
    """A stored table of the wrong length or with a split outside 0 .. 64 is
    refused before the device is touched (no GPU needed)."""
    import ctypes

    from paper_2503_18056_gb300 import _native

    lib = _native.lib
    bad = (ctypes.c_int * 176)(*([65] * 176))
    assert lib.tt_set_autotune_table(bad, 176) == -1
    short = (ctypes.c_int * 10)(*([1] * 10))
    assert lib.tt_set_autotune_table(short, 10) == -1
    assert lib.tt_set_autotune_table(None, 176) == -1
    out = (ctypes.c_int * 4)()
    assert lib.tt_get_autotune_table(out, 4) == -1
