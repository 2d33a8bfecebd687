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
