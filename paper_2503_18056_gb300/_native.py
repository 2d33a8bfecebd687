"""ctypes declarations for libttsn.so (the C ABI of include/ttsn.h).

Argument marshalling only: every step of the TT-S_N path runs in the library's
CUDA kernels.  Importing this module fails loudly if the library has not been
built (``python -c "import __graft_entry__ as g; g.build()"``).
"""
import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libttsn.so")

TT_MAX_D = 8
TT_OK, TT_WARN_RANK_CAPPED = 0, 1
STATUS_NAMES = {0: "TT_OK", 1: "TT_WARN_RANK_CAPPED", -1: "TT_ERR_ARG", -2: "TT_ERR_OOM",
                -3: "TT_ERR_CUDA", -4: "TT_ERR_NOT_CONVERGED", -5: "TT_ERR_TIMEOUT",
                -6: "TT_ERR_STATE", -7: "TT_ERR_TOO_LARGE", -8: "TT_ERR_NONFINITE"}
TT_BC_PERIODIC, TT_BC_VACUUM, TT_BC_OUTFLOW = 0, 1, 2
TT_FP64, TT_MIXED = 0, 1
TT_LAYOUT_GROUPED, TT_LAYOUT_SPLIT = 0, 1
TT_FLUX_UPWIND, TT_FLUX_RUSANOV, TT_FLUX_HLL, TT_FLUX_RUSANOV_TAU = 0, 1, 2, 3
TT_ROUND_GRAM, TT_ROUND_RANDOMIZED, TT_ROUND_TTSVD = 0, 1, 2
TT_EIG_ONE_SIDED, TT_EIG_TWO_SIDED = 0, 1
TT_STEP_NO_SOURCE, TT_STEP_NO_ROUND = 1, 2


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
# tt_exchange_fn: (ctx, kind, buf_dev, count, stream) -> int
EXCHANGE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t,
                               ctypes.c_void_p)
TT_XCHG_SUM, TT_XCHG_HALO = 0, 1
TT_AUTOTUNE_ENTRIES = 8 * 22
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)


class Allocator(ctypes.Structure):
    _fields_ = [("ctx", ctypes.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN)]


class ProblemDesc(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int), ("n", ctypes.c_int * 3), ("L", ctypes.c_double * 3),
        ("n_theta", ctypes.c_int), ("n_phi", ctypes.c_int),
        ("c", ctypes.c_double), ("a_r", ctypes.c_double), ("cfl", ctypes.c_double),
        ("dt", ctypes.c_double), ("bc", ctypes.c_int * 3),
        ("sigma_a", ctypes.c_void_p), ("sigma_s", ctypes.c_void_p), ("cv", ctypes.c_void_p),
        ("T0", ctypes.c_void_p), ("Tr0", ctypes.c_void_p),
        ("eps", ctypes.c_double), ("max_rank", ctypes.c_int),
        ("rounds_per_step", ctypes.c_int), ("precision", ctypes.c_int),
        ("layout", ctypes.c_int), ("flux", ctypes.c_int), ("flux_param", ctypes.c_double * 2),
    ]


class StepInfo(ctypes.Structure):
    _fields_ = [
        ("d", ctypes.c_int), ("ranks", ctypes.c_int * (TT_MAX_D + 1)),
        ("grown", ctypes.c_int * (TT_MAX_D + 1)), ("discarded", ctypes.c_double * TT_MAX_D),
        ("norm", ctypes.c_double), ("capped", ctypes.c_int), ("sweeps", ctypes.c_int),
    ]

    def as_dict(self):
        d = self.d
        return {"ranks": list(self.ranks[: d + 1]), "grown": list(self.grown[: d + 1]),
                "discarded": list(self.discarded[: max(d - 1, 0)]), "norm": self.norm,
                "capped": bool(self.capped), "sweeps": self.sweeps}


class TTError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libttsn.so is not built at %s; run __graft_entry__.build()" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    vp, i, d, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    ip = ctypes.POINTER(ctypes.c_int)
    dp = ctypes.POINTER(ctypes.c_double)
    sig = {
        "tt_create": [ctypes.POINTER(ProblemDesc), vp, ctypes.POINTER(vp)],
        "tt_create_tt": [i, ip, ip, vp, ctypes.POINTER(vp)],
        "tt_sn_step": [vp, i, ctypes.POINTER(StepInfo)],
        "tt_sn_step_ex": [vp, i, i, ip, ctypes.POINTER(StepInfo)],
        "tt_round": [vp, d, i, ip, ctypes.POINTER(StepInfo)],
        "tt_energy": [vp, vp, vp, dp],
        "tt_to_full": [vp, vp, sz],
        "tt_get_ranks": [vp, ip, i],
        "tt_get_dims": [vp, ip, ip],
        "tt_get_core": [vp, i, vp, sz],
        "tt_set_cores": [vp, ctypes.POINTER(vp), ip],
        "tt_set_T": [vp, vp],
        "tt_sync": [vp],
        "tt_dgemm": [i, i, i, i, i, d, vp, i, vp, i, d, vp, i, vp],
        "tt_gram": [i, i, vp, i, vp, i, vp],
        "tt_gram_noalloc": [i, i, vp, i, vp, i, vp],
        "tt_gram_mixed": [i, i, vp, i, vp, i, vp],
        "tt_gemm_nt_mixed": [i, i, i, vp, i, vp, i, vp, i, vp],
        "tt_set_precision": [vp, i],
        "tt_batch_create": [ctypes.POINTER(ProblemDesc), i, i, ctypes.POINTER(vp)],
        "tt_batch_step": [vp, i, ctypes.POINTER(StepInfo)],
        "tt_batch_size": [vp, ip],
        "tt_batch_handle": [vp, i, ctypes.POINTER(vp)],
        "tt_batch_sync": [vp],
        "tt_syev": [i, vp, i, vp, vp, i, vp, ip],
        "tt_syev_ex": [i, vp, i, vp, vp, i, i, vp, ip],
        "tt_syev_psd": [i, vp, i, vp, vp, i, i, vp, ip],
        "tt_set_max_sweeps": [vp, i],
        "tt_set_graph": [vp, i],
        "tt_autotune": [vp, ip],
        "tt_set_autotune_table": [ip, i],
        "tt_get_autotune_table": [ip, i],
        "tt_batch_set_graph": [vp, i],
        "tt_pchol": [i, vp, i, vp, vp, ip],
        "tt_set_inflow": [vp, i, i, vp, vp, vp],
        "tt_set_sketch": [vp, ctypes.POINTER(vp), ip],
        "tt_set_rounding": [vp, i],
        "tt_set_eigensolver": [vp, i],
        "tt_wait_probe": [vp],
        "tt_profile": [vp, i],
        "tt_profile_read": [vp, i, dp, ctypes.POINTER(ctypes.c_longlong),
                            ctypes.POINTER(ctypes.c_longlong), dp, dp],
        "tt_bench_fp64_mma": [dp, vp],
        "tt_bench_bf16_mma": [dp, vp],
        "tt_tape_begin": [vp, i],
        "tt_tape_objective": [vp, dp, ip],
        "tt_sn_step_adjoint": [vp, vp, dp],
        "tt_tape_clear": [vp],
        "tt_set_sources": [vp, i, vp, vp, vp],
        "tt_create_ex": [ctypes.POINTER(ProblemDesc), vp, ctypes.POINTER(Allocator), ctypes.POINTER(vp)],
        "tt_get_cores": [vp, ctypes.POINTER(vp), ip],
        "tt_create_shard": [ctypes.POINTER(ProblemDesc), vp, i, i, EXCHANGE_FN, vp, ctypes.POINTER(vp)],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.tt_last_error.argtypes = []
    lib.tt_last_error.restype = ctypes.c_char_p
    lib.tt_destroy.argtypes = [vp]
    lib.tt_destroy.restype = None
    lib.tt_batch_destroy.argtypes = [vp]
    lib.tt_batch_destroy.restype = None
    lib.tt_kernel_launches.argtypes = []
    lib.tt_kernel_launches.restype = ctypes.c_ulonglong
    return lib


lib = _load()

#: every symbol the header declares (checked by the CPU test suite)
EXPORTED = ["tt_create", "tt_create_tt", "tt_sn_step", "tt_sn_step_ex", "tt_round", "tt_energy",
            "tt_to_full", "tt_get_ranks", "tt_get_dims", "tt_get_core", "tt_set_cores",
            "tt_set_T", "tt_sync", "tt_last_error", "tt_destroy", "tt_dgemm", "tt_gram",
            "tt_syev", "tt_gram_noalloc", "tt_gram_mixed", "tt_gemm_nt_mixed",
            "tt_set_precision", "tt_profile", "tt_profile_read", "tt_kernel_launches", "tt_bench_fp64_mma",
            "tt_bench_bf16_mma", "tt_batch_create", "tt_batch_step", "tt_batch_size",
            "tt_batch_handle", "tt_batch_sync", "tt_batch_destroy", "tt_tape_begin",
            "tt_tape_objective", "tt_sn_step_adjoint", "tt_tape_clear", "tt_set_sources",
            "tt_create_ex", "tt_get_cores", "tt_pchol", "tt_set_inflow", "tt_set_sketch",
            "tt_set_rounding", "tt_set_eigensolver", "tt_wait_probe", "tt_create_shard", "tt_syev_ex", "tt_syev_psd", "tt_set_max_sweeps", "tt_set_graph",
            "tt_batch_set_graph", "tt_autotune", "tt_set_autotune_table", "tt_get_autotune_table"]

PHASES = ["transport", "gram_right", "eig", "gram_left", "small", "update", "energy"]


def check(status, allow_warn=True):
    if status == TT_OK or (allow_warn and status == TT_WARN_RANK_CAPPED):
        return status
    raise TTError(status, lib.tt_last_error().decode())
