"""GB300 (sm_103a) tensor-train discrete-ordinates thermal radiation transport.

A thin PyTorch-facing wrapper over libttsn (include/ttsn.h).  PyTorch supplies
device memory and the CUDA stream; the TT-S_N step itself (transport core
apply, quadrature, quartic temperature solve, source assembly, Gram sweeps,
Jacobi eigensolves, truncation and core updates) runs in the library's kernels.
There is no CPU fallback: importing this package without the built library
raises ImportError.

``TTSN`` is one problem: grouped (three cores) or split (one core per spatial
axis) layout, FP64 or the BF16-digit precision form, upwind / Rusanov / HLL
fluxes, periodic / vacuum / outflow faces, inflow faces (``set_inflow``),
fixed sources (``set_sources``), Gram-SVD or randomized rounding
(``set_sketch``, ``set_rounding``), the adjoint tape (``tape_begin``,
``escape_gradient``) and ``EscapeEnergy`` as a torch.autograd.Function.
``TTSN.run`` steps with a per-step record (ranks, discarded tails,
compression factor, energies, GPU ms; JSON lines with ``log=``);
``state_dict`` / ``load_state_dict`` checkpoint and resume a run; any object
with ``alloc``/``free`` (``TorchAllocator`` for torch's caching allocator) can
supply the device memory.  ``TTSNBatch`` steps many independent problems
together; ``TensorTrain`` is a bare TT for the rounding entry points;
``dgemm``, ``gram``, ``gram_mixed``, ``gemm_nt_mixed``, ``syev`` and ``pchol``
expose the kernel-level calls.  Failures come back as ``TTError`` with the
library's status (argument, out of memory, bounded wait ran out, eigensolver
sweep limit, Inf/NaN met by a rounding).
"""
import ctypes
import os

import numpy as np
import torch

from . import _native
from ._native import (TT_BC_OUTFLOW, TT_BC_PERIODIC, TT_BC_VACUUM, TT_FP64, TT_LAYOUT_GROUPED, TT_LAYOUT_SPLIT,
                      TT_MIXED, TT_STEP_NO_ROUND, TT_STEP_NO_SOURCE, TTError, StepInfo, check, lib)

__all__ = ["TTSN", "TTSNBatch", "shard", "TorchAllocator", "compression_factor", "step_record", "EscapeEnergy", "escape_energy", "TensorTrain", "dgemm", "gram", "gram_mixed", "gemm_nt_mixed", "syev", "syev_psd", "pchol",
           "TTError", "TT_BC_PERIODIC", "TT_BC_VACUUM", "TT_BC_OUTFLOW", "TT_FP64", "TT_MIXED", "TT_STEP_NO_SOURCE",
           "TT_STEP_NO_ROUND", "TT_LAYOUT_GROUPED", "TT_LAYOUT_SPLIT"]


def _stream_ptr(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev(x, n=None):
    t = torch.as_tensor(x, dtype=torch.float64, device="cuda").contiguous()
    if n is not None and t.numel() != n:
        raise ValueError("expected %d values, got %d" % (n, t.numel()))
    return t


def _dev_or_host(x, n=None):
    """A contiguous float64 CPU tensor as it is (the library copies host
    memory itself, without a device staging tensor), anything else on the
    device."""
    if isinstance(x, torch.Tensor) and x.device.type == "cpu" and x.dtype == torch.float64 and x.is_contiguous():
        if n is not None and x.numel() != n:
            raise ValueError("expected %d values, got %d" % (n, x.numel()))
        return x
    return _dev(x, n)


def _int_array(vals):
    if vals is None:
        return None
    arr = (ctypes.c_int * len(vals))(*[int(v) for v in vals])
    return arr


class _Handle:
    def __init__(self):
        self._h = ctypes.c_void_p()
        self.stream = None

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib.tt_destroy(h)
            self._h = None

    # -- common TT access
    def ranks(self):
        d, n = self.dims()
        buf = (ctypes.c_int * (d + 1))()
        check(lib.tt_get_ranks(self._h, buf, d + 1))
        return list(buf)

    def core_views(self):
        """Borrowed device views (pointer, shape) of the cores (tt_get_cores);
        valid until the TT next changes."""
        d, _ = self.dims()
        ptrs = (ctypes.c_void_p * d)()
        shapes = (ctypes.c_int * (3 * d))()
        check(lib.tt_get_cores(self._h, ptrs, shapes))
        return [(ptrs[k], tuple(shapes[3 * k:3 * k + 3])) for k in range(d)]

    def dims(self):
        d = ctypes.c_int()
        n = (ctypes.c_int * _native.TT_MAX_D)()
        check(lib.tt_get_dims(self._h, ctypes.byref(d), n))
        return d.value, list(n[: d.value])

    def cores(self, into=None):
        """Copies of the cores, (r_{k-1}, n_k, r_k) each: new device tensors,
        or, with ``into`` (one flat float64 tensor per core, device or host --
        pinned host memory copies at the host link's speed -- with room for
        the core), views of those buffers written in place."""
        d, n = self.dims()
        r = self.ranks()
        if into is not None and len(into) < d:
            raise ValueError("into needs one buffer per core (%d), got %d" % (d, len(into)))
        out = []
        for k in range(d):
            shape = (r[k], n[k], r[k + 1])
            if into is None:
                t = torch.empty(shape, dtype=torch.float64, device="cuda")
            else:
                buf = into[k]
                if buf.dtype != torch.float64 or not buf.is_contiguous() or buf.numel() < r[k] * n[k] * r[k + 1]:
                    raise ValueError("into[%d] must be a contiguous float64 tensor of at least %d values"
                                     % (k, r[k] * n[k] * r[k + 1]))
                t = buf.view(-1)[: r[k] * n[k] * r[k + 1]].view(shape)
            check(lib.tt_get_core(self._h, k, ctypes.c_void_p(t.data_ptr()), t.numel()))
            out.append(t)
        return out

    def set_cores(self, cores):
        """Replace the TT by ``cores`` (copied in; device tensors, or float64
        CPU tensors -- pinned ones copy at the host link's speed -- which the
        library reads directly).  The count and every shape are checked against
        the handle's mode sizes before the library copies anything: core k must
        be (r_{k-1}, n_k, r_k) with r_0 = r_d = 1 and each r_{k-1} equal to the
        previous core's last dimension."""
        d, n = self.dims()
        ts = [_dev_or_host(c) for c in cores]
        if len(ts) != d:
            raise ValueError("expected %d cores, got %d" % (d, len(ts)))
        prev = 1
        for k, t in enumerate(ts):
            if t.dim() != 3:
                raise ValueError("core %d must be 3-dimensional, got shape %s" % (k, tuple(t.shape)))
            r0, nk, r1 = (int(x) for x in t.shape)
            if r0 != prev or nk != n[k] or r1 < 1 or (k == d - 1 and r1 != 1):
                raise ValueError("core %d has shape %s; expected (%d, %d, r) with r %s"
                                 % (k, tuple(t.shape), prev, n[k], "= 1" if k == d - 1 else ">= 1"))
            prev = r1
        ranks = [1] + [int(t.shape[2]) for t in ts[:-1]] + [1]
        ptrs = (ctypes.c_void_p * len(ts))(*[t.data_ptr() for t in ts])
        check(lib.tt_set_cores(self._h, ptrs, _int_array(ranks)))

    def set_sketch(self, cores):
        """Gaussian sketch TT of the randomized rounding (tt_set_sketch); None removes it."""
        if cores is None:
            check(lib.tt_set_sketch(self._h, None, None))
            return
        ts = [_dev(c) for c in cores]
        ranks = [1] + [int(t.shape[2]) for t in ts[:-1]] + [1]
        ptrs = (ctypes.c_void_p * len(ts))(*[t.data_ptr() for t in ts])
        check(lib.tt_set_sketch(self._h, ptrs, _int_array(ranks)))

    def set_rounding(self, method):
        """'gram' (default), 'randomized' (App. A.3) or 'ttsvd' (the QR-based
        rounding of App. A.1) for the following roundings (tt_set_rounding)."""
        m = {"gram": _native.TT_ROUND_GRAM, "randomized": _native.TT_ROUND_RANDOMIZED,
             "ttsvd": _native.TT_ROUND_TTSVD}[method]
        check(lib.tt_set_rounding(self._h, m))

    def full(self):
        d, n = self.dims()
        out = torch.empty(n, dtype=torch.float64, device="cuda")
        check(lib.tt_to_full(self._h, ctypes.c_void_p(out.data_ptr()), out.numel()))
        return out

    def round(self, eps=0.0, max_rank=0, forced=None):
        info = StepInfo()
        check(lib.tt_round(self._h, float(eps), int(max_rank or 0), _int_array(forced),
                           ctypes.byref(info)))
        return info.as_dict()

    def sync(self):
        check(lib.tt_sync(self._h))

    def set_precision(self, precision):
        check(lib.tt_set_precision(self._h, int(precision)))

    def set_graph(self, enable=True):
        """Captured steps (tt_set_graph): one recorded step replayed as a CUDA
        graph, sizes decided on the device, no host synchronisation inside."""
        check(lib.tt_set_graph(self._h, int(bool(enable))))

    def set_eigensolver(self, method):
        """'one_sided' (default: pivoted Cholesky + one-sided Jacobi) or
        'two_sided' (Jacobi on K) for the rounding's eigensolves (tt_set_eigensolver)."""
        m = {"one_sided": _native.TT_EIG_ONE_SIDED, "two_sided": _native.TT_EIG_TWO_SIDED}[method]
        check(lib.tt_set_eigensolver(self._h, m))

    def set_max_sweeps(self, max_sweeps):
        """Sweep limit of the Jacobi eigensolves of this handle's roundings (1 .. 40)."""
        check(lib.tt_set_max_sweeps(self._h, int(max_sweeps)))

    def profile(self, enable=True):
        check(lib.tt_profile(self._h, int(bool(enable))))

    def profile_read(self):
        out = {}
        for k, name in enumerate(_native.PHASES):
            ms, fl, by = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
            la, ca = ctypes.c_longlong(), ctypes.c_longlong()
            check(lib.tt_profile_read(self._h, k, ctypes.byref(ms), ctypes.byref(la),
                                      ctypes.byref(ca), ctypes.byref(fl), ctypes.byref(by)))
            out[name] = {"ms": ms.value, "launches": la.value, "calls": ca.value,
                         "flops": fl.value, "bytes": by.value}
        return out


class TensorTrain(_Handle):
    """A bare TT (no physics) for the rounding entry points."""

    def __init__(self, cores, stream=None):
        super().__init__()
        ts = [_dev(c) for c in cores]
        d = len(ts)
        n = [int(t.shape[1]) for t in ts]
        ranks = [1] + [int(t.shape[2]) for t in ts[:-1]] + [1]
        self.stream = stream
        check(lib.tt_create_tt(d, _int_array(n), _int_array(ranks), _stream_ptr(stream),
                               ctypes.byref(self._h)))
        self.set_cores(ts)


def compression_factor(dims, ranks):
    """The compression factor C of Sec. 5.1: entries of the full tensor over
    entries of its TT cores, prod_k n_k / sum_k r_{k-1} n_k r_k (for the
    three-core layout N_c N_theta N_phi / (r_1 N_c + r_1 r_2 N_theta + r_2 N_phi))."""
    full = 1.0
    for m in dims:
        full *= float(m)
    stored = sum(float(ranks[k]) * float(dims[k]) * float(ranks[k + 1]) for k in range(len(dims)))
    return full / stored


def step_record(step, t, info, totals, dims, ms=None):
    """One line of a run log: step index and time, ranks entering and leaving
    the rounding, discarded tail per bond, ||X||, rank-cap flag, Jacobi sweeps,
    compression factor, radiation and material energy (sum E dV, sum C_v T dV),
    and the step's GPU time in ms when measured."""
    rec = {"step": int(step), "t": float(t), "ranks": list(info["ranks"]), "grown": list(info["grown"]),
           "discarded": [float(x) for x in info["discarded"]], "norm": float(info["norm"]),
           "capped": bool(info["capped"]), "sweeps": int(info["sweeps"]),
           "compression": compression_factor(dims, info["ranks"]),
           "E_rad": float(totals[0]), "E_mat": float(totals[1]),
           "E_total": float(totals[0]) + float(totals[1])}
    if ms is not None:
        rec["ms"] = float(ms)
    return rec


class TorchAllocator:
    """Device memory from torch's CUDA caching allocator: the handle's buffers
    then count in torch.cuda.memory_allocated() and share torch's cached
    blocks.  Any object with the same two methods can serve as a handle's
    allocator; ``alloc`` returns 0 when it cannot serve a request, which the
    library reports as TT_ERR_OOM."""

    def alloc(self, nbytes, stream):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
        except Exception:
            return 0

    def free(self, ptr, nbytes, stream):
        torch.cuda.caching_allocator_delete(int(ptr))


def _c_allocator(obj):
    """Wrap an object with alloc(nbytes, stream) -> pointer (0: refused) and
    free(ptr, nbytes, stream) as a tt_allocator.  The callbacks run on the
    calling thread (ctypes takes the GIL for them)."""
    def alloc(ctx, nbytes, stream):
        try:
            return int(obj.alloc(int(nbytes), stream)) or None
        except Exception:
            return None

    def free(ctx, ptr, nbytes, stream):
        obj.free(int(ptr), int(nbytes), stream)

    a = _native.Allocator()
    a.ctx = None
    a.alloc = _native.ALLOC_FN(alloc)
    a.free = _native.FREE_FN(free)
    return a


class TTSN(_Handle):
    """A TT-S_N problem on the current CUDA stream, in the paper's three-core
    layout (``layout=TT_LAYOUT_GROUPED``) or with one core per spatial axis
    (``TT_LAYOUT_SPLIT``; uniform sigma_a and sigma_s), with the upwind,
    Rusanov (S+ = rusanov_s c), HLL (hll_beta, hll_tau_threshold) or Rusanov
    with the optical-depth speed S+ = c |n| min(1, 1/tau_c) ("rusanov_tau",
    tau_c from Eq. tauc with beta = hll_beta) flux.

    Fields are array-likes of N_c values in C order of the grid (axis 0
    slowest); they are copied to the device and then into the library.
    """

    def __init__(self, n, L, n_theta, n_phi, sigma_a, cv, T0, Tr0=None, sigma_s=None, c=1.0,
                 a_r=1.0, dt=0.0, cfl=0.5, bc=TT_BC_PERIODIC, eps=1e-6, max_rank=0,
                 rounds_per_step=1, precision=TT_FP64, stream=None, allocator=None,
                 layout=TT_LAYOUT_GROUPED, flux="upwind", rusanov_s=1.0, hll_beta=1.0,
                 hll_tau_threshold=1.0, shard=None):
        super().__init__()
        ndim = len(n)
        nc = 1
        for m in n:
            nc *= int(m)
        if isinstance(bc, int):
            bc = [bc] * ndim
        self.nc = nc
        self.n = tuple(int(m) for m in n)
        self.shard = None
        self.n_theta, self.n_phi = int(n_theta), int(n_phi)
        self.stream = stream
        # the library's rule for dt <= 0: CFL times the smallest cell width over c
        self.dt = float(dt) if dt > 0 else float(cfl) * min(float(L[a]) / self.n[a] for a in range(ndim)) / float(c)
        self.steps_taken = 0
        f = {"sigma_a": _dev(sigma_a, nc), "cv": _dev(cv, nc), "T0": _dev(T0, nc)}
        f["Tr0"] = _dev(Tr0, nc) if Tr0 is not None else None
        f["sigma_s"] = _dev(sigma_s, nc) if sigma_s is not None else None
        desc = _native.ProblemDesc()
        desc.ndim = ndim
        for a in range(3):
            desc.n[a] = self.n[a] if a < ndim else 1
            desc.L[a] = float(L[a]) if a < ndim else 1.0
            desc.bc[a] = int(bc[a]) if a < ndim else 0
        desc.n_theta, desc.n_phi = self.n_theta, self.n_phi
        desc.c, desc.a_r, desc.cfl, desc.dt = float(c), float(a_r), float(cfl), float(dt)
        for key in ("sigma_a", "cv", "T0", "Tr0", "sigma_s"):
            setattr(desc, key, f[key].data_ptr() if f[key] is not None else None)
        desc.eps, desc.max_rank = float(eps), int(max_rank or 0)
        desc.rounds_per_step, desc.precision = int(rounds_per_step), int(precision)
        desc.layout = int(layout)
        self.layout = int(layout)
        kinds = {"upwind": _native.TT_FLUX_UPWIND, "rusanov": _native.TT_FLUX_RUSANOV,
                 "hll": _native.TT_FLUX_HLL, "rusanov_tau": _native.TT_FLUX_RUSANOV_TAU}
        desc.flux = kinds[flux] if isinstance(flux, str) else int(flux)
        if desc.flux == _native.TT_FLUX_RUSANOV:
            desc.flux_param[0] = float(rusanov_s)
        elif desc.flux == _native.TT_FLUX_HLL:
            desc.flux_param[0], desc.flux_param[1] = float(hll_beta), float(hll_tau_threshold)
        elif desc.flux == _native.TT_FLUX_RUSANOV_TAU:
            desc.flux_param[0] = float(hll_beta)  # beta of Eq. tauc
        self._alloc = None
        if allocator == "torch":
            allocator = TorchAllocator()
        if allocator is not None:
            if not (hasattr(allocator, "alloc") and hasattr(allocator, "free")):
                raise ValueError("allocator must be None, 'torch' or an object with alloc() and free()")
            self._alloc = _c_allocator(allocator)
        if shard is not None:
            # a slab of layers [p0, p1) of axis 0 (tt_create_shard); shard =
            # (p0, p1, exchanger) with the exchanger's sum_ and halo_ methods
            from .shard import exchange_callback
            p0, p1, exchanger = int(shard[0]), int(shard[1]), shard[2]
            if allocator is not None:
                raise ValueError("a shard takes its device memory from the stream-ordered pool")
            self._xcb = exchange_callback(exchanger)
            check(lib.tt_create_shard(ctypes.byref(desc), _stream_ptr(stream), p0, p1, self._xcb, None,
                                      ctypes.byref(self._h)))
            self.shard = (p0, p1)
            self.n = (p1 - p0,) + self.n[1:]
            self.nc = nc // int(n[0]) * (p1 - p0)
        else:
            check(lib.tt_create_ex(ctypes.byref(desc), _stream_ptr(stream),
                                   ctypes.byref(self._alloc) if self._alloc is not None else None,
                                   ctypes.byref(self._h)))
        self._keep = f  # inputs stay alive until creation finished (copied in)

    @staticmethod
    def problem_kwargs(p):
        """Constructor keywords from a problem dict (grid, ordinates, constants,
        fields of shape n); an all-zero sigma_s is passed as absent."""
        sig_s = p.get("sigma_s")
        return dict(n=p["n"], L=p["L"], n_theta=p["n_theta"], n_phi=p["n_phi"],
                    sigma_a=p["sigma_a"].reshape(-1), cv=p["cv"].reshape(-1),
                    T0=p["T0"].reshape(-1), Tr0=p["Tr0"].reshape(-1),
                    sigma_s=(sig_s.reshape(-1) if sig_s is not None and np.any(sig_s) else None),
                    c=p["c"], a_r=p["a_r"], dt=p["dt"], bc=list(p["bc"]), eps=p["eps"],
                    max_rank=p.get("max_rank", 0))

    @classmethod
    def from_problem(cls, p, **over):
        kw = cls.problem_kwargs(p)
        kw.update(over)
        obj = cls(**kw)
        if p.get("sources"):
            obj.set_sources(p["sources"])
        for (axis, side), (g, th, ph) in sorted((p.get("inflow") or {}).items()):
            obj.set_inflow(axis, side, g, th, ph)
        return obj

    def set_inflow(self, axis, side, g=None, theta=None, phi=None):
        """Incoming intensity g (x) theta (x) phi on face ``side`` (0 low, 1 high)
        of a vacuum axis (tt_set_inflow); g=None removes it."""
        if g is None:
            check(lib.tt_set_inflow(self._h, int(axis), int(side), None, None, None))
            return
        gd = _dev(np.asarray(g).reshape(-1), self.nc)
        td, pd = _dev(theta, self.n_theta), _dev(phi, self.n_phi)
        check(lib.tt_set_inflow(self._h, int(axis), int(side), ctypes.c_void_p(gd.data_ptr()),
                                ctypes.c_void_p(td.data_ptr()), ctypes.c_void_p(pd.data_ptr())))

    def set_sources(self, sources):
        """Fixed external sources: a list of (x (N_c), theta (n_theta), phi (n_phi))
        array-likes, S = sum_k x_k (x) theta_k (x) phi_k added as c dt S per step."""
        k = len(sources)
        if k == 0:
            check(lib.tt_set_sources(self._h, 0, None, None, None))
            return
        x = torch.stack([_dev(np.asarray(s[0]).reshape(-1), self.nc) for s in sources]).contiguous()
        th = torch.stack([_dev(s[1], self.n_theta) for s in sources]).contiguous()
        ph = torch.stack([_dev(s[2], self.n_phi) for s in sources]).contiguous()
        check(lib.tt_set_sources(self._h, k, ctypes.c_void_p(x.data_ptr()),
                                 ctypes.c_void_p(th.data_ptr()), ctypes.c_void_p(ph.data_ptr())))

    def step(self, nsteps=1, flags=0, forced=None):
        info = StepInfo()
        check(lib.tt_sn_step_ex(self._h, int(nsteps), int(flags), _int_array(forced),
                                ctypes.byref(info)))
        self.steps_taken += int(nsteps)
        return info.as_dict()

    def energy(self, totals=True):
        """(E, T, (sum E dV, sum C_v T dV)) of this handle's cells.  On a spatial
        shard the totals are the whole grid's, summed through the exchange, so
        every shard must ask for them together; totals=False skips them (and
        the exchange) and returns None in their place."""
        E = torch.empty(self.nc, dtype=torch.float64, device="cuda")
        T = torch.empty(self.nc, dtype=torch.float64, device="cuda")
        tot = (ctypes.c_double * 2)()
        check(lib.tt_energy(self._h, ctypes.c_void_p(E.data_ptr()), ctypes.c_void_p(T.data_ptr()),
                            tot if totals else None))
        return E, T, ((tot[0], tot[1]) if totals else None)

    def set_T(self, T):
        t = _dev_or_host(T, self.nc)
        check(lib.tt_set_T(self._h, ctypes.c_void_p(t.data_ptr())))

    def compression(self):
        """Compression factor C of the current TT (Sec. 5.1)."""
        return compression_factor(self.dims()[1], self.ranks())

    def run(self, nsteps, log=None, time_steps=True):
        """Take ``nsteps`` steps one at a time and return one ``step_record``
        per step (ranks, discarded tails, compression, energies, GPU ms timed
        with CUDA events on the handle's stream); with ``log`` (a path or a
        writable file) the records are also written as JSON lines."""
        import json

        dims = self.dims()[1]
        stream = self.stream if self.stream is not None else torch.cuda.current_stream()
        out = []
        fh = open(log, "a") if isinstance(log, (str, os.PathLike)) else log
        try:
            for _ in range(int(nsteps)):
                ms = None
                if time_steps:
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                info = self.step()
                if time_steps:
                    e1.record(stream)
                    e1.synchronize()
                    ms = e0.elapsed_time(e1)
                _, _, totals = self.energy()
                rec = step_record(self.steps_taken, self.steps_taken * self.dt, info, totals, dims, ms)
                out.append(rec)
                if fh is not None:
                    fh.write(json.dumps(rec) + "\n")
                    fh.flush()
        finally:
            if fh is not None and fh is not log:
                fh.close()
        return out

    def state_dict(self):
        """Checkpoint of the evolving state: the TT cores and the material
        temperature (device copies; torch.save-able).  Fields, constants, the
        flux, sources and inflow faces are the problem's and are not saved."""
        return {"cores": [c.clone() for c in self.cores()], "T": self.energy(totals=False)[1].clone(),
                "steps_taken": self.steps_taken}

    def load_state_dict(self, state):
        """Resume from ``state_dict()``: the following steps continue bit for bit."""
        self.set_cores(state["cores"])
        self.set_T(state["T"])
        self.steps_taken = int(state.get("steps_taken", 0))

    def full(self):
        return super().full().reshape(self.n + (self.n_theta, self.n_phi))

    # -- adjoint form
    def tape_begin(self, checkpoint_every=1):
        """Record the following steps for the escape-energy gradient."""
        check(lib.tt_tape_begin(self._h, int(checkpoint_every)))

    def escape_energy(self):
        """(Q, taped steps): the boundary-escape energy of the taped steps so far."""
        q = ctypes.c_double()
        m = ctypes.c_int()
        check(lib.tt_tape_objective(self._h, ctypes.byref(q), ctypes.byref(m)))
        return q.value, m.value

    def escape_gradient(self):
        """Reverse sweep over the taped steps: (Q, dQ/dsigma_a as a CUDA tensor of
        N_c doubles).  Releases the tape; the state stays at the last step."""
        g = torch.empty(self.nc, dtype=torch.float64, device="cuda")
        q = ctypes.c_double()
        check(lib.tt_sn_step_adjoint(self._h, ctypes.c_void_p(g.data_ptr()), ctypes.byref(q)))
        return q.value, g

    def tape_clear(self):
        check(lib.tt_tape_clear(self._h))


class EscapeEnergy(torch.autograd.Function):
    """Q(sigma_a): the boundary-escape energy of ``steps`` TT-S_N steps from a
    problem's initial state, differentiable in sigma_a (a CUDA float64 tensor of
    N_c values).  ``problem`` holds TTSN keyword arguments other than sigma_a.
    Forward tapes the run (checkpoints every ``checkpoint_every`` steps);
    backward is the library's reverse sweep with the rounding factors frozen."""

    @staticmethod
    def forward(ctx, sigma_a, problem, steps, checkpoint_every=1):
        tt = TTSN(sigma_a=sigma_a.detach(), **problem)
        tt.tape_begin(checkpoint_every)
        tt.step(int(steps))
        q, _ = tt.escape_energy()
        ctx.tt = tt  # the taped run, reversed in backward
        ctx.sigma_shape = sigma_a.shape
        return torch.tensor(q, dtype=torch.float64, device=sigma_a.device)

    @staticmethod
    def backward(ctx, gq):
        if ctx.tt is None:
            raise RuntimeError("EscapeEnergy: the taped run was already reversed and released; "
                               "backward through it can run once (retain_graph cannot keep the tape)")
        _, grad = ctx.tt.escape_gradient()
        ctx.tt = None
        return (gq * grad).view(ctx.sigma_shape), None, None, None


def escape_energy(sigma_a, problem, steps, checkpoint_every=1):
    """Differentiable boundary-escape energy (see EscapeEnergy)."""
    return EscapeEnergy.apply(sigma_a, problem, steps, checkpoint_every)


class _BorrowedTTSN(TTSN):
    """View of one problem of a batch (the batch owns the handle)."""

    def __init__(self, h, n, n_theta, n_phi, dt=None):
        _Handle.__init__(self)
        self._h = h
        self.nc = 1
        for m in n:
            self.nc *= int(m)
        self.n = tuple(int(m) for m in n)
        self.n_theta, self.n_phi = int(n_theta), int(n_phi)
        self.dt = float(dt) if dt is not None else float("nan")
        self.steps_taken = 0

    def __del__(self):
        self._h = None  # owned by the batch


class TTSNBatch:
    """Independent TT-S_N problems of uneven sizes stepped together (each on its
    own stream, advanced concurrently by host threads in the library, or as
    captured steps with set_graph).  Many streams share the GPU's hardware
    work queues: with CUDA_DEVICE_MAX_CONNECTIONS (environment, read when the
    CUDA context is created; default 8) raised to 32 the 64-problem batch of
    the bench runs 1.25x (host threads) and 2x (captured) faster."""

    def __init__(self, problems, threads=0, precision=TT_FP64):
        keep = []
        descs = (_native.ProblemDesc * len(problems))()
        for i, p in enumerate(problems):
            nc = int(np.prod(p["n"]))
            f = {k: _dev(p[k].reshape(-1), nc) for k in ("sigma_a", "cv", "T0", "Tr0", "sigma_s")}
            keep.append(f)
            d = descs[i]
            ndim = len(p["n"])
            d.ndim = ndim
            for a in range(3):
                d.n[a] = int(p["n"][a]) if a < ndim else 1
                d.L[a] = float(p["L"][a]) if a < ndim else 1.0
                d.bc[a] = int(p["bc"][a]) if a < ndim else 0
            d.n_theta, d.n_phi = int(p["n_theta"]), int(p["n_phi"])
            d.c, d.a_r, d.cfl, d.dt = float(p["c"]), float(p["a_r"]), float(p.get("cfl", 0.5)), float(p["dt"])
            for key in ("sigma_a", "cv", "T0", "Tr0", "sigma_s"):
                setattr(d, key, f[key].data_ptr())
            d.eps, d.max_rank = float(p["eps"]), int(p.get("max_rank") or 0)
            d.rounds_per_step, d.precision = 1, int(precision)
        torch.cuda.synchronize()
        self._b = ctypes.c_void_p()
        check(lib.tt_batch_create(descs, len(problems), int(threads), ctypes.byref(self._b)))
        self.problems = problems
        self.count = len(problems)

    def __del__(self):
        b = getattr(self, "_b", None)
        if b is not None and b.value:
            lib.tt_batch_destroy(b)
            self._b = None

    def step(self, nsteps=1):
        infos = (StepInfo * self.count)()
        check(lib.tt_batch_step(self._b, int(nsteps), infos))
        return [x.as_dict() for x in infos]

    def sync(self):
        check(lib.tt_batch_sync(self._b))

    def set_graph(self, enable=True):
        """Captured steps for every problem (tt_batch_set_graph)."""
        check(lib.tt_batch_set_graph(self._b, int(bool(enable))))

    def problem(self, i):
        h = ctypes.c_void_p()
        check(lib.tt_batch_handle(self._b, int(i), ctypes.byref(h)))
        p = self.problems[i]
        return _BorrowedTTSN(h, p["n"], p["n_theta"], p["n_phi"], p.get("dt"))


def dgemm(A, B, trans_a=False, trans_b=False, alpha=1.0, stream=None):
    """C = alpha op(A) op(B) on the FP64 tensor pipe (library kernel)."""
    A, B = _dev(A), _dev(B)
    M = A.shape[1] if trans_a else A.shape[0]
    K = A.shape[0] if trans_a else A.shape[1]
    N = B.shape[0] if trans_b else B.shape[1]
    C = torch.empty((M, N), dtype=torch.float64, device="cuda")
    check(lib.tt_dgemm(int(trans_a), int(trans_b), M, N, K, float(alpha),
                       ctypes.c_void_p(A.data_ptr()), A.shape[1], ctypes.c_void_p(B.data_ptr()),
                       B.shape[1], 0.0, ctypes.c_void_p(C.data_ptr()), N, _stream_ptr(stream)))
    return C


def gram(A, stream=None):
    """G = A^T A (library split-K Gram kernel)."""
    A = _dev(A)
    m, n = A.shape
    G = torch.empty((n, n), dtype=torch.float64, device="cuda")
    check(lib.tt_gram(m, n, ctypes.c_void_p(A.data_ptr()), n, ctypes.c_void_p(G.data_ptr()), n,
                      _stream_ptr(stream)))
    return G


def gram_mixed(A, stream=None):
    """G = A^T A with exact BF16 digit products (library kernel, tt_gram_mixed)."""
    A = _dev(A)
    m, n = A.shape
    G = torch.empty((n, n), dtype=torch.float64, device="cuda")
    check(lib.tt_gram_mixed(m, n, ctypes.c_void_p(A.data_ptr()), n, ctypes.c_void_p(G.data_ptr()), n,
                            _stream_ptr(stream)))
    return G


def gemm_nt_mixed(A, B, stream=None):
    """C = A B^T with exact BF16 digit products (library kernel, tt_gemm_nt_mixed)."""
    A, B = _dev(A), _dev(B)
    M, K = A.shape
    N = B.shape[0]
    C = torch.empty((M, N), dtype=torch.float64, device="cuda")
    check(lib.tt_gemm_nt_mixed(M, N, K, ctypes.c_void_p(A.data_ptr()), K, ctypes.c_void_p(B.data_ptr()),
                               K, ctypes.c_void_p(C.data_ptr()), N, _stream_ptr(stream)))
    return C


def gram_noalloc(A, G=None, stream=None):
    """G = A^T A through tt_gram_noalloc: the library allocates nothing (the
    caller provides A and, optionally, the output G; n <= 1024)."""
    A = _dev(A)
    m, n = A.shape
    if G is None:
        G = torch.empty((n, n), dtype=torch.float64, device=A.device)
    else:
        # the library gets only a raw pointer and writes n rows of n doubles
        # at stride ldg: refuse any G that cannot hold them
        if not isinstance(G, torch.Tensor) or G.dtype != torch.float64:
            raise ValueError("G must be a float64 tensor")
        if G.device != A.device:
            raise ValueError("G is on %s, A on %s" % (G.device, A.device))
        if tuple(G.shape) != (n, n):
            raise ValueError("G must have shape (%d, %d), got %s" % (n, n, tuple(G.shape)))
        if n > 0 and (G.stride(1) != 1 or G.stride(0) < n):
            raise ValueError("G must be row-major with unit column stride and row stride >= n")
    ldg = int(G.stride(0)) if n > 0 else n
    check(lib.tt_gram_noalloc(m, n, ctypes.c_void_p(A.data_ptr()), n, ctypes.c_void_p(G.data_ptr()),
                              ldg, _stream_ptr(stream)))
    return G


def pchol(G, stream=None):
    """(W with W^T W = G, rank): pivoted Cholesky of a symmetric PSD matrix,
    stopped at eps_mach times the largest diagonal entry (tt_pchol)."""
    G = _dev(G)
    n = G.shape[0]
    W = torch.empty((n, n), dtype=torch.float64, device="cuda")
    rank = ctypes.c_int()
    check(lib.tt_pchol(n, ctypes.c_void_p(G.data_ptr()), n, ctypes.c_void_p(W.data_ptr()),
                       _stream_ptr(stream), ctypes.byref(rank)))
    return W[: rank.value].clone(), rank.value


def syev(G, stream=None, allow_unconverged=False, max_sweeps=40):
    """(lam descending, Vt with eigenvectors as rows, sweeps) by parallel Jacobi
    with at most max_sweeps sweeps (tt_syev_ex)."""
    G = _dev(G)
    n = G.shape[0]
    lam = torch.empty(n, dtype=torch.float64, device="cuda")
    Vt = torch.empty((n, n), dtype=torch.float64, device="cuda")
    sweeps = ctypes.c_int()
    st = lib.tt_syev_ex(n, ctypes.c_void_p(G.data_ptr()), n, ctypes.c_void_p(lam.data_ptr()),
                        ctypes.c_void_p(Vt.data_ptr()), n, int(max_sweeps), _stream_ptr(stream),
                        ctypes.byref(sweeps))
    if not (allow_unconverged and st == -4):
        check(st)
    return lam, Vt, sweeps.value


def syev_psd(K, stream=None, allow_unconverged=False, max_sweeps=40):
    """(lam descending, Vt with eigenvectors as rows, sweeps) of a positive
    semidefinite K by pivoted Cholesky and one-sided Jacobi (tt_syev_psd)."""
    K = _dev(K)
    n = K.shape[0]
    lam = torch.empty(n, dtype=torch.float64, device="cuda")
    Vt = torch.empty((n, n), dtype=torch.float64, device="cuda")
    sweeps = ctypes.c_int()
    st = lib.tt_syev_psd(n, ctypes.c_void_p(K.data_ptr()), n, ctypes.c_void_p(lam.data_ptr()),
                         ctypes.c_void_p(Vt.data_ptr()), n, int(max_sweeps), _stream_ptr(stream),
                         ctypes.byref(sweeps))
    if not (allow_unconverged and st == -4):
        check(st)
    return lam, Vt, sweeps.value


def autotune(path=None, stream=None):
    """Measure the FP64 products' split of K per (tiles, depth) bucket on this
    GPU and install the table (tt_autotune); returns it as a list and, with
    path, stores it as JSON for load_autotune."""
    import json

    buf = (ctypes.c_int * _native.TT_AUTOTUNE_ENTRIES)()
    check(lib.tt_autotune(_stream_ptr(stream), buf))
    table = list(buf)
    if path is not None:
        with open(path, "w") as fh:
            json.dump({"layout": "index floor(log2 tiles) * 22 + floor(log2 K); 0 = built-in rule",
                       "splits": table}, fh)
    return table


def load_autotune(path_or_table):
    """Install a stored autotune table (a JSON file from autotune(path) or a list)."""
    import json

    table = path_or_table
    if isinstance(path_or_table, (str, os.PathLike)):
        with open(path_or_table) as fh:
            table = json.load(fh)["splits"]
    buf = (ctypes.c_int * len(table))(*[int(x) for x in table])
    check(lib.tt_set_autotune_table(buf, len(table)))


def autotune_table():
    """The installed autotune table (all zero: the built-in rule)."""
    buf = (ctypes.c_int * _native.TT_AUTOTUNE_ENTRIES)()
    check(lib.tt_get_autotune_table(buf, _native.TT_AUTOTUNE_ENTRIES))
    return list(buf)


def kernel_launches():
    """Kernels launched by libttsn in this process so far."""
    return int(lib.tt_kernel_launches())


def fp64_mma_peak(stream=None):
    """Measured FP64 tensor-pipe throughput of this GPU in TFLOP/s."""
    v = ctypes.c_double()
    check(lib.tt_bench_fp64_mma(ctypes.byref(v), _stream_ptr(stream)))
    return v.value


def bf16_mma_peak(stream=None):
    """Measured warp-level BF16 tensor MMA (mma.sync) throughput in TFLOP/s."""
    v = ctypes.c_double()
    check(lib.tt_bench_bf16_mma(ctypes.byref(v), _stream_ptr(stream)))
    return v.value
