#!/usr/bin/env python
"""Benchmark of the TT-S_N step-then-truncate time step on GB300.

Workload (default ``blob_3d``): 3D 128^3 cells on [0,1]^3, 32 x 64 ordinates
(2048), sigma_a = 1e2 inside a seeded union of 16 spheres and 1e-2 elsewhere,
T = 1 in a sphere of radius 0.1 at the centre and 1e-3 outside, radiation in
equilibrium with T, vacuum boundaries, CFL 0.5, eps = 1e-6, ranks capped at
128, FP64.  The intensity is held in the paper's three-core layout
(X: N_c x r1, Theta: r1 x 32 x r2, Phi: r2 x 64).

A "step" is one full time step (transport core apply, quadrature, quartic,
source assembly, Gram-SVD rounding, energy-conserving temperature update).
Warm-up: W steps of the same trajectory on the same handle, after which the
state is reset to t = 0; then exactly K steps (steps 1..K of the trajectory)
are timed with CUDA events on the library's stream, bracketed by a barrier and
torch.cuda.synchronize().  The grown spatial core (>= N_c x 8 doubles = 134 MB
from the first step, GBs later) is larger than L2, so no flush is added.

Reported: steps/s (value), equivalent cell-ordinate updates/s, an end-to-end
number through the public API with host-resident state, per-phase GPU times,
the roofline of the dominant kernel family, SM clocks sampled during the timed
region, the library's kernel launches, and the FP64 oracle timed on a bounded
sample on the host cores (``cpu_baseline``).  ``--impl reference`` times the
oracle itself (the slow CPU program) on the same metric.

Multi-GPU: the step does not shard here (one problem per GPU); ``--gpus N``
under torchrun runs N independent replicas ("scaling": "weak").
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# hardware work queues for the batched leg's 64 streams (the default 8 makes
# unrelated streams wait on one another); read when the CUDA context is made
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

import workloads  # noqa: E402

METRIC = "TT-SN steps/s (equiv. cell·ordinate updates/s), mixed vs FP64 at stated err"
DEFAULT_STEPS = 12
DEFAULT_WARMUP = 3
OVERSAMPLE = 8  # extra sketch columns of the randomized-rounding companion run


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=DEFAULT_STEPS)
    ap.add_argument("--warmup", type=int, default=DEFAULT_WARMUP)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="blob_3d", choices=["blob_3d", "small_2d"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true", help="skip the precision-form companion run")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-form leg")
    ap.add_argument("--batch-steps", type=int, default=5)
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint-form leg")
    ap.add_argument("--no-beams", action="store_true", help="skip the crossing-beam precision leg")
    ap.add_argument("--beams-preroll", type=int, default=100)
    ap.add_argument("--beams-steps", type=int, default=20)
    ap.add_argument("--no-split", action="store_true", help="skip the split-layout leg")
    ap.add_argument("--split-steps", type=int, default=5, help="timed steps of the 3D split-layout run")
    ap.add_argument("--no-fluxes", action="store_true", help="skip the Rusanov/HLL leg")
    ap.add_argument("--no-schedule", action="store_true", help="skip the rounds-per-step leg")
    ap.add_argument("--no-line-source", action="store_true", help="skip the line-source leg")
    ap.add_argument("--line-source-steps", type=int, default=121,
                    help="timed steps of the line-source leg (0: to t = 1, 568 steps)")
    ap.add_argument("--no-randomized", action="store_true", help="skip the randomized-rounding companion run")
    ap.add_argument("--no-ttsvd", action="store_true", help="skip the TT-SVD against Gram-SVD rounding comparison")
    ap.add_argument("--no-autotune", action="store_true", help="keep the built-in split rule (no tt_autotune)")
    ap.add_argument("--only", choices=["adjoint", "beams", "batch", "split", "fluxes", "schedule", "line_source"], default=None,
                    help="run only this companion leg and print its JSON (profiling)")
    ap.add_argument("--cpu-budget", type=float, default=20.0, help="seconds of oracle work for cpu_baseline")
    ap.add_argument("--ref-budget", type=float, default=120.0,
                    help="seconds of oracle stepping for --impl reference")
    ap.add_argument("--json-out", default=None)
    return ap.parse_args()


def workload_desc(p):
    nd = len(p["n"])
    return ("%s: %dD %s cells, %dx%d ordinates, layout grouped-space 3 cores (X,Theta,Phi), "
            "eps=%g, rank cap %s, %s boundaries, CFL %g, FP64" % (
                p["name"], nd, "x".join(str(m) for m in p["n"]), p["n_theta"], p["n_phi"],
                p["eps"], p.get("max_rank"), "vacuum" if p["bc"][0] == 1 else "periodic", p["cfl"]))


def cells_ordinates(p):
    return int(np.prod(p["n"])) * p["n_theta"] * p["n_phi"]


# ---------------------------------------------------------------- clocks
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        with open(self.f.name) as fh:
            lines = fh.readlines()
        os.unlink(self.f.name)
        return parse_clock_rows(lines)


def parse_clock_rows(lines):
    """Summary of nvidia-smi samples in ClockSampler.QUERY order (csv, no
    header, no units): median SM clock under load, the largest max clock, the
    throttle reasons seen active at least once, the sample count and the
    median power; None without samples."""
    rows = []
    for line in lines:
        parts = [x.strip() for x in line.split(",")]
        if len(parts) >= 9:
            rows.append(parts)
    if not rows:
        return None
    sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
    mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
    pw = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
    return {"sm_mhz": statistics.median(sm) if sm else None,
            "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows),
            "power_w_median": statistics.median(pw) if pw else None}


# ---------------------------------------------------------------- ours
def run_ours(args, rank, world, local_rank):
    import torch

    import paper_2503_18056_gb300 as ttsn

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    p = workloads.problem(args.workload)
    stream = torch.cuda.Stream(device=dev)
    tune = None
    if not args.no_autotune:
        # the products' split per (tiles, depth) bucket, measured on this GPU
        # before anything is timed; every leg below runs with it
        t_tune = time.perf_counter()
        table = ttsn.autotune(stream=stream)
        torch.cuda.synchronize()
        tune = {"s": round(time.perf_counter() - t_tune, 2), "table": table,
                "layout": "index floor(log2 tiles) * 22 + floor(log2 K); 0 = built-in rule"}
    with torch.cuda.stream(stream):
        g = ttsn.TTSN.from_problem(p, max_rank=p.get("max_rank", 0), stream=stream)
        init_cores = [c.clone() for c in g.cores()]
        _, T0, _ = g.energy()
        T0 = T0.clone()
        g.profile(False)

        def reset():
            g.set_cores(init_cores)
            g.set_T(T0)

        # warm-up: the first W steps of the trajectory, then back to t = 0
        for _ in range(args.warmup):
            g.step()
        reset()
        fp64_peak = ttsn.fp64_mma_peak(stream) if rank == 0 else None
        torch.cuda.synchronize()

        g.profile(True)
        clocks = ClockSampler(local_rank)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        ranks_hist = []
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()
        clocks.start()
        l0 = ttsn.kernel_launches()
        ev[0].record(stream)
        for k in range(args.steps):
            info = g.step()
            ev[k + 1].record(stream)
            ranks_hist.append(info["ranks"][1:-1])
        torch.cuda.synchronize()
        launches = ttsn.kernel_launches() - l0
        if world > 1:
            dist.barrier()
        clk = clocks.stop()
        step_ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
        total_ms = ev[0].elapsed_time(ev[args.steps])
        prof = g.profile_read()
        g.profile(False)
        E, T, tot = g.energy()

        # precision form on the same steps, replaying the FP64 run's ranks
        mixed = None
        if not args.no_mixed:
            E64, T64 = E.clone(), T.clone()
            gm = ttsn.TTSN.from_problem(p, max_rank=p.get("max_rank", 0), stream=stream,
                                        precision=ttsn.TT_MIXED)
            for _ in range(args.warmup):
                gm.step()
            gm.set_cores(init_cores)
            gm.set_T(T0)
            bf16_peak = ttsn.bf16_mma_peak(stream) if rank == 0 else None
            torch.cuda.synchronize()
            gm.profile(True)
            evm = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
            mclocks = ClockSampler(local_rank)
            torch.cuda.synchronize()
            mclocks.start()
            evm[0].record(stream)
            for k in range(args.steps):
                gm.step(forced=ranks_hist[k])
                evm[k + 1].record(stream)
            torch.cuda.synchronize()
            mclk = mclocks.stop()
            mx_ms = evm[0].elapsed_time(evm[args.steps])
            mprof = gm.profile_read()
            gm.profile(False)
            Em, Tm, _ = gm.energy()
            err_E = ((Em - E64).abs().max() / E64.abs().max()).item()
            err_T = ((Tm - T64).abs().max() / T64.abs().max()).item()
            mixed = dict(total_ms=mx_ms, step_ms=[evm[k].elapsed_time(evm[k + 1]) for k in range(args.steps)],
                         prof=mprof, err_E=err_E, err_T=err_T, bf16_peak=bf16_peak, clocks=mclk)
            del gm
            torch.cuda.synchronize()

        # randomized rounding (App. A.3) on the same steps at the FP64 run's
        # ranks, with a Gaussian sketch at the rank cap drawn on the device
        randomized = None
        if not args.no_randomized:
            E64, T64 = E.clone(), T.clone()
            gr = ttsn.TTSN.from_problem(p, max_rank=p.get("max_rank", 0), stream=stream)
            d_, n_ = gr.dims()
            cap = (p.get("max_rank") or 128) + OVERSAMPLE
            sk = [1] + [min(cap, int(np.prod(n_[:k + 1])), int(np.prod(n_[k + 1:]))) for k in range(d_ - 1)] + [1]
            r_over = [[min(r + OVERSAMPLE, sk[b + 1]) for b, r in enumerate(rk)] for rk in ranks_hist]
            gen = torch.Generator(device=dev).manual_seed(1234)
            omega = [torch.randn((sk[k], n_[k], sk[k + 1]), dtype=torch.float64, device=dev, generator=gen)
                     for k in range(d_)]
            gr.set_sketch(omega)
            del omega
            gr.set_rounding("randomized")
            for k in range(args.warmup):
                gr.step(forced=r_over[k])
            gr.set_cores(init_cores)
            gr.set_T(T0)
            torch.cuda.synchronize()
            gr.profile(True)
            evr = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
            evr[0].record(stream)
            for k in range(args.steps):
                gr.step(forced=r_over[k])
                evr[k + 1].record(stream)
            torch.cuda.synchronize()
            rprof = gr.profile_read()
            gr.profile(False)
            Er, Tr, _ = gr.energy()
            r_ms = evr[0].elapsed_time(evr[args.steps])
            randomized = dict(total_ms=r_ms, prof=rprof,
                              err_E=((Er - E64).abs().max() / E64.abs().max()).item(),
                              err_T=((Tr - T64).abs().max() / T64.abs().max()).item())
            del gr
            torch.cuda.synchronize()

        # QR-based TT-SVD rounding (App. A.1) against the Gram-SVD rounding on
        # one step from the same capped state (the end of the FP64 run): the
        # paper's cost comparison of the two roundings (Sec. 4.2, Table 3)
        ttsvd = None
        if not args.no_ttsvd:
            cap_cores = [c.clone() for c in g.cores()]
            _, cap_T, _ = g.energy()
            cap_T = cap_T.clone()
            legs = {}
            for method in ("gram", "ttsvd"):
                gt = ttsn.TTSN.from_problem(p, max_rank=p.get("max_rank", 0), stream=stream)
                gt.set_rounding(method)
                forced = legs["gram"]["ranks"] if method == "ttsvd" else None
                for timed in (False, True):  # the first step sizes the buffers
                    gt.set_cores(cap_cores)
                    gt.set_T(cap_T)
                    torch.cuda.synchronize()
                    gt.profile(timed)
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    info = gt.step(forced=forced)
                    e1.record(stream)
                    torch.cuda.synchronize()
                tprof = gt.profile_read()
                gt.profile(False)
                Et, _, _ = gt.energy()
                legs[method] = dict(ms=e0.elapsed_time(e1), ranks=info["ranks"][1:-1], E=Et.clone(),
                                    rounding_ms=sum(v["ms"] for k_, v in tprof.items()
                                                    if k_ not in ("transport", "energy")),
                                    phases={k_: round(v["ms"], 3) for k_, v in tprof.items()})
                del gt
                torch.cuda.synchronize()
            Eg, Ets = legs["gram"].pop("E"), legs["ttsvd"].pop("E")
            ttsvd = dict(legs=legs, err_E=((Ets - Eg).abs().max() / Eg.abs().max()).item(), step=args.steps + 1)
            del cap_cores
            torch.cuda.synchronize()

        # end to end through the public API: the state lives on the host between
        # steps (pinned), copied in before and out after every step
        e2e = None
        if not args.no_e2e:
            # pinned host buffers at the rank cap, allocated before the timed
            # region; each step's cores are copied out into views of them and
            # read back in from there by the library (no device staging)
            _, dims = g.dims()
            cap = int(p.get("max_rank") or 0) or min(dims[0], dims[1] * dims[2])
            caps = [dims[0] * cap, cap * dims[1] * cap, cap * dims[2]]
            pool = [torch.empty(max(c_, 1), dtype=torch.float64).pin_memory() for c_ in caps]
            host_cores = []
            for k_, c in enumerate(init_cores):
                hv = pool[k_][:c.numel()].view(c.shape)
                hv.copy_(c)
                host_cores.append(hv)
            host_T = T0.cpu().pin_memory()
            h2d = d2h = 0
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for k in range(args.steps):
                g.set_cores(host_cores)
                g.set_T(host_T)
                h2d += sum(c.numel() for c in host_cores) * 8 + host_T.numel() * 8
                g.step()
                host_cores = g.cores(into=pool)  # straight into the pinned buffers
                _, Td, _ = g.energy()
                host_T.copy_(Td, non_blocking=True)
                torch.cuda.synchronize()
                d2h += sum(c.numel() for c in host_cores) * 8 + host_T.numel() * 8
            torch.cuda.synchronize()
            e2e_s = time.perf_counter() - t0
            e2e = {"value": args.steps / e2e_s, "unit": "steps/s",
                   "h2d_bytes_per_step": h2d // args.steps, "d2h_bytes_per_step": d2h // args.steps}
    batched = None
    if not args.no_batch:
        batched = run_batch(args, torch, ttsn)
    adjoint = None
    if not args.no_adjoint:
        adjoint = run_adjoint(args, torch, ttsn)
    split = None
    if not args.no_split:
        split = run_split(args, torch, ttsn)
    fluxes = None
    if not args.no_fluxes:
        fluxes = run_fluxes(args, torch, ttsn)
    schedule = None
    if not args.no_schedule:
        schedule = run_schedule(args, torch, ttsn)
    line_source = None
    if not args.no_line_source:
        line_source = run_line_source(args, torch, ttsn)
    beams = None
    if not args.no_beams:
        beams = run_beams(args, torch, ttsn, fp64_peak, mixed["bf16_peak"] if mixed else None)
    res = dict(total_ms=total_ms, step_ms=step_ms, ranks=ranks_hist, prof=prof, launches=launches, autotune=tune,
               clocks=clk, e2e=e2e, fp64_peak=fp64_peak, totals=tot, p=p, mixed=mixed, batched=batched,
               adjoint=adjoint, beams=beams, split=split, fluxes=fluxes, schedule=schedule, line_source=line_source,
               randomized=randomized, ttsvd=ttsvd)
    return res


def run_beams(args, torch, ttsn, fp64_peak, bf16_peak):
    """Precision form on the crossing-beam workload (256^2 cells, 64 x 128
    ordinates, two collimated sources, eps 1e-5, ranks <= 96): P untimed FP64
    steps into the crossing regime, then K_p FP64 steps and the same K_p steps
    in the precision form from the same state at the FP64 ranks, each timed
    with CUDA events on its handle's stream; E and T compared after them."""
    p = workloads.crossing_beams()
    stream = torch.cuda.Stream()
    kp = args.beams_steps
    with torch.cuda.stream(stream):
        g = ttsn.TTSN.from_problem(p, stream=stream)
        g.step(args.beams_preroll)
        start = [c.clone() for c in g.cores()]
        T0 = g.energy()[1].clone()
        gm = ttsn.TTSN.from_problem(p, stream=stream, precision=ttsn.TT_MIXED)
        gm.step(3)  # warm-up of the precision form's kernels
        out = {}
        ranks = []
        for name, h in (("fp64", g), ("mixed", gm)):
            h.set_cores(start)
            h.set_T(T0)
            torch.cuda.synchronize()
            h.profile(True)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for k in range(kp):
                if name == "fp64":
                    ranks.append(h.step()["ranks"][1:-1])
                else:
                    h.step(forced=ranks[k])
            e1.record(stream)
            torch.cuda.synchronize()
            out[name] = (e0.elapsed_time(e1), h.profile_read())
            h.profile(False)
        E64, T64, _ = g.energy()
        Em, Tm, _ = gm.energy()
    upd = int(np.prod(p["n"])) * p["n_theta"] * p["n_phi"]
    v64 = kp / (out["fp64"][0] * 1e-3)
    vmx = kp / (out["mixed"][0] * 1e-3)
    roof = tc_gram_roofline(out["mixed"][1]["gram_left"], read_peaks())
    return {"workload": "crossing beams: 2D 256^2 cells, 64x128 ordinates, two collimated 4x4-cell "
                        "sources (x=0 edge toward +x, y=0 edge toward +y, +-10 deg windows, strengths "
                        "1 and 0.5), sigma_a 1e-3, T 1e-3, vacuum, eps 1e-5, ranks <= 96; steps %d..%d"
                        % (args.beams_preroll + 1, args.beams_preroll + kp),
            "fp64_steps_per_s": v64, "mixed_steps_per_s": vmx, "speedup": vmx / v64,
            "fp64_updates_per_s": v64 * upd, "mixed_updates_per_s": vmx * upd,
            "err_vs_fp64": {"E_max_rel": float((Em - E64).abs().max() / E64.abs().max()),
                            "T_max_rel": float((Tm - T64).abs().max() / T64.abs().max())},
            "ranks_last": ranks[-1],
            "phases_ms": {n: {k: round(v["ms"], 3) for k, v in out[n][1].items()} for n in out},
            "mixed_roofline": roof}


def run_split(args, torch, ttsn):
    """Split-space layout (one core per spatial axis, then theta and phi).
    (a) The 2D 32^2 x (8 x 16) Gaussian-pulse problem as four cores (x, y,
    theta, phi), 10 steps from t = 0 at eps 1e-8, beside the same steps in the
    grouped three-core layout; (b) a 3D 128^3 x (32 x 64) problem as five cores
    with uniform sigma_a = 1 (the split layout needs a uniform absorption
    factor), the hot sphere, vacuum, eps 1e-6, ranks <= 128: 2 warm-up steps,
    then K_s timed steps.  CUDA events on each handle's stream."""
    out = {}
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        p = workloads.problem("small_2d")
        res2 = {}
        for name, layout in (("split", ttsn.TT_LAYOUT_SPLIT), ("grouped", ttsn.TT_LAYOUT_GROUPED)):
            ttsn.TTSN.from_problem(p, layout=layout, stream=stream).step(p["steps"])  # warm-up
            g = ttsn.TTSN.from_problem(p, layout=layout, stream=stream)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            l0 = ttsn.kernel_launches()
            e0.record(stream)
            info = g.step(p["steps"])
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            res2[name] = {"steps_per_s": p["steps"] / (ms * 1e-3), "ms_per_step": ms / p["steps"],
                          "gpu_launches": ttsn.kernel_launches() - l0,
                          "ranks_last": info["ranks"][1:-1]}
        upd = int(np.prod(p["n"])) * p["n_theta"] * p["n_phi"]
        for v in res2.values():
            v["updates_per_s"] = v["steps_per_s"] * upd
        out["small_2d"] = dict(workload="2D 32^2 cells, 8x16 ordinates, sigma_a 1, Gaussian T pulse, "
                                        "periodic, CFL 0.5, eps 1e-8, steps 1..10; split = 4 cores "
                                        "(x, y, theta, phi), grouped = 3 cores", **res2)
        n = (128, 128, 128)
        p3 = workloads.problem("blob_3d", sigma_a=np.ones(n))
        g = ttsn.TTSN.from_problem(p3, layout=ttsn.TT_LAYOUT_SPLIT, stream=stream)
        r0 = g.ranks()
        g.step(2)
        torch.cuda.synchronize()
        g.profile(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ranks = []
        for _ in range(args.split_steps):
            ranks.append(g.step()["ranks"][1:-1])
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        prof = g.profile_read()
        g.profile(False)
        upd3 = int(np.prod(n)) * p3["n_theta"] * p3["n_phi"]
        v = args.split_steps / (ms * 1e-3)
        out["sphere_3d"] = {"workload": "3D 128^3 cells, 32x64 ordinates, 5 cores (x, y, z, theta, phi), "
                                        "uniform sigma_a 1, hot sphere T 1 (r 0.1) in 1e-3, vacuum, CFL 0.5, "
                                        "eps 1e-6, ranks <= 128; steps 3..%d" % (2 + args.split_steps),
                            "steps_per_s": v, "updates_per_s": v * upd3, "ms_per_step": ms / args.split_steps,
                            "ranks_initial": r0[1:-1], "ranks": ranks,
                            "phases_ms": {k: round(x["ms"], 3) for k, x in prof.items()}}
    return out


def run_fluxes(args, torch, ttsn):
    """The Rusanov and HLL fluxes on the paper's Gaussian-diffusion setup, and
    the hohlraum of Sec. 5.1 (inflow faces).  Diffusion:
    (128^2 cells on 5 x 5, 8 x 16 ordinates, rho kappa_s = 1e3, no absorption,
    t0 = 200, eps 1e-6): Rusanov at S+ = 0 (the paper's choice), HLL
    (beta 1, tau_threshold 1) and Rusanov with the optical-depth speed
    S+ = c |n| min(1, 1/tau_c) (beta 1); K_f steps from the initial state timed with
    CUDA events after an untimed run of the same length, then E compared
    with the analytic solution A / (4 pi D (t0 + t)) exp(-r^2 / (4 D (t0 + t)))."""
    p = workloads.gaussian_diffusion()
    kf = 400
    xc = workloads.cell_centres(p["n"], p["L"])
    r2 = sum((x - c0) ** 2 for x, c0 in zip(xc, p["centre"]))
    s4 = 4.0 * p["D"] * (p["t0"] + kf * p["dt"])
    Ea = (p["amp"] / (np.pi * s4) * np.exp(-r2 / s4)).reshape(-1)
    stream = torch.cuda.Stream()
    out = {"workload": "Gaussian diffusion: 2D 128^2 cells on 5x5, 8x16 ordinates, sigma_s 1e3, sigma_a 0, "
                       "t0 200, vacuum, CFL 0.5, eps 1e-6; steps 1..%d" % kf}
    with torch.cuda.stream(stream):
        for name, kw in (("rusanov_s0", dict(flux="rusanov", rusanov_s=0.0)),
                         ("hll", dict(flux="hll", hll_beta=1.0, hll_tau_threshold=1.0)),
                         ("rusanov_tau", dict(flux="rusanov_tau", hll_beta=1.0))):
            ttsn.TTSN.from_problem(p, stream=stream, **kw).step(kf)  # warm-up
            g = ttsn.TTSN.from_problem(p, stream=stream, **kw)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info = g.step(kf)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            E, _, _ = g.energy()
            v = kf / (ms * 1e-3)
            out[name] = {"steps_per_s": v, "updates_per_s": v * int(np.prod(p["n"])) * p["n_theta"] * p["n_phi"],
                         "E_rel_l2_err_vs_analytic": float(np.linalg.norm(E.cpu().numpy() - Ea) / np.linalg.norm(Ea)),
                         "ranks_last": info["ranks"][1:-1]}
        # the hohlraum of Sec. 5.1: inflow faces, upwinding, to t = 0.75
        h = workloads.hohlraum()
        steps = int(round(h["t_lim"] / h["dt"]))
        ttsn.TTSN.from_problem(h, stream=stream).step(8)  # warm-up
        g = ttsn.TTSN.from_problem(h, stream=stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info = g.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        E, _, _ = g.energy()
        J = h["c"] * E.cpu().numpy().reshape(h["n"]) / (4 * np.pi)
        xc = workloads.cell_centres(h["n"], h["L"])
        Ja = _hohlraum_J(steps * h["dt"], xc[0], xc[1], h["c"])
        sub = (xc[0] < 1.0) & (xc[1] < 1.0)
        v = steps / (ms * 1e-3)
        out["hohlraum"] = {"workload": "hohlraum (Sec. 5.1): 2D 256^2 on [0,2]^2, 32x64 ordinates, unit isotropic "
                                      "inflow on x = 0 and y = 0, vacuum, upwind, eps 1e-4, steps 1..%d (t = 0.75)" % steps,
                           "steps_per_s": v, "updates_per_s": v * int(np.prod(h["n"])) * h["n_theta"] * h["n_phi"],
                           "J_L1_err_vs_analytic": float(np.mean(np.abs(J - Ja)[sub])),
                           "ranks_last": info["ranks"][1:-1]}
    return out


def _hohlraum_J(t, x, y, c=1.0):
    """Analytic mean intensity of the hohlraum (Sec. 5.1): unit isotropic
    inflow through the x = 0 and y = 0 faces of an empty domain."""
    def part(u, v):
        ct = c * t
        with np.errstate(invalid="ignore", divide="ignore"):
            eta = np.arccos(np.minimum(v / np.sqrt(np.maximum(ct ** 2 - u ** 2, 1e-300)), 1.0))
            r = np.sqrt(u ** 2 + v ** 2)
            val = 0.5 - (np.pi - eta) * u / (2 * np.pi * ct) - np.arcsin(u * np.sin(eta) / r) / (2 * np.pi)
        return np.where(u < ct, val, 0.0)
    return part(x, y) + part(y, x)


def run_line_source(args, torch, ttsn):
    """The line source of Sec. 5.4 at the paper's size: 500^2 cells on
    [-1.1, 1.1]^2, 32 x 64 ordinates, Gaussian pulse (width 0.03, U0 = 1), no
    material, vacuum, CFL 0.4, eps 1e-4, the first K_ls steps (to t = 1 with
    --line-source-steps 0), timed with CUDA events after a short untimed run,
    in FP64 and in the precision form (free ranks).  Reported beside the
    paper's figures: the ranks after 120 steps and at the end, the change of
    the radiation energy sum_i E_i dV relative to U0 (rounding moves energy
    between E and T; the front stays inside the domain), and the phases of
    two further profiled steps."""
    p = workloads.line_source()
    steps = int(round(p["t_lim"] / p["dt"]))
    if args.line_source_steps > 0:
        steps = max(121, min(steps, args.line_source_steps))
    stream = torch.cuda.Stream()
    upd = int(np.prod(p["n"])) * p["n_theta"] * p["n_phi"]
    out = {"workload": "line source (Sec. 5.4): 2D 500^2 on [-1.1,1.1]^2, 32x64 ordinates, Gaussian pulse "
                       "width 0.03, U0 1, sigma 0, vacuum, upwind, CFL 0.4, eps 1e-4, steps 1..%d (t = %.3g)"
                       % (steps, steps * p["dt"])}
    E = {}
    with torch.cuda.stream(stream):
        for name, prec in (("fp64", ttsn.TT_FP64), ("mixed", ttsn.TT_MIXED)):
            ttsn.TTSN.from_problem(p, stream=stream, precision=prec).step(8)  # warm-up
            g = ttsn.TTSN.from_problem(p, stream=stream, precision=prec)
            _, _, (e_rad0, _) = g.energy()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info120 = g.step(120)
            info = g.step(steps - 120)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            E[name], _, (e_rad, _) = g.energy()
            g.profile(True)
            g.step(2)
            prof = g.profile_read()
            g.profile(False)
            v = steps / (ms * 1e-3)
            out[name] = {"steps_per_s": v, "updates_per_s": v * upd, "ms_per_step": ms / steps,
                         "ranks_step_120": info120["ranks"][1:-1], "ranks_last": info["ranks"][1:-1],
                         "radiation_energy_change_over_U0": float(abs(e_rad - e_rad0) / p["U0"]),
                         "phases_ms_2_steps": {k: round(x["ms"], 3) for k, x in prof.items()}}
    out["mixed"]["speedup_vs_fp64"] = out["mixed"]["steps_per_s"] / out["fp64"]["steps_per_s"]
    out["mixed"]["E_max_rel_diff_vs_fp64_free_ranks"] = float((E["mixed"] - E["fp64"]).abs().max() / E["fp64"].abs().max())
    return out


def run_schedule(args, torch, ttsn):
    """Rounds per step (Sec. 4.2): the default single rounding after the source
    stage against the paper's schedule of rounding after transport and again
    after the source, on the 128^2 x (32 x 64) random-field problem (20
    steps, eps 1e-6), each timed with CUDA events after an untimed run."""
    p = workloads.grf_problem()
    stream = torch.cuda.Stream()
    out = {"workload": "2D 128^2, 32x64 ordinates, sigma_a = exp(GRF), vacuum, eps 1e-6, steps 1..%d" % p["steps"]}
    E = {}
    with torch.cuda.stream(stream):
        for rounds in (1, 2):
            ttsn.TTSN.from_problem(p, stream=stream, rounds_per_step=rounds).step(p["steps"])
            g = ttsn.TTSN.from_problem(p, stream=stream, rounds_per_step=rounds)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info = g.step(p["steps"])
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            E[rounds] = g.energy()[0]
            out["rounds_%d" % rounds] = {"steps_per_s": p["steps"] / (ms * 1e-3), "ranks_last": info["ranks"][1:-1]}
    out["E_max_rel_diff"] = float((E[2] - E[1]).abs().max() / E[1].abs().max())
    return out


def run_adjoint(args, torch, ttsn):
    """Adjoint form: gradient of the boundary-escape energy of 20 steps of the
    128^2 x (32 x 64) random-field problem (eps 1e-6, checkpoints every 5 steps)
    with respect to sigma_a.  One untimed warm-up gradient, then the taped
    forward, the reverse sweep and an untaped forward, each timed with CUDA
    events on the problem's stream."""
    p = workloads.grf_problem()
    every = 5
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        def run(tape):
            g = ttsn.TTSN.from_problem(p, stream=stream)
            torch.cuda.synchronize()
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            e[0].record(stream)
            if tape:
                g.tape_begin(every)
            info = g.step(p["steps"])
            e[1].record(stream)
            out = None
            if tape:
                out = g.escape_gradient()
            e[2].record(stream)
            torch.cuda.synchronize()
            return g, info, e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2]), out

        run(True)  # warm-up
        l0 = ttsn.kernel_launches()
        _, info, fwd_ms, bwd_ms, (q, grad) = run(True)
        launches = ttsn.kernel_launches() - l0
        _, _, plain_ms, _, _ = run(False)
    return {"workload": "2D %dx%d cells, %dx%d ordinates, sigma_a = exp(Gaussian random field, corr. 0.1), "
                        "vacuum, %d steps, eps %g, checkpoints every %d steps"
                        % (p["n"][0], p["n"][1], p["n_theta"], p["n_phi"], p["steps"], p["eps"], every),
            "gradients_per_s": 1e3 / (fwd_ms + bwd_ms), "forward_taped_ms": fwd_ms,
            "backward_ms": bwd_ms, "forward_untaped_ms": plain_ms,
            "backward_over_forward": bwd_ms / plain_ms, "gpu_launches": launches,
            "Q": q, "grad_l2": float(grad.norm()), "ranks_last": info["ranks"][1:-1]}


def run_batch(args, torch, ttsn):
    """Batched form: the 64-problem workload (uneven 2D grids, ordinates, ranks,
    tolerances), W warm-up batch steps, state reset, K_b timed batch steps."""
    ps = workloads.batch_problems(64, seed=0)
    batch = ttsn.TTSNBatch(ps)
    init = []
    for i in range(len(ps)):
        pr = batch.problem(i)
        init.append(([c.clone() for c in pr.cores()], pr.energy()[1].clone()))
    batch.step(args.warmup)
    for i, (cores, T0) in enumerate(init):
        pr = batch.problem(i)
        pr.set_cores(cores)
        pr.set_T(T0)
    batch.sync()
    torch.cuda.synchronize()
    kb = args.batch_steps
    t0 = time.perf_counter()
    infos = batch.step(kb)
    batch.sync()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    upd = sum(int(np.prod(p["n"])) * p["n_theta"] * p["n_phi"] for p in ps)
    ranks = [inf["ranks"][1:-1] for inf in infos]
    # the same K_b steps with one host thread (problems one after another)
    seq = ttsn.TTSNBatch(ps, threads=1)
    seq.step(args.warmup)
    for i, (cores, T0) in enumerate(init):
        pr = seq.problem(i)
        pr.set_cores(cores)
        pr.set_T(T0)
    seq.sync()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    seq.step(kb)
    seq.sync()
    torch.cuda.synchronize()
    dt_seq = time.perf_counter() - t1
    del seq
    # the same K_b steps as captured steps: every problem's recorded step
    # replayed as a CUDA graph on its own stream, sizes decided on the device,
    # one synchronisation per problem per call
    cap = ttsn.TTSNBatch(ps)
    cap.set_graph(True)
    cap.step(args.warmup)
    for i, (cores, T0) in enumerate(init):
        pr = cap.problem(i)
        pr.set_cores(cores)
        pr.set_T(T0)
    cap.sync()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    cinfos = cap.step(kb)
    cap.sync()
    torch.cuda.synchronize()
    dt_cap = time.perf_counter() - t2
    same = all(cinfos[i]["ranks"] == infos[i]["ranks"] and
               torch.equal(cap.problem(i).full(), batch.problem(i).full()) for i in range(len(ps)))
    del cap
    return {"workload": "64 independent 2D problems, grids U{64^2,128^2,256^2}, ordinates U{16x32,32x64}, "
                        "sigma_a log-U[1e-2,1e2], Gaussian T pulses, eps U{1e-4,1e-6}, rank caps U[8,96], "
                        "periodic (seed 0); each problem on its own stream, host threads advance them",
            "problem_steps_per_s": len(ps) * kb / dt, "batch_steps_per_s": kb / dt, "steps": kb,
            "warmup": args.warmup, "updates_per_s": upd * kb / dt,
            "timing": "host wall clock around tt_batch_step with device synchronisation on both sides",
            "one_thread_problem_steps_per_s": len(ps) * kb / dt_seq,
            "concurrency_speedup": dt_seq / dt,
            "captured": {"problem_steps_per_s": len(ps) * kb / dt_cap,
                         "speedup_vs_host_threads": dt / dt_cap,
                         "same_bits_as_host_driven": bool(same),
                         "how": "tt_batch_set_graph: every problem's recorded step a branch of one CUDA graph "
                                "(device-decided ranks), one graph launch per batch step"},
            "ranks_last_min_max": [min(min(r) for r in ranks), max(max(r) for r in ranks)]}


# ncu DRAM read + write bytes of one left-Gram launch at the bench's rank cap
# (2,097,152 x 897), scaled by the rows from an ncu capture (dram__bytes_read
# and _write) of the same kernel and split (64 row splits) on a 500,000 x 897
# operand: 23.26 GB.
GRAM_LEFT_CAP_TRAFFIC = (23020594176 + 235760896) * 2097152 / 500000


def roofline_of(prof, fp64_peak, peaks):
    # dominant phase by GPU time
    name = max(prof, key=lambda k: prof[k]["ms"])
    ph = prof[name]
    if ph["ms"] <= 0 or ph["launches"] <= 0:
        return name, None
    avg_ms = ph["ms"] / max(ph["calls"], 1)
    if ph["flops"] > 0:
        achieved = ph["flops"] / (ph["ms"] * 1e-3) / 1e12
        peak = fp64_peak
        traffic = GRAM_LEFT_CAP_TRAFFIC if name == "gram_left" else None
        return name, {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                      "frac": achieved / peak if peak else None, "traffic": traffic,
                      "traffic_note": "ncu DRAM read+write bytes of one capped 2,097,152 x 897 launch (scaled "
                                      "by the rows from a 500,000 x 897 capture)" if traffic else None,
                      "kernel": name, "dtype": "f64", "avg_phase_ms": avg_ms,
                      "launches": ph["launches"], "calls": ph["calls"],
                      "peak_source": "measured FP64 tensor pipe (mma.m8n8k4.f64 chains on all SMs, "
                                     "tt_bench_fp64_mma); MEASURED_PEAKS.json has no FP64 figure"}
    achieved = ph["bytes"] / (ph["ms"] * 1e-3) / 1e9
    peak = peaks.get("hbm_gbs", 6800.0)
    return name, {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                  "frac": achieved / peak, "traffic": None, "kernel": name, "avg_phase_ms": avg_ms,
                  "launches": ph["launches"], "calls": ph["calls"],
                  "peak_source": "MEASURED_PEAKS.json hbm_gbs"}


def cpu_baseline(p, budget_s, gpu_step_ms):
    """The FP64 oracle (paper-form Gram-SVD rounding) as it stands, on the host
    cores: the first m steps of the same trajectory, m bounded by budget_s."""
    from oracle.ttstep import TTSN as OracleTTSN

    I0 = p["c"] * p["a_r"] * p["Tr0"] ** 4 / (4 * np.pi)
    ref = OracleTTSN(p["n"], p["L"], p["n_theta"], p["n_phi"], p["c"], p["a_r"], p["dt"], p["bc"],
                     p["sigma_a"], p["cv"], p["T0"],
                     OracleTTSN.isotropic_cores(I0.reshape(-1), p["n_theta"], p["n_phi"]),
                     eps=p["eps"], max_rank=p.get("max_rank"), rounding="gram")
    t_total, m, last = 0.0, 0, 0.0
    # stop before a step whose predicted cost (ranks grow, so costs grow ~3x per
    # step early on) would overshoot the budget
    while m < len(gpu_step_ms) and (m == 0 or t_total + 3.0 * last <= budget_s):
        t0 = time.perf_counter()
        ref.step()
        last = time.perf_counter() - t0
        t_total += last
        m += 1
    cores = _blas_threads()
    gpu_same = m / (sum(gpu_step_ms[:m]) * 1e-3) if m else None
    return {"value": m / t_total if t_total else None, "unit": "steps/s", "cores": cores,
            "kind": "oracle",
            "sample": "steps 1..%d of the same trajectory (oracle TT stepper, NumPy FP64, paper-form "
                      "Gram-SVD rounding), %.1f s of host time" % (m, t_total),
            "gpu_value_same_steps": gpu_same}


def _blas_threads():
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads") for i in threadpool_info() if i.get("user_api") == "blas"]
        if n:
            return int(max(n))
    except Exception:
        pass
    return os.cpu_count()


def tc_gram_roofline(gl, peaks):
    """Roofline of the precision form's left Gram (tcgen05, 28 BF16 digit
    products per FP64 term): executed BF16 rate against the measured dense
    BF16 tensor throughput (sustained: the Gram runs inside long steps)."""
    if gl["ms"] <= 0 or gl["flops"] <= 0:
        return None
    peak = peaks.get("bf16_tflops_sustained") or peaks.get("bf16_tflops")
    src = "MEASURED_PEAKS.json bf16_tflops_sustained (cuBLAS bf16 GEMM under the power cap)"
    if not peak:
        peak, src = 1700.0, "fallback sustained bf16 figure"
    ex = 28.0 * gl["flops"] / (gl["ms"] * 1e-3) / 1e12
    return {"bound": "tensor", "kernel": "gram_left (tcgram_kernel, tcgen05)",
            "dtype": "bf16 digits (7 x 7 bits, 28 products per term), fp32 exact block sums",
            "achieved": ex, "peak": peak, "unit": "TFLOP/s", "frac": ex / peak,
            "fp64_equivalent_tflops": gl["flops"] / (gl["ms"] * 1e-3) / 1e12, "peak_source": src}


def read_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


# ---------------------------------------------------------------- reference (oracle) arm
def run_reference(args):
    from oracle.ttstep import TTSN as OracleTTSN

    p = workloads.problem(args.workload)
    I0 = p["c"] * p["a_r"] * p["Tr0"] ** 4 / (4 * np.pi)

    def fresh():
        return OracleTTSN(p["n"], p["L"], p["n_theta"], p["n_phi"], p["c"], p["a_r"], p["dt"], p["bc"],
                          p["sigma_a"], p["cv"], p["T0"],
                          OracleTTSN.isotropic_cores(I0.reshape(-1), p["n_theta"], p["n_phi"]),
                          eps=p["eps"], max_rank=p.get("max_rank"), rounding="gram")

    # warm-up: W repetitions of the first step from fresh states (the oracle has
    # nothing to compile; this pages in NumPy/BLAS)
    for _ in range(args.warmup):
        fresh().step()
    # timed: steps 1..m of the same trajectory as our arm, m <= K, stopping once
    # the reference budget is spent (a step at the rank cap costs minutes here)
    ref = fresh()
    t0 = time.perf_counter()
    m = 0
    while m < args.steps and (m == 0 or time.perf_counter() - t0 < args.ref_budget):
        ref.step()
        m += 1
    dt = time.perf_counter() - t0
    v = m / dt
    cores = _blas_threads()
    sample = ("steps 1..%d of the same trajectory (of %d requested; %.0f s budget), NumPy FP64 oracle "
              "with the paper-form Gram-SVD rounding" % (m, args.steps, args.ref_budget))
    line = {"metric": METRIC, "value": v, "unit": "steps/s", "n_gpus": args.gpus, "steps": m,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / m, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": workload_desc(p), "steps_timed": "1..%d" % m},
            "updates_per_s": v * cells_ordinates(p),
            "cpu_baseline": {"value": v, "unit": "steps/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    return line


def aggregate_over_ranks(total_ms, steps, world, device="cuda"):
    """Whole-job timing of the replicas: the slowest rank's time (all-reduce
    MAX over the process group when world > 1) and value = the steps all ranks
    did over that time.  Returns (max total_ms, steps/s)."""
    if world > 1:
        import torch
        import torch.distributed as dist

        t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return total_ms, world * steps / (total_ms * 1e-3)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        if rank != 0:
            return 0
        line = run_reference(args)
        print(json.dumps(line))
        return 0

    if args.only:
        import torch

        import paper_2503_18056_gb300 as ttsn

        if args.only == "adjoint":
            out = run_adjoint(args, torch, ttsn)
        elif args.only == "beams":
            out = run_beams(args, torch, ttsn, ttsn.fp64_mma_peak(), ttsn.bf16_mma_peak())
        elif args.only == "split":
            out = run_split(args, torch, ttsn)
        elif args.only == "fluxes":
            out = run_fluxes(args, torch, ttsn)
        elif args.only == "schedule":
            out = run_schedule(args, torch, ttsn)
        elif args.only == "line_source":
            out = run_line_source(args, torch, ttsn)
        else:
            out = run_batch(args, torch, ttsn)
        print(json.dumps({args.only: out}))
        return 0
    if world > 1:
        import torch
        import torch.distributed as dist

        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    res = run_ours(args, rank, world, local_rank)
    steps = args.steps
    total_ms, value = aggregate_over_ranks(res["total_ms"], steps, world,
                                           "cuda" if world > 1 else "cpu")
    if rank != 0:
        if world > 1:
            import torch.distributed as dist

            dist.destroy_process_group()
        return 0
    p = res["p"]
    peaks = read_peaks()
    dom, roof = roofline_of(res["prof"], res["fp64_peak"], peaks)
    prof_out = {k: {"ms": round(v["ms"], 3), "launches": v["launches"], "calls": v["calls"],
                    "share": round(v["ms"] / max(sum(x["ms"] for x in res["prof"].values()), 1e-9), 4),
                    "tflops": (v["flops"] / (v["ms"] * 1e-3) / 1e12) if v["ms"] > 0 and v["flops"] > 0 else None,
                    "gbs": (v["bytes"] / (v["ms"] * 1e-3) / 1e9) if v["ms"] > 0 and v["bytes"] > 0 else None}
                for k, v in res["prof"].items()}
    line = {
        "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": steps,
        "warmup": args.warmup, "ms_per_step": total_ms / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_desc(p), "parallelism": "replicas" if world > 1 else "single",
                   "steps_timed": "steps 1..%d of the trajectory from t=0 (state reset after warm-up)" % steps,
                   "ranks_first": res["ranks"][0], "ranks_last": res["ranks"][-1],
                   "l2": "inputs larger than L2 (grown spatial core >= 134 MB from step 1)"},
        "updates_per_s": value * cells_ordinates(p),
        "step_ms": [round(x, 3) for x in res["step_ms"]],
        "e2e": res["e2e"], "gpu_launches": res["launches"], "clocks": res["clocks"],
        "roofline": roof, "phases": prof_out,
    }
    mx = res["mixed"]
    if mx is not None:
        mv = world * steps / (mx["total_ms"] * 1e-3)
        mroof = tc_gram_roofline(mx["prof"]["gram_left"], peaks)
        line["mixed"] = {
            "value": mv, "unit": "steps/s", "speedup_vs_fp64": mv / value,
            "updates_per_s": mv * cells_ordinates(p),
            "ranks": "replayed from the FP64 run (forced), steps 1..%d" % steps,
            "err_vs_fp64": {"E_max_rel": mx["err_E"], "T_max_rel": mx["err_T"]},
            "dtype": "bf16 exact-split digits + fp32/double-float accumulation; fp64 eigensolves, decisions, T",
            "step_ms": [round(x, 3) for x in mx["step_ms"]],
            "phases": {k: {"ms": round(v["ms"], 3), "launches": v["launches"]} for k, v in mx["prof"].items()},
            "clocks": mx.get("clocks"), "roofline": mroof}
    rz = res.get("randomized")
    if rz is not None:
        rv = world * steps / (rz["total_ms"] * 1e-3)
        line["randomized"] = {
            "value": rv, "unit": "steps/s", "speedup_vs_fp64_gram": rv / value,
            "ranks": "the FP64 Gram-SVD run's ranks + %d (oversampled sketch, forced), steps 1..%d" % (OVERSAMPLE, steps),
            "sketch": "Gaussian TT at the rank cap + %d (torch.randn, seed 1234), leading blocks at each step's ranks"
                      % OVERSAMPLE,
            "err_vs_fp64_gram": {"E_max_rel": rz["err_E"], "T_max_rel": rz["err_T"]},
            "phases": {k: {"ms": round(v["ms"], 3), "launches": v["launches"]} for k, v in rz["prof"].items()}}
    ts = res.get("ttsvd")
    if ts is not None:
        lg, lt = ts["legs"]["gram"], ts["legs"]["ttsvd"]
        line["ttsvd"] = {
            "workload": "one step (step %d of the trajectory) from the capped state at the end of the FP64 run, "
                        "TT-SVD at the Gram-SVD step's ranks" % ts["step"],
            "gram_step_ms": round(lg["ms"], 3), "ttsvd_step_ms": round(lt["ms"], 3),
            "gram_rounding_ms": round(lg["rounding_ms"], 3), "ttsvd_rounding_ms": round(lt["rounding_ms"], 3),
            "rounding_ratio": lt["rounding_ms"] / max(lg["rounding_ms"], 1e-9), "ranks": lt["ranks"],
            "E_max_rel_diff": ts["err_E"], "phases": {"gram": lg["phases"], "ttsvd": lt["phases"]},
            "how": "QR by three eigen-form Cholesky-QR passes (first shifted), SVD of Rf by the Jacobi "
                   "eigensolver on its Jordan-Wielandt matrix; FP64"}
    if res.get("autotune") is not None:
        line["autotune"] = res["autotune"]
    if res.get("batched") is not None:
        line["batched"] = res["batched"]
    if res.get("adjoint") is not None:
        line["adjoint"] = res["adjoint"]
    if res.get("beams") is not None:
        line["beams"] = res["beams"]
    if res.get("split") is not None:
        line["split"] = res["split"]
    if res.get("fluxes") is not None:
        line["fluxes"] = res["fluxes"]
    if res.get("schedule") is not None:
        line["schedule"] = res["schedule"]
    if res.get("line_source") is not None:
        line["line_source"] = res["line_source"]
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(p, args.cpu_budget, res["step_ms"])
    s = json.dumps(line)
    print(s)
    if args.json_out:
        with open(args.json_out, "w") as f:
            f.write(s + "\n")
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
