#!/usr/bin/env python
"""Throughput of the implicit JFNK step on one GB300: Mpt*steps/s at Newton tolerance 1e-8.

Workload: the 2-D dry thermal in stable stratification (N = 0.01 1/s), 1024 x 512
grid on 20 km x 10 km, cos^2 warm bubble 2 K + seeded 0.01 K white noise,
Smagorinsky Cs = 0.18, trapezoidal step dt = 1 s solved by inexact Newton with
GMRES(30) and the field-block preconditioner, float32 stencils / Krylov basis
with float64 Newton residual, Hessenberg / Givens and update.  One "step" is one
implicit time step (every Newton correction and Krylov iteration it needs).

Prints one JSON line (rank 0).  ``--impl reference`` times the float64 CPU
oracle on bounded samples of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "thermal_stable_1024x512"
METRICS = {
    "thermal_stable_1024x512": "Mpt*steps/s at Newton tol 1e-8 (2D stable dry thermal 1024x512, mixed FP32/FP64 JFNK)",
}


def metric_name(workload: str, fp64: bool = False) -> str:
    """The metric label: the workload and the precision the step runs in."""
    if not fp64 and workload in METRICS:
        return METRICS[workload]
    label = "2D stable dry thermal 1024x512" if workload == WORKLOAD else workload
    return "Mpt*steps/s at Newton tol 1e-8 (%s, %s JFNK)" % (label, "FP64" if fp64 else "mixed FP32/FP64")
# Krylov iterations of the first implicit step of this workload, measured with the
# float64 oracle (3 Newton corrections: 156 + 174 + 230 GMRES(30) iterations);
# used to scale the oracle's bounded samples to whole steps.
ORACLE_ITERS_PER_STEP = 560
ORACLE_NEWTON_PER_STEP = 3


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default=WORKLOAD)
    p.add_argument("--fp64-steps", type=int, default=3, help="steps of the plain float64 path (0: skip)")
    p.add_argument("--e2e-steps", type=int, default=3, help="host-buffer steps through jfnk_step_host")
    p.add_argument("--cpu-seconds", type=float, default=20.0, help="budget of the oracle sample (0: skip)")
    p.add_argument("--no-kernel-timing", action="store_true")
    p.add_argument("--kt-every", type=int, default=5,
                   help="inside the timed region, time the dominant family at Krylov steps j = K/2 mod K")
    p.add_argument("--cycle-graph", type=int, default=-1,
                   help="Krylov steps per captured graph segment (0: stream launches; -1: the library's default)")
    p.add_argument("--precision", default="mixed", choices=["mixed", "fp64"],
                   help="precision of the main timed run (fp64: the plain float64 path, for profiling it)")
    p.add_argument("--precision-check", type=int, default=1,
                   help="1: report the per-field error of the mixed step against the float64 GPU step from "
                        "the same state (256x128 with the same physics, and the workload itself); 0 skips it")
    p.add_argument("--precond", default="block", choices=["block", "schur", "nonlinear"],
                   help="preconditioner of the main timed run (block: the paper's field-block one on the "
                        "right; nonlinear: the same field block as the nonlinear preconditioning of "
                        "Section 2.5.2, i.e. Newton on M^-1 R)")
    p.add_argument("--nonlinear-steps", type=int, default=10,
                   help="steps of the nonlinear-preconditioning leg on the same workload (0 skips it)")
    p.add_argument("--schur-sweeps", type=int, default=32,
                   help="Helmholtz sweeps of the acoustic Schur-complement leg (0 skips it)")
    p.add_argument("--unet-forward", type=int, default=0,
                   help="only time this many applies of the learned-preconditioner network (profiling)")
    p.add_argument("--learned", default="thermal_stable_256x128:40:3,thermal_stable_1024x512:5:2",
                   help="learned-preconditioner legs workload:epochs:steps,... ('' skips)")
    p.add_argument("--learned3d", default="thermal3d_256x256x128:4:2:48",
                   help="3-D learned-preconditioner leg workload:epochs:steps:pairs, with the Schur-complement "
                        "and plain float64 arms ('' skips)")
    return p.parse_args()


# ---------------------------------------------------------------- clocks
class Clocks:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.proc = None
        self.lines = []
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]), "source": "measured"}
    except (OSError, KeyError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "source": "fallback"}


def unet_flops_per_point(dim: int = 2) -> float:
    """Algorithmic FLOPs of one network apply per full-resolution grid point: 2 k^2
    cin cout per layer and output pixel (L0a counts its nf real input channels,
    L0d its nf used outputs); level-1 layers are on 1/4 of the points (1/8 in 3-D),
    level-2 layers on 1/16 (1/64)."""
    nf, r1, r2 = (4, 1 / 4, 1 / 16) if dim == 2 else (5, 1 / 8, 1 / 64)
    return (2 * 9 * nf * 16 + 2 * 9 * 16 * 16                                  # L0a, L0b
            + (2 * 9 * 16 * 32 + 2 * 9 * 32 * 32) * r1                         # L1a, L1b
            + (2 * 9 * 32 * 64 + 2 * 9 * 64 * 64) * r2                         # L2a, L2b
            + 2 * 9 * 96 * 32 * r1 + 2 * 9 * 48 * 16 + 2 * 16 * nf)            # L1c, L0c, L0d


UNET_FLOPS_PER_POINT = unet_flops_per_point(2)


def unet_apply_timing(jfnk, torch, s, npt: int, reps: int, stream, dim: int = 2) -> dict:
    """CUDA-event time of the network apply alone (jfnk_unet_forward) and its tensor roofline,
    for the tcgen05 convolutions (the default engine) and, beside them, the mma.sync ones."""
    nf = 4 if dim == 2 else 5
    x = torch.randn(nf * npt, device="cuda", dtype=torch.float32, generator=torch.Generator("cuda").manual_seed(5))
    y = torch.empty_like(x)
    peaks = measured_peaks()
    flops = unet_flops_per_point(dim) * npt
    out = {}
    for engine, tag in ((jfnk.UNET_MMA_SYNC, "mma_sync"), (jfnk.UNET_TCGEN05, "tcgen05")):
        s.unet_set_engine(engine)
        for _ in range(3):
            s.unet_forward(x, y)
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(reps):
            s.unet_forward(x, y)
        a1.record(stream)
        a1.synchronize()
        s.unet_status()
        ms = a0.elapsed_time(a1) / reps
        out[tag] = {"ms_per_apply": ms, "achieved": flops / (ms / 1e3) / 1e12}
    achieved = out["tcgen05"]["achieved"]
    return {"ms_per_apply": out["tcgen05"]["ms_per_apply"], "flops_per_apply": flops, "bound": "tensor",
            "achieved": achieved, "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
            "frac": achieved / peaks["bf16_tflops"],
            "peak_source": peaks["source"] + " (MEASURED_PEAKS.json bf16_tflops, burst)",
            "kernel": "conv_tc (tcgen05.mma kind::f16, bf16 in TMEM-accumulated float32, 8 launches per apply: L0d composed into L0c)",
            "mma_sync": out["mma_sync"]}


def ncu_fp64_pipe():
    """(pipe fraction, ncu launch time in us) of the float64 Jacobian product from
    profiles/ncu_traffic.txt, when the captured source still has that hash; else None."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    src = os.path.join(ROOT, "paper_2007_10411_gb300", "csrc", "stencil.cu")
    try:
        sha = hashlib.sha1(open(src, "rb").read()).hexdigest()
        for line in open(path):
            t = line.split()
            if len(t) >= 5 and t[0] == "fp64_pipe_jv" and t[4] == sha:
                return float(t[1]), float(t[2])
    except (OSError, ValueError):
        pass
    return None


def ncu_traffic() -> dict:
    """Per-algorithmic-byte DRAM traffic of the kernels captured with ncu (profiles/ncu_traffic.txt).

    Lines: ``<family> <traffic/algorithmic ratio> <source sha1 of the .cu file>``; a ratio is used
    only when the kernel source still has that hash.
    """
    import hashlib
    out = {}
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    srcs = {"krylov": os.path.join(ROOT, "paper_2007_10411_gb300", "csrc", "krylov.cu"),
            "stencil": os.path.join(ROOT, "paper_2007_10411_gb300", "csrc", "stencil.cu")}
    hashes = {}
    for k, p in srcs.items():
        try:
            hashes[k] = hashlib.sha1(open(p, "rb").read()).hexdigest()
        except OSError:
            hashes[k] = None
    try:
        for line in open(path):
            t = line.split()
            if len(t) >= 4 and not t[0].startswith("#") and t[0] != "fp64_pipe_jv":
                fam, ratio, src, sha = t[0], float(t[1]), t[2], t[3]
                if hashes.get(src) == sha:
                    out[fam] = ratio
    except OSError:
        pass
    return out


# ---------------------------------------------------------------- multi-rank
def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Largest value over all ranks of the default process group (the slowest rank's time)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(points: int, steps: int, world: int, slowest_ms: float) -> float:
    """Whole-job Mpt*steps/s: every rank steps its own replica; time = slowest rank."""
    return points * steps * world / (slowest_ms / 1e3) / 1e6


# ---------------------------------------------------------------- oracle sample
def oracle_sample(case: dict, seconds: float, iters_per_step: float, newton_per_step: float):
    """Time the float64 oracle on a bounded sample of one step of the workload.

    The sample is the Newton set-up (F(u^n), R, F(u)) plus as many GMRES(m)
    iterations (preconditioner, finite-difference Jv, CGS2) of the first Newton
    solve as fit in ``seconds``; the step time is extrapolated as
    setup * newton + per_iteration * iterations_per_step.
    """
    import numpy as np

    from oracle.krylov import gmres
    from oracle.operators import Model
    from paper_2007_10411_gb300 import synth

    m = Model(case)
    if case.get("init", {}).get("kind") == "rest" and "H0" in case["init"]:
        m.set_heat_flux(synth.heat_flux(case))          # heat island: the surface flux drives the step
    U = synth.initial_state(case)
    t0 = time.perf_counter()
    f = m.rhs_f(U)
    R = m.residual(U, f)
    FU = m.F(U)
    t_setup = time.perf_counter() - t0
    o = case["opts"]
    pc = (lambda v: m.precond(U, v, o["pc_sweeps"])) if o["precond"] == 1 else None
    probe = 2
    t1 = time.perf_counter()
    gmres(lambda v: m.jv_scaled(U, FU, v), -m.scale(R), probe, 1e-30, 0, precond=pc, flexible=True)
    t_probe = (time.perf_counter() - t1) / probe
    k = int(max(1, min(o["krylov_m"], (seconds - t_setup) / max(t_probe, 1e-9))))
    t2 = time.perf_counter()
    rec = {}
    gmres(lambda v: m.jv_scaled(U, FU, v), -m.scale(R), k, 1e-30, 0, precond=pc, flexible=True, record=rec)
    t_it = (time.perf_counter() - t2) / rec["iters"]
    step_s = t_setup * newton_per_step + t_it * iters_per_step
    npt = int(np.prod(synth.shape(case)[1:]))
    return {
        "value": npt / step_s / 1e6,
        "step_seconds": step_s,
        "sample": "oracle (numpy float64) on the %dx%d workload: Newton set-up + %d GMRES iterations "
                  "of step 1 (%.1f s), extrapolated to %.0f iterations and %.0f Newton corrections per step"
                  % (case["grid"]["nx"], case["grid"]["nz"], rec["iters"], t_setup + t_it * rec["iters"],
                     iters_per_step, newton_per_step),
        "seconds_used": time.perf_counter() - t0,
    }


def cpu_threads() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ---------------------------------------------------------------- reference arm
def run_reference(args, rank: int):
    if rank != 0:
        return
    from paper_2007_10411_gb300 import synth
    case = synth.case(args.workload)
    per = []
    sample = None
    budget = 6.0
    sampled = []
    for i in range(args.warmup + args.steps):
        r = oracle_sample(case, budget, ORACLE_ITERS_PER_STEP, ORACLE_NEWTON_PER_STEP)
        if i >= args.warmup:
            per.append(r["step_seconds"])
            sampled.append(r["seconds_used"])
            sample = r["sample"]
    step_s = statistics.mean(per)
    sample_s = statistics.mean(sampled)
    npt = int(__import__("math").prod(synth.shape(case)[1:]))
    value = npt / step_s / 1e6
    line = {
        "impl": "reference",
        "metric": metric_name(args.workload, args.precision == "fp64" or case["opts"]["precision"] == synth.PREC_FP64),
        "value": value, "unit": "Mpt*steps/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": step_s * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "grid": list(synth.shape(case)[:0:-1]),
                   "extrapolated": True,
                   "note": "float64 numpy oracle; a whole step of this workload takes the oracle about "
                           "440 s on 8 cores, so each 'step' times a bounded sample (Newton set-up + a few "
                           "GMRES iterations) and ms_per_step is that sample extrapolated to %d GMRES "
                           "iterations and %d Newton corrections; the time actually spent per sampled step "
                           "is sample_seconds_per_step" % (ORACLE_ITERS_PER_STEP, ORACLE_NEWTON_PER_STEP),
                   "sample_seconds_per_step": sample_s},
        "cpu_baseline": {"value": value, "unit": "Mpt*steps/s", "cores": cpu_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "Mpt*steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- our arm
def run_batch(args, rank: int, world: int, local_rank: int):
    """The batched heat-island workload: every instance stepped concurrently (jfnk_step_batch)."""
    import numpy as np
    import torch

    import __graft_entry__
    from paper_2007_10411_gb300 import jfnk, synth

    __graft_entry__.build()
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist_
        dist = dist_
    three_d = args.workload.startswith("uhi3d_batch")
    if three_d:
        n_inst = int(args.workload[len("uhi3d_batch"):] or 4)
        cases = synth.uhi3d_batch(n=n_inst)
    else:
        n_inst = int(args.workload[len("uhi_batch"):] or 16)
        cases = synth.uhi_batch(n=n_inst)
    if args.precond == "schur":
        cases = [synth.with_options(c, precond=jfnk.PC_SCHUR, pc_sweeps=args.schur_sweeps) for c in cases]
    elif args.precond == "nonlinear":
        cases = [synth.with_options(c, precond=jfnk.PC_NONLINEAR) for c in cases]
    stream = torch.cuda.current_stream()
    batch = jfnk.Batch(cases, stream=stream)
    if args.cycle_graph >= 0:
        batch.set_cycle_graph(args.cycle_graph)
    for i, c in enumerate(cases):
        batch.set_surface_flux(i, torch.from_numpy(synth.heat_flux(c)).cuda())
    U0 = [synth.initial_state(c) for c in cases]
    states = [torch.from_numpy(u).cuda() for u in U0]
    points = sum(int(np.prod(synth.shape(c)[1:])) for c in cases)
    # heat-content budget: the surface flux adds mean(H) * area * dt / (rho0 cp) to
    # sum(theta) dV every step; its drift is what the step adds beyond that
    heat_in = []
    for c in cases:
        H = synth.heat_flux(c)
        area = c["grid"]["lx"] * (c["grid"]["ly"] if c["grid"]["dim"] == 3 else 1.0)
        heat_in.append(float(np.mean(H)) * area * c["opts"]["dt"] / (c["strat"]["rho0"] * c["strat"]["cp"]))
    b_start = [batch.budgets(i, states[i]) for i in range(n_inst)]
    for _ in range(args.warmup):
        batch.step(states)
    torch.cuda.synchronize()
    # kernel breakdown: one more warm batch step with CUDA events around every launch of
    # every family (the instances run concurrently, so a launch shares the GPU with others)
    kbreak = None
    if not args.no_kernel_timing:
        batch.kernel_timing()
        batch.step([s.clone() for s in states])
        torch.cuda.synchronize()
        kbreak = batch.kernel_timing_read()
        batch.kernel_timing(())
    if dist is not None:
        dist.barrier()
    clocks = Clocks(local_rank)
    t0 = time.perf_counter()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    stats = [batch.step(states) for _ in range(args.steps)]
    e1.record(stream)
    e1.synchronize()
    wall_ms = (time.perf_counter() - t0) * 1e3
    clk = clocks.stop()
    ms = max_over_ranks(max(e0.elapsed_time(e1), 0.0), dist, "cuda")
    value = job_throughput(points, args.steps, world, ms)
    b_end = [batch.budgets(i, states[i]) for i in range(n_inst)]
    nsteps = args.warmup + args.steps
    budget = []
    for i in range(n_inst):
        gained = b_end[i]["sum_theta"] - b_start[i]["sum_theta"]
        budget.append({"heat_gained": gained, "heat_input": heat_in[i] * nsteps,
                       "heat_drift_rel": (gained - heat_in[i] * nsteps) / (heat_in[i] * nsteps) if heat_in[i] else None,
                       "sum_div": b_end[i]["sum_div"], "E_k": b_end[i]["E_k"], "E_p": b_end[i]["E_p"]})
    e2e = None
    if args.e2e_steps > 0:
        hosts = [d.cpu().pin_memory() for d in states]   # continue the timed region's trajectory
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            for h, d in zip(hosts, states):
                d.copy_(h, non_blocking=True)
            batch.step(states)
            for h, d in zip(hosts, states):
                h.copy_(d, non_blocking=True)
            torch.cuda.synchronize()
        el = max_over_ranks((time.perf_counter() - t0) * 1e3, dist, "cuda")
        nbytes = sum(8 * int(np.prod(synth.shape(c))) for c in cases)
        e2e = {"value": job_throughput(points, args.e2e_steps, world, el), "unit": "Mpt*steps/s",
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes}
    precision = None
    if args.precision_check and rank == 0:
        # instance 0: one mixed step against the float64 GPU step from the same state
        batch.close()
        del states
        torch.cuda.empty_cache()
        c0 = cases[0]
        H0 = torch.from_numpy(synth.heat_flux(c0)).cuda()
        outs = []
        for prec in (synth.PREC_MIXED, synth.PREC_FP64):
            s_ = jfnk.Solver(synth.with_options(c0, precision=prec), stream=stream)
            s_.set_surface_flux(H0)
            u_ = torch.from_numpy(U0[0].copy()).cuda()
            st_ = s_.step(u_)
            torch.cuda.synchronize()
            outs.append((u_.cpu().numpy(), st_))
            s_.close()
            del u_
            torch.cuda.empty_cache()
        (gm, stm), (gd, std) = outs
        names = ["u", "w", "theta", "p"] if c0["grid"]["dim"] == 2 else ["u", "v", "w", "theta", "p"]
        precision = {"fields": names, "instance": 0, "tolerance": 1e-4,
                     "vs_fp64_gpu": {"state": _rel_per_field(gm, gd), "increment": _rel_per_field(gm - U0[0], gd - U0[0]),
                                     "converged": stm["converged"] and std["converged"]}}
    if rank != 0:
        return
    per_inst = [[s[i] for s in stats] for i in range(n_inst)]
    roof, kernels = None, None
    if kbreak:
        peaks = measured_peaks()
        kernels = {k: {"launches": a["launches"], "ms_total": a["ms"],
                       "achieved_gbs": a["bytes"] / (a["ms"] / 1e3) / 1e9}
                   for k, a in kbreak.items() if a["launches"] and a["ms"] > 0}
        dom = max(kernels, key=lambda k: kernels[k]["ms_total"])
        roof = {"kernel": dom, "bound": "hbm", "achieved": kernels[dom]["achieved_gbs"], "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": kernels[dom]["achieved_gbs"] / peaks["hbm_gbs"], "traffic": None,
                "algorithmic_bytes_per_launch": kbreak[dom]["bytes"] / kbreak[dom]["launches"],
                "peak_source": peaks["source"] + " (MEASURED_PEAKS.json hbm_gbs)",
                "timing": "CUDA events around every launch of this family over one batch step, instances "
                          "running concurrently (a launch shares the GPU with the other instances' kernels)"}
    cpu = None
    if args.cpu_seconds > 0:
        c0 = cases[0]
        it0 = statistics.mean(s["gmres_iters"] for s in per_inst[0])
        nw0 = statistics.mean(s["newton_iters"] for s in per_inst[0])
        where = "instance 0 of the batch"
        if three_d:
            # a 384 x 384 x 128 residual alone takes the oracle minutes: sample the same
            # physics on a 96 x 96 x 32 grid
            c0 = synth.with_options(c0, nx=96, ny=96, nz=32)
            where = "instance 0's physics on a 96x96x32 grid"
        r = oracle_sample(c0, args.cpu_seconds, max(it0, 1.0), max(nw0, 1.0))
        cpu = {"value": r["value"], "unit": "Mpt*steps/s", "cores": cpu_threads(), "kind": "oracle",
               "sample": where + ": " + r["sample"]}
    line = {
        "metric": metric_name(args.workload), "value": value, "unit": "Mpt*steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "wall_ms_per_step": wall_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "instances": n_inst, "points": points,
                   "grids": [list(synth.shape(c)[:0:-1]) for c in cases],
                   "H0": [round(c["init"]["H0"], 2) for c in cases],
                   "precision": "mixed", "krylov_m": cases[0]["opts"]["krylov_m"],
                   "precond": pc_label(args.precond, cases[0]),
                   "execution": "one handle + stream per instance, host thread per instance",
                   "parallelism": "replicas" if world > 1 else "single"},
        "precision_error": precision,
        "budgets": {"steps": nsteps, "per_instance": budget,
                    "note": "sum(theta) dV gained over all steps against the surface heat input "
                            "mean(H) area dt / (rho0 cp) per step; sum_div = global mass flux"},
        "newton_per_step": [statistics.mean(s["newton_iters"] for s in p) for p in per_inst],
        "gmres_iters_per_step": [statistics.mean(s["gmres_iters"] for s in p) for p in per_inst],
        "converged": all(s["converged"] for st in stats for s in st),
        "clocks": clk, "e2e": e2e, "roofline": roof, "kernels": kernels, "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)


def grid_points(c: dict) -> int:
    g = c["grid"]
    return g["nx"] * g["nz"] * (g["ny"] if g["dim"] == 3 else 1)


def learned_leg(jfnk, synth, torch, stream, name: str, epochs: int, steps: int, barrier, slowest,
                capacity: int = 900, others: bool = False) -> dict:
    """Learned right preconditioner against the field-block one on one workload.

    Training pairs: every Arnoldi step of two plain steps from the initial
    state (at most `capacity`); Adam, lr 3e-4.  Then `steps` timed steps from
    the same state with each preconditioner (CUDA events on the solver's
    stream).  With `others`, the same steps with the acoustic Schur-complement
    preconditioner (16 sweeps) and with the plain float64 path (field block).
    """
    c = synth.with_options(synth.case(name), precision=synth.PREC_MIXED, precond=jfnk.PC_UNET)
    npt = grid_points(c)
    dim = c["grid"]["dim"]
    s = jfnk.Solver(c, stream=stream)
    s.set_precond(jfnk.PC_BLOCK)
    s.unet_init(7)
    s.unet_capture(capacity, jfnk.PAIRS_ARNOLDI)
    u = torch.from_numpy(synth.initial_state(c).reshape(-1).copy()).cuda()
    for _ in range(2):
        s.step(u)
    pairs = s.unet_pair_count()
    barrier()
    t0 = time.perf_counter()
    hist = s.unet_train(epochs, 3e-4)
    train_s = time.perf_counter() - t0
    s.unet_capture(0, 0)
    out = {"workload": name, "pairs": pairs, "epochs": epochs, "train_s": train_s,
           "loss_first_epoch": hist[0], "loss_last_epoch": hist[-1], "steps": steps}
    for mode, tag in ((jfnk.PC_BLOCK, "block"), (jfnk.PC_UNET, "learned")):
        s.set_precond(mode)
        v = u.clone()
        barrier()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        st = [s.step(v) for _ in range(steps)]
        a1.record(stream)
        a1.synchronize()
        ms = slowest(a0.elapsed_time(a1))
        out[tag] = {"value": npt * steps / (ms / 1e3) / 1e6, "ms_per_step": ms / steps,
                    "gmres_iters_per_step": statistics.mean(x["gmres_iters"] for x in st),
                    "newton_per_step": statistics.mean(x["newton_iters"] for x in st),
                    "converged": all(x["converged"] for x in st),
                    "pc_switches": sum(x.get("pc_switches", 0) for x in st),
                    "pc_fallback": sum(int(x.get("pc_fallback", False)) for x in st)}
    out["learned_over_block"] = out["learned"]["value"] / out["block"]["value"]
    out["network_apply"] = unet_apply_timing(jfnk, torch, s, npt, 20 if dim == 2 else 5, stream, dim)
    s.close()
    if others:
        arms = (("schur", synth.with_options(c, precond=jfnk.PC_SCHUR, pc_sweeps=16)),
                ("fp64", synth.with_options(c, precision=synth.PREC_FP64, precond=jfnk.PC_BLOCK)))
        for tag, co in arms:
            so = jfnk.Solver(co, stream=stream)
            v = u.clone()
            so.step(v.clone())                        # warm (first-call set-up)
            barrier()
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            st = [so.step(v) for _ in range(steps)]
            a1.record(stream)
            a1.synchronize()
            ms = slowest(a0.elapsed_time(a1))
            so.close()
            out[tag] = {"value": npt * steps / (ms / 1e3) / 1e6, "ms_per_step": ms / steps,
                        "gmres_iters_per_step": statistics.mean(x["gmres_iters"] for x in st),
                        "newton_per_step": statistics.mean(x["newton_iters"] for x in st),
                        "converged": all(x["converged"] for x in st)}
        out["learned_over_fp64"] = out["learned"]["value"] / out["fp64"]["value"]
        out["learned_over_schur"] = out["learned"]["value"] / out["schur"]["value"]
    return out


def run_unet_forward(args):
    """Time `--unet-forward` applies of a network with seeded random weights (profiling entry)."""
    import numpy as np
    import torch

    import __graft_entry__
    from paper_2007_10411_gb300 import jfnk, synth

    __graft_entry__.build()
    torch.cuda.set_device(0)
    c = synth.with_options(synth.case(args.workload), precision=synth.PREC_MIXED, precond=jfnk.PC_UNET)
    npt = grid_points(c)
    stream = torch.cuda.current_stream()
    s = jfnk.Solver(c, stream=stream)
    s.unet_init(1)
    rng = np.random.Generator(np.random.PCG64(3))
    s.unet_set_weights((0.05 * rng.standard_normal(s.unet_num_weights())).astype(np.float32))
    r = unet_apply_timing(jfnk, torch, s, npt, args.unet_forward, stream, c["grid"]["dim"])
    r.update({"workload": args.workload, "applies": args.unet_forward})
    print(json.dumps(r), flush=True)
    s.close()


def pc_label(precond: str, case: dict) -> str:
    sw = case["opts"]["pc_sweeps"]
    if precond == "schur":
        return "acoustic Schur complement (%d Helmholtz sweeps)" % sw
    if precond == "nonlinear":
        return "field-block Chebyshev (%d sweeps) as nonlinear preconditioner (Newton on M^-1 R)" % sw
    return "field-block Chebyshev (%d sweeps)" % sw


def _rel_per_field(got, ref):
    import numpy as np
    return [float(np.linalg.norm(got[f] - ref[f]) / max(np.linalg.norm(ref[f]), 1e-300)) for f in range(ref.shape[0])]


def precision_leg(jfnk, synth, torch, stream, case, U0) -> dict:
    """Per-field relative L2 error of one mixed-precision step (u, w, theta, p), on the state
    and on the step's increment, against the float64 GPU step from the same state: (a) at
    256x128 with the workload's physics, (b) on the workload itself.  (The comparison with
    the float64 oracle's step is the GPU test suite's: tests/test_gpu_precision.py.)"""

    def gpu_step(c, U):
        s = jfnk.Solver(c, stream=stream)
        u = torch.from_numpy(U.copy()).cuda()
        st = s.step(u)
        torch.cuda.synchronize()
        out = u.cpu().numpy()
        s.close()
        return out, st

    out = {"fields": ["u", "w", "theta", "p"][:U0.shape[0]], "tolerance": 1e-4}
    small = synth.case("thermal_stable_256x128")
    for c, U in ((small, synth.initial_state(small)), (case, U0)):
        got, st = gpu_step(c, U)
        ref, st64 = gpu_step(synth.with_options(c, precision=synth.PREC_FP64), U)
        out["vs_fp64_gpu_" + "x".join(str(v) for v in synth.shape(c)[:0:-1])] = {
            "state": _rel_per_field(got, ref), "increment": _rel_per_field(got - U, ref - U),
            "converged": st["converged"] and st64["converged"]}
    return out


def nonlinear_leg(jfnk, synth, torch, stream, case, U0, steps: int, barrier, slowest, world: int) -> dict:
    """The same workload with the nonlinear preconditioning of Section 2.5.2 (JFNK_PC_NONLINEAR:
    Newton on M^-1 W R, GMRES on M^-1 J from the left, the same field-block M as the headline)."""
    c = synth.with_options(case, precond=jfnk.PC_NONLINEAR)
    npt = c["grid"]["nx"] * c["grid"]["nz"]
    s = jfnk.Solver(c, stream=stream)
    u = torch.from_numpy(U0.reshape(-1).copy()).cuda()
    for _ in range(3):
        s.step(u)
    s.autotune(u)
    barrier()
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    st = [s.step(u) for _ in range(steps)]
    a1.record(stream)
    a1.synchronize()
    ms = slowest(a0.elapsed_time(a1))
    s.close()
    return {"precond": "field block (%d Chebyshev sweeps) as nonlinear preconditioner: Newton on M^-1 W R"
                       % c["opts"]["pc_sweeps"],
            "value": npt * steps * world / (ms / 1e3) / 1e6, "unit": "Mpt*steps/s", "steps": steps,
            "ms_per_step": ms / steps,
            "gmres_iters_per_step": statistics.mean(x["gmres_iters"] for x in st),
            "newton_per_step": statistics.mean(x["newton_iters"] for x in st),
            "converged": all(x["converged"] for x in st)}


def schur_leg(jfnk, synth, torch, stream, case, U0, steps: int, sweeps: int, barrier, slowest, world: int) -> dict:
    """The same workload with the acoustic Schur-complement preconditioner (JFNK_PC_SCHUR)."""
    c = synth.with_options(case, precond=jfnk.PC_SCHUR, pc_sweeps=sweeps)
    npt = c["grid"]["nx"] * c["grid"]["nz"]
    s = jfnk.Solver(c, stream=stream)
    u = torch.from_numpy(U0.reshape(-1).copy()).cuda()
    for _ in range(3):
        s.step(u)
    tiles = s.autotune(u)
    s.kernel_timing()
    b0 = torch.cuda.Event(enable_timing=True)
    b1 = torch.cuda.Event(enable_timing=True)
    b0.record(stream)
    for _ in range(2):
        s.step(u)
    b1.record(stream)
    b1.synchronize()
    kt, kms = s.kernel_timing_read(), b0.elapsed_time(b1)
    s.kernel_timing(())
    barrier()
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    st = [s.step(u) for _ in range(steps)]
    a1.record(stream)
    a1.synchronize()
    ms = slowest(a0.elapsed_time(a1))
    peaks = measured_peaks()
    kernels = {k: {"launches": a["launches"], "ms_total": a["ms"], "share_of_step": a["ms"] / kms,
                   "achieved_gbs": a["bytes"] / (a["ms"] / 1e3) / 1e9,
                   "frac_of_hbm": a["bytes"] / (a["ms"] / 1e3) / 1e9 / peaks["hbm_gbs"]}
               for k, a in kt.items() if a["launches"] and a["ms"] > 0}
    s.close()
    dom = max(kernels, key=lambda k: kernels[k]["ms_total"])
    ratios = ncu_traffic()
    tkey = dom + "_schur" if dom == "precond" else dom
    per_launch = kt[dom]["bytes"] / kt[dom]["launches"]
    roof = {"kernel": dom, "bound": "hbm", "achieved": kernels[dom]["achieved_gbs"], "peak": peaks["hbm_gbs"],
            "unit": "GB/s", "frac": kernels[dom]["frac_of_hbm"], "algorithmic_bytes_per_launch": per_launch,
            "traffic": (ratios[tkey] * per_launch) if tkey in ratios else None,
            "timing": "CUDA events around every launch of this family over 2 steps"}
    return {"precond": "acoustic Schur complement, %d Helmholtz Chebyshev sweeps" % sweeps, "roofline": roof,
            "value": npt * steps * world / (ms / 1e3) / 1e6, "unit": "Mpt*steps/s", "steps": steps,
            "ms_per_step": ms / steps,
            "gmres_iters_per_step": statistics.mean(x["gmres_iters"] for x in st),
            "newton_per_step": statistics.mean(x["newton_iters"] for x in st),
            "converged": all(x["converged"] for x in st), "tiles": list(tiles), "kernels": kernels,
            "kernels_timing": "per-family CUDA events over 2 steps before the timed steps"}


def run_ours(args, rank: int, world: int, local_rank: int):
    import numpy as np
    import torch

    import __graft_entry__
    from paper_2007_10411_gb300 import jfnk, synth

    __graft_entry__.build()
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist_
        dist = dist_

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def slowest(v: float) -> float:
        return max_over_ranks(v, dist, "cuda")

    case = synth.case(args.workload)
    if args.precision == "fp64":
        case = synth.with_options(case, precision=synth.PREC_FP64)
    if args.precond == "schur":
        case = synth.with_options(case, precond=jfnk.PC_SCHUR, pc_sweeps=args.schur_sweeps)
    elif args.precond == "nonlinear":
        case = synth.with_options(case, precond=jfnk.PC_NONLINEAR)
    npt = synth.shape(case)[1:]
    npt = int(__import__("math").prod(npt))
    n = synth.n_fields(case) * npt
    stream = torch.cuda.current_stream()
    solver = jfnk.Solver(case, stream=stream)
    if args.cycle_graph >= 0:
        solver.set_cycle_graph(args.cycle_graph)
    U0 = synth.initial_state(case)
    u = torch.from_numpy(U0).cuda()
    for _ in range(args.warmup):
        solver.step(u)
    tiles = solver.autotune(u)              # set-up, outside the timed region
    # Kernel breakdown: two more warm steps with CUDA events around every timed
    # family; the dominant family is then the only one timed inside the timed
    # region (events on every launch would slow the host side of the step).
    breakdown, dom = None, None
    if not args.no_kernel_timing:
        solver.kernel_timing()
        b0 = torch.cuda.Event(enable_timing=True)
        b1 = torch.cuda.Event(enable_timing=True)
        b0.record(stream)
        for _ in range(2):
            solver.step(u)
        b1.record(stream)
        b1.synchronize()
        breakdown = (solver.kernel_timing_read(), b0.elapsed_time(b1))
        dom = max(breakdown[0], key=lambda k: breakdown[0][k]["ms"])
        solver.kernel_timing((dom,), every=args.kt_every)
        solver.step(u)                      # warm: captures the cycle graphs with this family's events
        solver.kernel_timing((dom,), every=args.kt_every)   # resets the accumulators
    stats = []
    barrier()
    clocks = Clocks(local_rank)
    launches0 = solver.launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        stats.append(solver.step(u))
    e1.record(stream)
    e1.synchronize()
    barrier()
    clk = clocks.stop()
    launches = solver.launch_count() - launches0
    ms = e0.elapsed_time(e1)
    ms = slowest(ms)
    kt = solver.kernel_timing_read() if not args.no_kernel_timing else None
    solver.kernel_timing(())
    value = job_throughput(npt, args.steps, world, ms)

    # end to end through the public API with host buffers (pinned), copies in the timed region;
    # the steps continue the trajectory of the timed region (same kind of work per step)
    e2e = None
    if args.e2e_steps > 0:
        uh = u.cpu().pin_memory()
        solver.step_host(uh)                       # warm
        barrier()
        t0 = time.perf_counter()
        est = [solver.step_host(uh) for _ in range(args.e2e_steps)]
        barrier()
        el = slowest(time.perf_counter() - t0)
        e2e = {"value": npt * args.e2e_steps * world / el / 1e6, "unit": "Mpt*steps/s",
               "h2d_bytes_per_step": n * 8, "d2h_bytes_per_step": n * 8,
               "gmres_iters_per_step": sum(x["gmres_iters"] for x in est) / len(est),
               "note": "jfnk_step_host on pinned host memory, continuing the timed region's trajectory; "
                       "host wall clock, no kernel-timing events"}

    # plain float64 JFNK on the same workload (the mixed-precision comparison)
    fp64 = None
    if args.fp64_steps > 0:
        c64 = synth.with_options(case, precision=synth.PREC_FP64)
        s64 = jfnk.Solver(c64, stream=stream)
        u64 = torch.from_numpy(U0).cuda()
        s64.step(u64)
        barrier()
        s64.kernel_timing(("jv",))
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        st64 = [s64.step(u64) for _ in range(args.fp64_steps)]
        a1.record(stream)
        a1.synchronize()
        ms64 = slowest(a0.elapsed_time(a1))
        kj = s64.kernel_timing_read()["jv"]
        s64.kernel_timing(())
        fp64 = {"value": npt * args.fp64_steps * world / (ms64 / 1e3) / 1e6,
                "ms_per_step": ms64 / args.fp64_steps,
                "gmres_iters_per_step": statistics.mean(s["gmres_iters"] for s in st64),
                "newton_per_step": statistics.mean(s["newton_iters"] for s in st64)}
        pipe = ncu_fp64_pipe()
        if kj["launches"] and pipe is not None:
            live_us = kj["ms"] / kj["launches"] * 1e3
            fp64["fp64_pipe"] = {
                "kernel": "stencil2d<double, MODE_JV> (float64 Jacobian product)", "bound": "fp64 pipe",
                "live_us_per_launch": live_us, "ncu_us_per_launch": pipe[1], "ncu_pipe_frac": pipe[0],
                "frac": pipe[0] * pipe[1] / live_us,
                "how": "FP64-pipe busy fraction from one ncu capture (profiles/ncu_traffic.txt), scaled by the "
                       "ratio of that launch time to the live per-launch time of this leg (CUDA events)"}
        s64.close()

    precision = None
    if args.precision_check and args.precision == "mixed" and case["grid"]["dim"] == 2 and rank == 0:
        precision = precision_leg(jfnk, synth, torch, stream, case, U0)

    nonlinear = None
    if args.nonlinear_steps > 0 and args.precond == "block":
        nonlinear = nonlinear_leg(jfnk, synth, torch, stream, case, U0, args.nonlinear_steps, barrier, slowest,
                                  world)

    schur = None
    if args.schur_sweeps > 1 and case["grid"]["dim"] == 2 and args.precond == "block":
        schur = schur_leg(jfnk, synth, torch, stream, case, U0, max(args.steps, 10), args.schur_sweeps,
                          barrier, slowest, world)

    learned = []
    if args.learned and case["grid"]["dim"] == 2:
        for item in args.learned.split(","):
            name, ep, st = item.split(":")
            learned.append(learned_leg(jfnk, synth, torch, stream, name, int(ep), int(st), barrier, slowest))

    learned3d = None
    if args.learned3d and case["grid"]["dim"] == 2:
        name, ep, st, cap = args.learned3d.split(":")
        learned3d = learned_leg(jfnk, synth, torch, stream, name, int(ep), int(st), barrier, slowest,
                                capacity=int(cap), others=True)

    if rank != 0:
        return
    iters = statistics.mean(s["gmres_iters"] for s in stats)
    newt = statistics.mean(s["newton_iters"] for s in stats)
    roof = None
    kernels = None
    if kt is not None:
        peaks = measured_peaks()
        ratios = ncu_traffic()
        kernels = {}
        bk, bms = breakdown
        for name, a in bk.items():
            if a["launches"] == 0 or a["ms"] <= 0:
                continue
            kernels[name] = {"launches": a["launches"], "ms_total": a["ms"],
                             "share_of_step": a["ms"] / bms,
                             "achieved_gbs": a["bytes"] / (a["ms"] / 1e3) / 1e9}
        a = kt[dom]      # the dominant family, timed inside the timed region
        tkey = dom + "_schur" if (dom == "precond" and args.precond == "schur") else dom
        per_launch_bytes = a["bytes"] / a["launches"]
        d = {"achieved_gbs": a["bytes"] / (a["ms"] / 1e3) / 1e9}
        roof = {"kernel": dom, "bound": "hbm", "achieved": d["achieved_gbs"], "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": d["achieved_gbs"] / peaks["hbm_gbs"],
                "traffic": (ratios[tkey] * per_launch_bytes) if tkey in ratios else None,
                "algorithmic_bytes_per_launch": per_launch_bytes,
                "peak_source": peaks["source"] + " (MEASURED_PEAKS.json hbm_gbs)",
                "timing": ("CUDA events inside the timed region around the %d launches of this family at "
                           "Krylov steps j = %d mod %d (every launch outside the GMRES cycles): sum of "
                           "algorithmic bytes / sum of event time" % (a["launches"], args.kt_every // 2,
                                                                     args.kt_every))}
    cpu = None
    if args.cpu_seconds > 0:
        r = oracle_sample(case, args.cpu_seconds, iters, newt)
        cpu = {"value": r["value"], "unit": "Mpt*steps/s", "cores": cpu_threads(), "kind": "oracle",
               "sample": r["sample"]}
    line = {
        "metric": metric_name(args.workload, case["opts"]["precision"] == synth.PREC_FP64),
        "value": value, "unit": "Mpt*steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if case["opts"]["precision"] == synth.PREC_FP64 else "f32/f64", "data": "synthetic",
        "config": {"workload": args.workload, "grid": list(synth.shape(case)[:0:-1]),
                   "points": npt, "precision": args.precision, "krylov_m": case["opts"]["krylov_m"],
                   "precond": pc_label(args.precond, case),
                   "parallelism": "replicas" if world > 1 else "single",
                   "tiles": {"jv": tiles[0], "precond": tiles[1]},
                   "l2": "working set > L2: the Krylov basis and directions (%d x %.1f MB) stream "
                         "through L2 every Arnoldi pass" % (2 * case["opts"]["krylov_m"] + 1, n * 4 / 1e6),
                   "newton_rtol": case["opts"]["newton_rtol"], "dt": case["opts"]["dt"]},
        "newton_per_step": newt, "gmres_iters_per_step": iters,
        "clocks": clk, "gpu_launches": launches, "e2e": e2e, "roofline": roof, "kernels": kernels,
        "kernels_timing": "per-family CUDA events over 2 steps right before the timed region" if kernels else None,
        "fp64_plain": fp64, "mixed_over_fp64": (value / fp64["value"]) if fp64 else None,
        "precision_error": precision,
        "nonlinear_pc": nonlinear,
        "nonlinear_over_block": (nonlinear["value"] / value) if nonlinear else None,
        "schur_pc": schur,
        "schur_over_block": (schur["value"] / value) if schur else None,
        "schur_over_fp64": (schur["value"] / fp64["value"]) if (schur and fp64) else None,
        "learned_pc": learned or None,
        "learned_pc_3d": learned3d,
        "learned_over_fp64_3d": learned3d["learned_over_fp64"] if learned3d else None,
        "learned_over_fp64": next((L["learned"]["value"] / fp64["value"] for L in learned
                                   if fp64 and L["workload"] == args.workload), None),
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.unet_forward > 0:
        run_unet_forward(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    if args.workload.startswith("uhi_batch") or args.workload.startswith("uhi3d_batch"):
        run_batch(args, rank, world, local_rank)
    else:
        run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
