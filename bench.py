#!/usr/bin/env python3
"""Benchmark of the HARM ideal-GRMHD step on GB300: zone-cycles/s of the
Fishbone-Moncrief torus (Kerr a = 0.9375, funky MKS, 192x96x96, WENO5,
Flux-CT, LLF, two-stage update, Noble-2D inversion with floors), the paper's
performance workload ("Performance" section: torus in spherical-type
coordinates, zone-cycles per second).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl kh|reference]

Prints ONE JSON line (rank 0). The timed region holds exactly K full steps
(both stages, ghost fills, Flux-CT, inversions, fixups and the CFL reduction)
bracketed by a barrier and device synchronisation on both sides, timed with
CUDA events on the stream the library launches on; max over ranks. Each
step is one kh_step call, timed two ways over K steps: replaying the step's
captured CUDA graph (kh_set_graph; captured by an untimed step first) and
launched kernel by kernel (the mixed step's kernels chained by programmatic
dependent launch); the faster is the headline (`mode` names it; `graph` and
`eager` carry both). The per-kernel timings (roofline, kernel_share) come
from the same K steps replayed once more with the library's group events
recorded inside the graph (`profiled_graph`). Inputs (~1 GB resident) are
larger than the 129 MB L2, so no flush is needed.

Beside the headline (mixed path) the line carries the FP64 path, the
statically refined torus (`smr`), the adjoint's cost (`adjoint`) and the
torus on a 128^3 MKS grid (`torus_128cubed`, the size the paper quotes its
A100 figure on; context only).

--impl reference times the FP64 CPU oracle (the method written from its
definitions) on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "zone-cycles/s on 1 GB300 (mixed vs FP64), % HBM roofline, err vs FP64 oracle"
UNIT = "zone-cycles/s"
WORKLOAD = dict(n1=192, n2=96, n3=96)
# Algorithmic HBM bytes per zone-cycle. FP64 step: each stage reads its input
# P (8 doubles) and U^n (8) and writes its output P (8); stage 2 also writes
# U^{n+1} (8): 56 doubles = 448 B. Mixed step: stage 1 reads P^n (FP64, 64 B)
# and U^n (64 B) and writes the FP32 P* (32 B); stage 2 reads P* (32 B) and U^n
# (64 B) and writes P^{n+1} (64 B) and U^{n+1} (64 B): 384 B. The axisymmetric
# geometry re-read per (i, j) column adds ~21 B (FP64) amortised over n3.
ALG_BYTES_PER_ZONE_CYCLE = {"fp64": 448.0, "mixed": 384.0}
DTYPE = {"fp64": "f64", "mixed": "f32+f64"}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=50)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["kh", "reference"], default="kh")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--n3", type=int, default=WORKLOAD["n3"], help="azimuthal zones (96 = the named workload)")
    p.add_argument("--no-smr", action="store_true", help="skip the statically refined torus leg")
    p.add_argument("--no-adjoint", action="store_true", help="skip the adjoint-cost leg")
    p.add_argument("--no-cube", action="store_true", help="skip the 128^3 MKS torus leg")
    p.add_argument("--no-fofc", action="store_true", help="skip the first-order flux correction leg")
    p.add_argument("--no-facect", action="store_true", help="skip the face-centred constrained transport leg")
    p.add_argument("--no-inverters", action="store_true", help="skip the primitive-recovery solver leg")
    p.add_argument("--no-workloads", action="store_true", help="skip the Orszag-Tang / explosion leg")
    p.add_argument("--no-fp64-inversion", action="store_true",
                   help="skip the mixed leg with the whole inversion in FP64")
    p.add_argument("--smr-only", action="store_true", help="run only the statically refined torus leg")
    p.add_argument("--smr-n3", type=int, default=64,
                   help="azimuthal zones of the refined torus's level-0 grid (64 = the named workload; 32 = "
                        "a half-size case of the same blocks, for profiler captures)")
    p.add_argument("--precisions", default="mixed,fp64",
                   help="comma list; the first is the headline, the others are reported beside it")
    a = p.parse_args()
    a.precisions = [x.strip() for x in a.precisions.split(",") if x.strip()]
    return a


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured", d.get("sm_max_mhz", 2070.0)
    return 6800.0, "fallback", 2070.0


# FP64 peak from unit counts and clock: 152 SMs x 4 FP64 flop/clk/SM (2 FMA)
# x the maximum SM clock.
def fp64_peak_tflops(sm_mhz: float) -> float:
    return 152 * 4 * sm_mhz * 1e6 / 1e12


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 20 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.tmp = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "20"], stdout=self.tmp, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.tmp.flush()
        self.tmp.seek(0)
        rows = [r.split(",") for r in self.tmp.read().strip().splitlines() if r.strip()]
        os.unlink(self.tmp.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for q, nm in enumerate(names):
                if len(r) > 5 + q and r[5 + q].strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def workload_cfg(n3: int):
    from paper_2408_01361_gb300 import inputs
    return inputs.torus_cfg(WORKLOAD["n1"], WORKLOAD["n2"], n3)


def workload_name(cfg) -> str:
    return (f"FM torus a=0.9375 FMKS {cfg['n1']}x{cfg['n2']}x{cfg['n3']} WENO5 LLF Flux-CT "
            f"2-stage Noble-2D, floors bsq/rho<100, 4e-2 u noise (seed 2)")


def max_over_ranks(ms: float, dist, dev) -> float:
    """The largest of every rank's elapsed time (the job's time: each rank's
    units count in the throughput only once the slowest rank is done); ms
    itself on a single process (dist None)."""
    if not dist:
        return ms
    import torch

    t = torch.tensor([ms], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def throughput(zones_per_rank: int, steps: int, world: int, ms: float) -> float:
    """Whole-job zone-cycles/s: the zones every rank stepped, over the
    slowest rank's time."""
    return zones_per_rank * steps * world / (ms * 1e-3)


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ---------------------------------------------------------------------------
# reference arm: the oracle on the host cores
# ---------------------------------------------------------------------------
def run_reference(args, world, rank):
    if rank != 0:
        return 0
    import numpy as np

    import oracle
    from paper_2408_01361_gb300 import inputs

    oracle.build()
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    cfg = workload_cfg(8)  # bounded sample: 8 of the 96 azimuthal zones, same (r, theta) grid
    P = inputs.torus_state(cfg, seed=2)
    U = oracle.prim_to_cons(cfg, P)
    dt = 0.5 * oracle.cfl_dt(cfg, P)
    nz = cfg["n1"] * cfg["n2"] * cfg["n3"]
    for _ in range(args.warmup):
        U, P, dt, _ = oracle.step(cfg, U, P, dt)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        U, P, dt, _ = oracle.step(cfg, U, P, dt)
    el = time.perf_counter() - t0
    value = nz * args.steps / el
    sample = f"192x96x8 slab of the torus (same r, theta grid; 8 of 96 azimuthal zones), {args.steps} steps"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(workload_cfg(WORKLOAD["n3"])), "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.get_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# the CUDA arm
# ---------------------------------------------------------------------------
def measure(args, cfg, P0, ctx, dev, stream, dist, world, oracle_step, e2e=True):
    """Warm-up + K timed steps (+ e2e) of one context; returns a dict."""
    import torch

    N1 = P0.shape[3]
    nz = cfg["n1"] * cfg["n2"] * cfg["n3"]

    def fresh():
        PB = ctx.to_device(P0)
        P, B = ctx.split(PB)
        U = ctx.empty(8)
        ctx.prim_to_cons(P, B, U)
        return U, PB, P, B

    U, PB, P, B = fresh()
    dt0 = ctx.cfl_dt(P, B)
    tuned = ctx.autotune(U, P, B, 0.5 * dt0)
    err = None
    if oracle_step is not None:
        ctx.step(U, P, B, oracle_step["dt"])
        err = err_vs(cfg, ctx.to_host(U, N1), ctx.to_host(PB, N1), oracle_step)
        U, PB, P, B = fresh()
    dt = dt0
    for _ in range(args.warmup):
        dt, _ = ctx.step(U, P, B, 0.5 * dt)

    def timed(graph, profile):
        """K steps between CUDA events on the library's stream (barrier and
        device synchronisation on both sides); graph: the step replayed as
        the captured CUDA graph (captured by an untimed step first);
        profile: the library's per-group events (inside the graph as
        event record nodes)."""
        nonlocal dt
        ctx.set_graph(graph)
        ctx.profile(profile)
        if graph:
            dt, _ = ctx.step(U, P, B, 0.5 * dt)  # capture
        sampler = ClockSampler(dev.index or 0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if dist:
            dist.barrier()
        torch.cuda.synchronize(dev)
        sampler.start()
        l0 = ctx.launches()
        nfail = 0
        e0.record(stream)
        for _ in range(args.steps):
            dt, nf = ctx.step(U, P, B, 0.5 * dt)
            nfail += nf
        e1.record(stream)
        torch.cuda.synchronize(dev)
        if dist:
            dist.barrier()
        clocks = sampler.stop()
        launches = ctx.launches() - l0
        ms = e0.elapsed_time(e1)
        prof = ctx.profile_read() if profile else None
        ctx.profile(False)
        ms = max_over_ranks(ms, dist, dev)
        return ms, prof, launches, clocks, nfail

    # the step as a CUDA graph (kh_set_graph) and launched kernel by kernel
    # (eager; the mixed step's kernels chained by programmatic dependent
    # launch): both timed over K steps, the faster is the headline
    gms, _, glaunches, gclocks, gnfail = timed(True, False)
    gnfp64 = int(ctx.stats().nfp64)  # zones of the last timed step whose inversion fell back to FP64
    # kernel timings: the same K steps replayed with the library's group
    # events inside the captured graph (event record nodes between the
    # groups; they lengthen the step, not the kernels they bracket)
    pms, prof, _, _, _ = timed(True, True)
    ems_, _, elaunches, eclocks, enfail = timed(False, False)
    enfp64 = int(ctx.stats().nfp64)
    use_graph = gms <= ems_
    ms, launches, clocks, nfail, nfp64 = ((gms, glaunches, gclocks, gnfail, gnfp64) if use_graph
                                          else (ems_, elaunches, eclocks, enfail, enfp64))
    out = {"value": throughput(nz, args.steps, world, ms), "ms": ms, "launches": launches,
           "clocks": clocks, "err": err, "nfail": nfail, "launch": {"tpb_flux": tuned[0], "tpb_update": tuned[1]},
           "nfp64": nfp64,
           "mode": ("CUDA graph replay of kh_step (kh_set_graph)" if use_graph else
                    "kh_step launched kernel by kernel (eager), the mixed step's kernels chained by "
                    "programmatic dependent launch; the faster of eager and graph replay")}
    out["graph"] = {"value": throughput(nz, args.steps, world, gms), "ms_per_step": gms / args.steps}
    out["prof"] = prof
    out["profiled_graph"] = {"value": throughput(nz, args.steps, world, pms), "ms_per_step": pms / args.steps,
                             "how": "the captured step with the per-group CUDA events recorded inside every "
                                    "replay; source of the kernel timings (roofline, kernel_share)"}
    out["eager"] = {"value": throughput(nz, args.steps, world, ems_), "ms_per_step": ems_ / args.steps}
    ctx.set_graph(use_graph)
    if use_graph:
        dt, _ = ctx.step(U, P, B, 0.5 * dt)  # capture (untimed) for the end-to-end leg
    if e2e and not args.no_e2e:
        # the state crosses the host link in the library's compact interior
        # order (kh_pack_state / kh_unpack_state: no ghost cells, no padding)
        stage_d = torch.empty(16 * nz, dtype=torch.float64, device=dev)
        host = torch.empty(16 * nz, dtype=torch.float64, pin_memory=True)
        ctx.pack_state(U, P, B, stage_d)
        host.copy_(stage_d)
        torch.cuda.synchronize(dev)
        if dist:
            dist.barrier()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.steps):
            stage_d.copy_(host, non_blocking=True)
            ctx.unpack_state(stage_d, U, P, B)
            dt, _ = ctx.step(U, P, B, 0.5 * dt)
            ctx.pack_state(U, P, B, stage_d)
            host.copy_(stage_d, non_blocking=True)
        f1.record(stream)
        torch.cuda.synchronize(dev)
        ems = max_over_ranks(f0.elapsed_time(f1), dist, dev)
        nbytes = host.numel() * 8
        copy_engine = {"value": throughput(nz, args.steps, world, ems), "unit": UNIT, "h2d_bytes_per_step": nbytes,
                       "d2h_bytes_per_step": nbytes,
                       "how": "pinned host buffer -> device buffer (copy engine) -> kh_unpack_state; kh_step; "
                              "kh_pack_state -> device buffer -> pinned host buffer"}
        # the same through the pinned host buffer itself: kh_unpack_state reads
        # it and kh_pack_state writes it over the host link (no staging copy)
        if dist:
            dist.barrier()
        torch.cuda.synchronize(dev)
        z0, z1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        z0.record(stream)
        for _ in range(args.steps):
            ctx.unpack_state(host, U, P, B)
            dt, _ = ctx.step(U, P, B, 0.5 * dt)
            ctx.pack_state(U, P, B, host)
        z1.record(stream)
        torch.cuda.synchronize(dev)
        zms = max_over_ranks(z0.elapsed_time(z1), dist, dev)
        direct = {"value": throughput(nz, args.steps, world, zms), "unit": UNIT, "h2d_bytes_per_step": nbytes,
                  "d2h_bytes_per_step": nbytes,
                  "how": "kh_unpack_state reading the pinned host buffer and kh_pack_state writing it, over the "
                         "host link (no staging copy); kh_step between"}
        best, other = (direct, copy_engine) if direct["value"] >= copy_engine["value"] else (copy_engine, direct)
        out["e2e"] = dict(best, alternative=other)
    return out


def measure_cube(args, dev, stream, precision, n=128):
    """The FM torus on an n^3 MKS grid (the size the paper quotes its A100
    figure on): warm-up, then timed steps with CUDA events; eager and as a
    CUDA graph."""
    import torch

    from paper_2408_01361_gb300 import inputs, kh

    cfg = dict(inputs.torus_cfg(n, n, n), coords="mks", name=f"fm torus mks {n}^3", precision=precision)
    P0 = inputs.torus_state(cfg, seed=2)
    ctx = kh.Context(cfg, device=dev)
    PB = ctx.to_device(P0)
    P, B = ctx.split(PB)
    del P0
    U = ctx.empty(8)
    ctx.prim_to_cons(P, B, U)
    dt = ctx.cfl_dt(P, B)
    ctx.autotune(U, P, B, 0.5 * dt)
    for _ in range(max(args.warmup, 3)):
        dt, _ = ctx.step(U, P, B, 0.5 * dt)
    steps = max(args.steps, 5)
    out = {"workload": f"FM torus a=0.9375 MKS {n}^3 WENO5 LLF Flux-CT 2-stage Noble-2D (seed 2)",
           "precision": precision, "zones": n ** 3}
    for graph in (False, True):
        ctx.set_graph(graph)
        if graph:
            dt, _ = ctx.step(U, P, B, 0.5 * dt)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(steps):
            dt, _ = ctx.step(U, P, B, 0.5 * dt)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / steps
        out["graph" if graph else "eager"] = {"value": n ** 3 / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms}
    ctx.set_graph(False)
    return out


def measure_fofc(args, cfg64, P0, dev, stream, precision):
    """The workload torus with the first-order flux correction on (trial
    update, flag ghosts, donor-cell faces, second Flux-CT per stage): timed
    steps with CUDA events, eager and as a CUDA graph, and the zones flagged
    per step."""
    import torch

    from paper_2408_01361_gb300 import kh

    cfg = dict(cfg64, precision=precision, fofc=True)
    nz = cfg["n1"] * cfg["n2"] * cfg["n3"]
    ctx = kh.Context(cfg, device=dev)
    PB = ctx.to_device(P0)
    P, B = ctx.split(PB)
    U = ctx.empty(8)
    ctx.prim_to_cons(P, B, U)
    dt = ctx.cfl_dt(P, B)
    ctx.autotune(U, P, B, 0.5 * dt)  # the plain step's choice (process-wide cache)
    for _ in range(max(args.warmup, 3)):
        dt, _ = ctx.step(U, P, B, 0.5 * dt)
    steps = max(args.steps, 5)
    out = {"precision": precision, "zones": nz}
    for graph in (False, True):
        ctx.set_graph(graph)
        if graph:
            dt, _ = ctx.step(U, P, B, 0.5 * dt)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(steps):
            dt, _ = ctx.step(U, P, B, 0.5 * dt)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / steps
        out["graph" if graph else "eager"] = {"value": nz / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms}
    ctx.set_graph(False)
    st = ctx.stats()
    out["nfofc_last_step"] = int(st.nfofc)
    out["nfloor_last_step"] = int(st.nfloor)
    ctx.close()
    return out


def measure_facect(args, cfg64, P0, dev, stream, precision, emf="gs05"):
    """The workload torus with face-centred constrained transport (its loop
    field on faces, upwinded edge EMFs): timed steps with CUDA events, eager
    and as a CUDA graph, and the face divergence after them."""
    import torch

    from paper_2408_01361_gb300 import inputs, kh

    cfg = dict(cfg64, precision=precision, bfield="face", emf=emf)
    nz = cfg["n1"] * cfg["n2"] * cfg["n3"]
    fB0 = inputs.torus_face_field(cfg)
    ctx = kh.Context(cfg, device=dev)
    PB = ctx.to_device(P0)
    P, B = ctx.split(PB)
    fB = ctx.to_device(fB0)
    del fB0
    ctx.set_face_field(fB)
    ctx.face_to_cell(fB, B)
    U = ctx.empty(8)
    ctx.prim_to_cons(P, B, U)
    dt = ctx.cfl_dt(P, B)
    ctx.autotune(U, P, B, 0.5 * dt)
    for _ in range(max(args.warmup, 3)):
        dt, _ = ctx.step(U, P, B, 0.5 * dt)
    steps = max(args.steps, 5)
    out = {"precision": precision, "emf": emf, "zones": nz}
    for graph in (False, True):
        ctx.set_graph(graph)
        if graph:
            dt, _ = ctx.step(U, P, B, 0.5 * dt)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(steps):
            dt, _ = ctx.step(U, P, B, 0.5 * dt)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / steps
        out["graph" if graph else "eager"] = {"value": nz / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms}
    ctx.set_graph(False)
    mx, l1 = ctx.face_divb(fB)
    out["face_divb_max"] = mx
    ctx.close()
    return out


def measure_inverters(args, cfg64, P0, dev, stream):
    """Primitive recovery by solver: the workload torus stepped with each, FP64
    and mixed (zone-cycles/s, graph; zones handed to the fixup per step; the
    mixed path runs Noble-2D in double-float, the others in FP64), and a stress
    set of random states (sigma to 1e4, |u~| to 50, an unrelated guess)
    recovered by kh_cons_to_prim (states/s, failures)."""
    import numpy as np
    import torch

    from paper_2408_01361_gb300 import inputs, kh

    nz = cfg64["n1"] * cfg64["n2"] * cfg64["n3"]
    out = {}
    scfg = inputs.torus_cfg(256, 128, 64)
    scfg["x1"] = (np.log(1.2), np.log(50.0))
    Ps = inputs.random_prims(scfg, seed=21, rho_range=(1e-6, 1.0), u_range=(1e-8, 1.0),
                             ut_scale=(30.0, 30.0, 30.0), b_scale=(60.0, 60.0, 60.0))
    far = inputs.random_prims(scfg, seed=22)
    far[5:] = Ps[5:]
    for inv in ("noble2d", "1dw", "kastaun"):
        r = {}
        for prec in ("fp64", "mixed"):
            cfg = dict(cfg64, precision=prec, inverter=inv)
            ctx = kh.Context(cfg, device=dev)
            PB = ctx.to_device(P0)
            P, B = ctx.split(PB)
            U = ctx.empty(8)
            ctx.prim_to_cons(P, B, U)
            dt = ctx.cfl_dt(P, B)
            ctx.autotune(U, P, B, 0.5 * dt)
            for _ in range(max(args.warmup, 3)):
                dt, _ = ctx.step(U, P, B, 0.5 * dt)
            ctx.set_graph(True)
            dt, _ = ctx.step(U, P, B, 0.5 * dt)
            steps = max(min(args.steps, 5), 3)
            nfail = 0
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize(dev)
            e0.record(stream)
            for _ in range(steps):
                dt, nf = ctx.step(U, P, B, 0.5 * dt)
                nfail += nf
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms = e0.elapsed_time(e1) / steps
            ctx.close()
            sfx = "" if prec == "fp64" else "_mixed"
            r["torus_graph" + sfx] = {"value": nz / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms}
            r["torus_fixup_zones_per_step" + sfx] = nfail / steps
        # stress set: every cell of a 262x134x70 grid, recovered from an unrelated guess
        c2 = dict(scfg, inverter=inv)
        ctx = kh.Context(c2, device=dev)
        PBs = ctx.to_device(Ps)
        Pd, Bd = ctx.split(PBs)
        Ud = ctx.empty(8)
        ctx.prim_to_cons(Pd, Bd, Ud)
        G = ctx.to_device(far)
        Pg, Bg = ctx.split(G)
        fails = ctx.cons_to_prim(Ud, Pg, Bg, None)  # warm-up and failure count
        G.copy_(ctx.to_device(far))
        e0.record(stream)
        ctx.cons_to_prim(Ud, Pg, Bg, None)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        cells = Ps[0].size
        r["stress_c2p"] = {"states": cells, "failures": int(fails), "failure_rate": fails / cells,
                           "states_per_s": cells / (e0.elapsed_time(e1) * 1e-3)}
        ctx.close()
        out[inv] = r
    return out


def measure_workloads(args, dev, stream, n=2048):
    """The Minkowski test problems as throughput workloads: the Orszag-Tang
    vortex and the cylindrical explosion on n^2 grids, mixed and FP64, timed
    as CUDA graphs after a warm-up."""
    import torch

    from paper_2408_01361_gb300 import inputs, kh

    out = {}
    for name, mk, st in (("orszag_tang", inputs.orszag_tang_cfg, inputs.orszag_tang_state),
                         ("explosion", inputs.explosion_cfg, inputs.explosion_state)):
        res = {"zones": n * n}
        for prec in args.precisions:
            cfg = dict(mk(n), precision=prec)
            ctx = kh.Context(cfg, device=dev)
            PB = ctx.to_device(st(cfg))
            P, B = ctx.split(PB)
            U = ctx.empty(8)
            ctx.prim_to_cons(P, B, U)
            dt = ctx.cfl_dt(P, B)
            ctx.autotune(U, P, B, dt)
            for _ in range(max(args.warmup, 3)):
                dt, _ = ctx.step(U, P, B, dt)
            ctx.set_graph(True)
            dt, _ = ctx.step(U, P, B, dt)
            steps = max(args.steps, 5)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize(dev)
            e0.record(stream)
            for _ in range(steps):
                dt, _ = ctx.step(U, P, B, dt)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms = e0.elapsed_time(e1) / steps
            res[prec] = {"value": n * n / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms}
            ctx.close()
        out[name] = res
    return out


def measure_smr(args, dev, stream, precision, face=False, integrator="vl2", fofc=False):
    """The statically refined torus (3 levels, 592 uneven blocks, 5.57 M zones)
    stepped as one mesh: every kernel covers all blocks, ghost zones of every
    block are filled by one gather, the step is replayed as a CUDA graph.
    face: face-centred CT with interface-matched upwinded EMFs (the loop
    field curled onto every block's faces from the shared corner potential).
    integrator: the time integrator ("vl2": the predictor-corrector; "rk1",
    "rk2", "ssprk54": Runge-Kutta stages over the whole mesh). fofc: the
    first-order flux correction in every stage (trial over all blocks, flags
    carried across block boundaries by the ghost map)."""
    import torch

    from paper_2408_01361_gb300 import inputs, kh

    base, blocks = inputs.smr_torus_layout(n3=args.smr_n3)
    base = dict(base, integrator=integrator, fofc=1 if fofc else 0)
    if face:
        base = dict(base, bfield="face", emf="gs05")
    norms = inputs.torus_norms(base)
    cfgs = [inputs.block_cfg(base, b) for b in blocks]
    Ps = [inputs.torus_state(c, seed=2, norms=norms) for c in cfgs]
    m = kh.Mesh(dict(base, precision=precision), blocks, device=dev)
    fB = None
    if face:
        fs = [inputs.torus_face_field(c, norms=norms) for c in cfgs]
        Ps = [inputs.cell_field_from_faces(c, f, P) for c, f, P in zip(cfgs, fs, Ps)]
        fB = m.faces_to_device(fs)
        del fs
        m.set_face_field(fB)
    P, B = m.to_device(Ps)
    del Ps
    U = m.empty(8)
    m.prim_to_cons(P, B, U)
    dt = m.cfl_dt(P, B)
    tuned = m.autotune(U, P, B, 0.5 * dt)
    m.set_graph(True)
    for _ in range(args.warmup):
        dt, _ = m.step(U, P, B, 0.5 * dt)
    sampler = ClockSampler(dev.index or 0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    sampler.start()
    l0 = m.launches()
    nfail = 0
    e0.record(stream)
    for _ in range(args.steps):
        dt, nf = m.step(U, P, B, 0.5 * dt)
        nfail += nf
    e1.record(stream)
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    from collections import Counter
    shapes = Counter(f"L{b['level']}:{b['n1']}x{b['n2']}x{b['n3']}" for b in blocks)
    out = {
        "workload": "FM torus (as above) on 3 static refinement levels: level 2 over the disc, level 1 around "
                    f"it, level 0 at the poles and outer radii; base {base['n1']}x{base['n2']}x{base['n3']}"
                    + ("; face-centred CT, interface-matched upwinded EMFs" if face else "")
                    + (f"; integrator {integrator}" if integrator != "vl2" else "")
                    + ("; first-order flux correction" if fofc else ""),
        "precision": precision, "dtype": DTYPE[precision], "blocks": len(blocks), "block_shapes": dict(shapes),
        "zones": m.zones, "ghost_cells": m.ghost_cells, "value": m.zones * args.steps / (ms * 1e-3), "unit": UNIT,
        "ms_per_step": ms / args.steps, "graph": True, "gpu_launches": m.launches() - l0, "clocks": clocks,
        "nfail_timed": nfail, "launch_config": {"tpb_flux": tuned[0], "tpb_update": tuned[1]},
    }
    if fofc:
        out["nfofc_last_step"] = int(m.stats().nfofc)  # zone-stages flagged by the last step's trials
    m.close()
    return out


def measure_adjoint(args, dev, stream, nsteps: int = 20):
    """Adjoint cost (C5 shapes): 20 FP64 steps forward keeping per-step
    checkpoints, then the 20 adjoint steps in reverse (kh_step_adjoint),
    each timed with CUDA events; the objective's seed is the gradient of the
    total energy."""
    import numpy as np
    import torch

    from paper_2408_01361_gb300 import inputs, kh

    dP = np.zeros(8)
    dP[0] = 1.0  # a density mode: the state only has to be representative
    out = {}
    for name, cfg in (("linear-mode box 64^3", inputs.linear_mode_cfg(64, ndim=3)),
                      ("FM torus 128x64x1 (2-D)", inputs.torus_cfg(128, 64, 1))):
        if cfg["coords"] == "minkowski":
            P0 = inputs.linear_mode_state(cfg, dP, 1.0, amp=1e-4)
        else:
            P0 = inputs.torus_state(cfg, seed=2)
        ctx = kh.Context(cfg, device=dev)
        PB = ctx.to_device(P0)
        P, B = PB[:5].clone(), PB[5:].clone()
        U = ctx.empty(8)
        ctx.prim_to_cons(P, B, U)
        dt = 0.5 * ctx.cfl_dt(P, B)
        ckpt = []
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(nsteps):
            ckpt.append((U.clone(), P.clone(), B.clone()))
            ctx.step(U, P, B, dt, sync=False)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        fwd = e0.elapsed_time(e1)
        gU = torch.zeros_like(U)
        gU[0] = 1.0
        gU[1] = -1.0
        gP, gB = None, None
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for (Uc, Pc, Bc) in reversed(ckpt):
            gU, gP, gB, _ = ctx.step_adjoint(Uc, Pc, Bc, dt, gU, gP, gB)
        a1.record(stream)
        torch.cuda.synchronize(dev)
        adj = a0.elapsed_time(a1)
        nz = cfg["n1"] * cfg["n2"] * cfg["n3"]
        out[name] = {"steps": nsteps, "forward_ms_per_step": fwd / nsteps, "adjoint_ms_per_step": adj / nsteps,
                     "adjoint_over_forward": adj / fwd, "zones": nz, "precision": "f64",
                     "finite": bool(torch.isfinite(gP).all() and torch.isfinite(gB).all())}
        ctx.close()
    return out


def roofline_of(prof, nz, precision, recon="weno5"):
    """Roofline of the kernel group with the largest share of the profiled
    step time, the others beside it. achieved = ALGORITHMIC flops per launch
    (the oracle-counted operations of the method's formulas per zone, x the
    zones of a launch) / the live CUDA-event launch time, against the
    unit-count peak of the path's arithmetic type (FP64 path: FP64; mixed
    path: FP32). `executed` gives the ncu-counted flops the kernel actually
    executes (double-float emulation, Newton iterations, the FP32 WENO's
    scale-free weights included) on the same footing."""
    hbm, hbm_kind, sm_max = peaks()
    groups = {k: v for k, v in prof.items() if v[1] > 0}
    top = max(groups, key=lambda k: groups[k][0])
    share = {k: round(v[0] / sum(x[0] for x in groups.values()), 4) for k, v in groups.items()}
    alg = algorithmic_flops_per_zone(recon)

    def one(group):
        ms, n = groups[group]
        avg = ms / n
        a = alg.get(group)
        byt = DRAM_BYTES_PER_ZONE.get((precision, group))
        if a is None:
            return {"kernel": group, "avg_launch_ms": avg}
        if precision == "fp64":
            peak, ex = fp64_peak_tflops(sm_max), FP64_FLOPS_PER_ZONE.get((precision, group))
            src = "FP64 from unit counts: 152 SMs x 4 flop/clk x max SM clock (a probe measured 1.20 TFLOP/s)"
        else:
            peak, ex = fp32_peak_tflops(sm_max), FP32_FLOPS_PER_ZONE.get((precision, group))
            src = "FP32 from unit counts: 152 SMs x 256 flop/clk x max SM clock (a probe measured 74.7 TFLOP/s)"
        achieved = a * nz / (avg * 1e-3) / 1e12
        out = {
            "bound": "alu", "kernel": group, "achieved": achieved, "peak": round(peak, 4), "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": byt * nz if byt else None, "peak_source": src,
            "avg_launch_ms": avg, "algorithmic_flops_per_zone": a, "fp_type": "f64" if precision == "fp64" else "f32",
            "dram_gbs": (byt * nz / (avg * 1e-3) / 1e9) if byt else None, "hbm_peak_gbs": hbm,
        }
        if ex:
            ea = ex * nz / (avg * 1e-3) / 1e12
            out["executed"] = {"flops_per_zone": ex, "achieved": ea, "frac": ea / peak}
        return out

    roof = one(top)
    others = [g for g in ("flux_x1", "flux_x2", "flux_x3", "update") if g in groups and g != top]
    roof["others"] = [one(g) for g in others]
    return roof, share


# Floating-point operations of the method's formulas per item, counted by the
# oracle's op-counting number type (oracle.count_ops; tests/test_oracle_opcount.py
# checks these constants): one WENO5 face value, one MC cell reconstruction,
# the LLF flux of one face from its two states, the connection sources of one
# zone, the conserved variables of one zone from its primitives.
ALG_OPS = {"weno5": 69.0, "mc": 11.0, "llf": 584.0, "sources": 411.0, "p2c": 172.0}


def algorithmic_flops_per_zone(recon: str = "weno5", ndim: int = 3) -> dict:
    """Per zone and launch: a face kernel reconstructs the left and right
    states of 8 variables and forms the LLF flux; the update forms the
    sources, the divergence and the update of 8 variables (per variable 2
    flops per direction, then S - div, x c dt, + U^n) and inverts p2c -- the
    inversion counted as one evaluation of p2c (its Newton iterations are
    data-dependent and not counted: a lower bound)."""
    rec = 2 * 8 * (ALG_OPS["weno5"] if recon == "weno5" else ALG_OPS["mc"] / 2.0)
    face = rec + ALG_OPS["llf"]
    update = ALG_OPS["sources"] + 8 * (2 * ndim + 3) + ALG_OPS["p2c"]
    return {"flux_x1": face, "flux_x2": face, "flux_x3": face, "update": update}


def run_kh(args, world, rank, local):
    import torch

    from paper_2408_01361_gb300 import build as kbuild
    from paper_2408_01361_gb300 import inputs, kh

    if not torch.cuda.is_available():
        raise SystemExit("bench.py: no CUDA device (the GB300 path has no CPU fallback)")
    kbuild.build()
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    stream = torch.cuda.current_stream(dev)

    if args.smr_only:
        out = {p: measure_smr(args, dev, stream, p) for p in args.precisions}
        rk = {"mixed": measure_smr(args, dev, stream, "mixed", integrator="ssprk54")}
        print(json.dumps({"smr": out, "smr_ssprk54": rk}), flush=True)
        return 0

    cfg64 = workload_cfg(args.n3)
    nz = cfg64["n1"] * cfg64["n2"] * cfg64["n3"]
    P0 = inputs.torus_state(cfg64, seed=2)

    # the oracle's step from the same state (CPU baseline + error reference)
    oracle_step, cpu = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ctx = kh.Context(cfg64, device=dev)
        PB = ctx.to_device(P0)
        dt1 = 0.5 * ctx.cfl_dt(*ctx.split(PB))
        ctx.close()
        oracle_step, cpu = cpu_leg(cfg64, P0, dt1)

    results = {}
    for prec in args.precisions:
        cfg = dict(cfg64, precision=prec)
        ctx = kh.Context(cfg, device=dev)
        results[prec] = measure(args, cfg, P0, ctx, dev, stream, dist, world, oracle_step)
        ctx.close()
    fp64inv = None
    if "mixed" in args.precisions and not args.no_fp64_inversion:
        # the precision split that keeps the whole Noble-2D inversion (and the
        # floors) in FP64 for every zone, beside the double-float headline
        cfg = dict(cfg64, precision="mixed", mixed_inversion="fp64")
        ctx = kh.Context(cfg, device=dev)
        fp64inv = measure(args, cfg, P0, ctx, dev, stream, dist, world, oracle_step, e2e=False)
        ctx.close()

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    head = args.precisions[0]
    r = results[head]
    roof, share = roofline_of(r["prof"], nz, head)
    roof["timing"] = ("average launch duration from CUDA events around the kernel group inside the profiled "
                      "graph replay of the same K steps (profiled_graph)")
    hbm, hbm_kind, _ = peaks()
    alg = ALG_BYTES_PER_ZONE_CYCLE[head]
    hbm_step = {"algorithmic_bytes_per_zone_cycle": alg, "achieved_gbs": alg * r["value"] / world / 1e9,
                "peak_gbs": hbm, "peak_kind": hbm_kind}
    hbm_step["frac"] = hbm_step["achieved_gbs"] / hbm
    line = {
        "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["ms"] / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPE[head], "data": "synthetic",
        "config": {"workload": workload_name(cfg64), "precision": head, "zones": nz,
                   "l2": "inputs larger than L2 (~1 GB resident), no flush",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "roofline": roof, "hbm_step": hbm_step, "kernel_share": share,
        "cpu_baseline": cpu, "err_vs_oracle": r["err"], "e2e": r.get("e2e"), "gpu_launches": r["launches"],
        "clocks": r["clocks"], "nfail_timed": r["nfail"], "nfp64_last_step": r["nfp64"], "launch_config": r["launch"],
        "mode": r["mode"], "graph": r["graph"], "profiled_graph": r["profiled_graph"], "eager": r["eager"],
    }
    for prec in args.precisions[1:]:
        q = results[prec]
        rf, sh = roofline_of(q["prof"], nz, prec)
        line[prec] = {"value": q["value"], "ms_per_step": q["ms"] / args.steps, "dtype": DTYPE[prec],
                      "err_vs_oracle": q["err"], "e2e": q.get("e2e"), "roofline": rf, "kernel_share": sh,
                      "gpu_launches": q["launches"], "clocks": q["clocks"], "nfail_timed": q["nfail"],
                      "launch_config": q["launch"], "mode": q["mode"], "graph": q["graph"],
                      "profiled_graph": q["profiled_graph"], "eager": q["eager"]}
        line[f"speedup_{head}_vs_{prec}"] = r["value"] / q["value"]
    if fp64inv is not None:
        q = fp64inv
        rf, sh = roofline_of(q["prof"], nz, "mixed")
        line["mixed_fp64_inversion"] = {
            "what": "mixed path with the whole Noble-2D inversion and the floors in FP64 for every zone "
                    "(FP32 stencil; FP64 U^n + increment; kh_coords.mixed_inversion = KH_MIXINV_FP64)",
            "value": q["value"], "ms_per_step": q["ms"] / args.steps, "dtype": "f32+f64",
            "err_vs_oracle": q["err"], "roofline": rf, "kernel_share": sh, "gpu_launches": q["launches"],
            "clocks": q["clocks"], "nfail_timed": q["nfail"], "launch_config": q["launch"], "mode": q["mode"],
            "graph": q["graph"], "eager": q["eager"],
            "headline_over_this": r["value"] / q["value"] if head == "mixed" else None}
    if not args.no_smr and world == 1:
        line["smr"] = {p: measure_smr(args, dev, stream, p) for p in args.precisions}
        line["smr_face_ct"] = {p: measure_smr(args, dev, stream, p, face=True) for p in args.precisions}
        line["smr_ssprk54"] = {"mixed": measure_smr(args, dev, stream, "mixed", integrator="ssprk54")}
        line["smr_fofc"] = {"mixed": measure_smr(args, dev, stream, "mixed", fofc=True)}
    if not args.no_cube and world == 1:
        line["torus_128cubed"] = {p: measure_cube(args, dev, stream, p) for p in args.precisions}
        line["torus_128cubed"]["context"] = "paper: ~35 M zone-cycles/s per A100 GPU on 128^3 production problems"
    if not args.no_fofc and world == 1:
        fo = {}
        for p in args.precisions:
            fo[p] = measure_fofc(args, cfg64, P0, dev, stream, p)
            fo[p]["cost_vs_plain_graph"] = results[p]["graph"]["value"] / fo[p]["graph"]["value"]
        line["fofc"] = fo
    if not args.no_facect and world == 1:
        fc = {}
        for p in args.precisions:
            fc[p] = measure_facect(args, cfg64, P0, dev, stream, p)
            fc[p]["cost_vs_flux_ct_graph"] = results[p]["graph"]["value"] / fc[p]["graph"]["value"]
        line["face_ct"] = fc
    if not args.no_workloads and world == 1:
        line["workloads_2d"] = measure_workloads(args, dev, stream)
    if not args.no_inverters and world == 1:
        line["inverters"] = measure_inverters(args, cfg64, P0, dev, stream)
    if not args.no_adjoint and world == 1:
        line["adjoint"] = measure_adjoint(args, dev, stream)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


# Per-zone figures of each kernel group from one ncu capture of the same
# kernels on the 192x96x64 torus (1 step, mixed and FP64; see profiles/):
# executed floating-point operations per zone and per launch (a DFMA or FFMA
# counts 2, DADD/DMUL/FADD/FMUL 1), and DRAM bytes (read + write) per zone
# per launch. Launch totals at the bench size scale by the zone count.
FP64_FLOPS_PER_ZONE: dict = {
    ("fp64", "update"): 947.0,
    ("fp64", "flux_x1"): 2102.3, ("fp64", "flux_x2"): 2091.0, ("fp64", "flux_x3"): 2083.5,
}
FP32_FLOPS_PER_ZONE: dict = {
    # paired instructions count 2 lanes (an FFMA2 = 4 flops)
    ("mixed", "flux_x1"): 1565.0, ("mixed", "flux_x2"): 1645.0, ("mixed", "flux_x3"): 1714.0,
    ("mixed", "update"): 1903.3,  # stages 1 and 2 (1919.3, 1887.3); FP64: 1 and 21 flops per zone
}
DRAM_BYTES_PER_ZONE: dict = {
    ("mixed", "update"): 279.8,  # the TMA-staged update (32x4 tiles): mean of stage 1 (232.0) and stage 2 (327.6)
    ("mixed", "flux_x1"): 44.4, ("mixed", "flux_x2"): 46.0, ("mixed", "flux_x3"): 47.7,
    ("fp64", "update"): 419.1,  # stage 1
    ("fp64", "flux_x1"): 118.0, ("fp64", "flux_x2"): 126.1, ("fp64", "flux_x3"): 128.3,
}
# FP32 peak from unit counts: 152 SMs x 128 lanes x 2 flop/clk x max SM clock
# (a probe measured 74.7 TFLOP/s at 2070 MHz).
def fp32_peak_tflops(sm_mhz: float) -> float:
    return 152 * 256 * sm_mhz * 1e6 / 1e12


def host_cores() -> dict:
    """The host's core count and this process's affinity (the cores the
    oracle's OpenMP threads may run on)."""
    n = os.cpu_count() or 1
    try:
        aff = sorted(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        aff = list(range(n))
    return {"nproc": n, "affinity_count": len(aff),
            "affinity": f"{aff[0]}-{aff[-1]}" if aff == list(range(aff[0], aff[-1] + 1)) else ",".join(map(str, aff))}


def _oracle_rate(oracle, cfg, P, U, dt, steps, dirichlet=None):
    """Zone-cycles/s of `steps` oracle steps from (U, P) with a fixed dt."""
    nz = cfg["n1"] * cfg["n2"] * cfg["n3"]
    t0 = time.perf_counter()
    for _ in range(steps):
        U, P, _, _ = oracle.step(cfg, U, P, dt, dirichlet)
    el = time.perf_counter() - t0
    return nz * steps / el, el, U, P


def cpu_leg(cfg, P0, dt):
    """The oracle as it stands on the host cores. The headline figure is one
    full step of the workload torus on all the cores this process may use
    (also the state the GPU's error is measured against); beside it, the
    survey's six legs: the 32^3 linear mode (C1), the 128x128 Bondi flow (C2)
    and the workload torus (C3), each single-threaded and on all cores (C3 on
    all cores for 10 steps, single-threaded for one)."""
    import numpy as np

    import oracle
    from paper_2408_01361_gb300 import inputs

    oracle.build()
    hc = host_cores()
    allc = hc["affinity_count"]
    oracle.set_threads(allc)
    U0 = oracle.prim_to_cons(cfg, P0)
    t0 = time.perf_counter()
    Uo, Po, dto, st = oracle.step(cfg, U0, P0, dt)
    el = time.perf_counter() - t0
    nz = cfg["n1"] * cfg["n2"] * cfg["n3"]
    cpu = {"value": nz / el, "unit": UNIT, "cores": oracle.get_threads(), "kind": "oracle",
           "sample": f"1 two-stage step of the full {cfg['n1']}x{cfg['n2']}x{cfg['n3']} torus ({el:.1f} s)",
           "host": hc}
    # the six legs
    dP = np.zeros(8)
    dP[0] = 1.0
    c1 = inputs.linear_mode_cfg(32, ndim=3)
    P1 = inputs.linear_mode_state(c1, dP, 1.0, amp=1e-4)
    U1 = oracle.prim_to_cons(c1, P1)
    dt1 = oracle.cfl_dt(c1, P1)
    c2 = inputs.bondi_cfg(128, 128)
    P2, d2 = inputs.bondi_state(c2, seed=1)
    U2 = oracle.prim_to_cons(c2, P2)
    dt2 = oracle.cfl_dt(c2, P2, d2)
    legs = {}
    for threads, label in ((1, "1 thread"), (allc, f"{allc} threads")):
        oracle.set_threads(threads)
        v1, e1, _, _ = _oracle_rate(oracle, c1, P1, U1, dt1, 20 if threads == 1 else 100)
        v2, e2, _, _ = _oracle_rate(oracle, c2, P2, U2, dt2, 20 if threads == 1 else 100, d2)
        n3 = 1 if threads == 1 else 10
        v3, e3, _, _ = _oracle_rate(oracle, cfg, Po, Uo, dto, n3)
        legs[label] = {
            "threads": oracle.get_threads(),
            "C1 linear mode 32^3": {"value": v1, "unit": UNIT, "seconds": e1},
            "C2 Bondi 128x128": {"value": v2, "unit": UNIT, "seconds": e2},
            f"C3 torus {cfg['n1']}x{cfg['n2']}x{cfg['n3']} ({n3} step{'s' if n3 > 1 else ''})":
                {"value": v3, "unit": UNIT, "seconds": e3},
        }
    oracle.set_threads(allc)
    cpu["legs"] = legs
    return {"U": Uo, "P": Po, "dt": dt}, cpu


def err_vs(cfg, Ug, Pg, ref):
    """Relative L1 per variable of the GPU's one-step state against the oracle's."""
    import numpy as np

    from paper_2408_01361_gb300 import inputs

    sl = (slice(None),) + inputs.interior(cfg)
    errs = {}
    for name, a, b in (("U", Ug[sl], ref["U"][sl]), ("P", Pg[sl], ref["P"][sl])):
        e = []
        for v in range(8):
            den = np.abs(b[v]).sum()
            e.append(float(np.abs(a[v] - b[v]).sum() / den) if den > 0 else float(np.abs(a[v]).sum()))
        errs[name] = e
    return {"rel_l1_per_var": errs, "max": max(max(errs["U"]), max(errs["P"])),
            "how": "1 step from the same state and dt vs the FP64 oracle"}


def main():
    args = parse()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, world, rank)
    return run_kh(args, world, rank, local)


if __name__ == "__main__":
    sys.exit(main())
