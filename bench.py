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
CUDA events on the stream the library launches on; max over ranks. Inputs
(~1 GB resident) are larger than the 129 MB L2, so no flush is needed.

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
# Algorithmic HBM bytes per zone-cycle of the FP64 step: each stage reads the
# stage input P (8 doubles) and U^n (8) and writes its output P (8); stage 2
# also writes U^{n+1} (8): 56 doubles = 448 B, plus the axisymmetric geometry
# re-read per (i, j) column and amortised over n3.
ALG_BYTES_PER_ZONE_CYCLE = 448.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["kh", "reference"], default="kh")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--n3", type=int, default=WORKLOAD["n3"], help="azimuthal zones (96 = the named workload)")
    return p.parse_args()


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
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

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
                 "-lms", "200"], stdout=self.tmp, stderr=subprocess.DEVNULL)
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
            f"2-stage Noble-2D FP64, floors bsq/rho<100, 4e-2 u noise (seed 2)")


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
def run_kh(args, world, rank, local):
    import numpy as np
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

    cfg = workload_cfg(args.n3)
    nz = cfg["n1"] * cfg["n2"] * cfg["n3"]
    P0 = inputs.torus_state(cfg, seed=2)
    ctx = kh.Context(cfg, device=dev)
    N1 = P0.shape[3]

    def fresh():
        PB = ctx.to_device(P0)
        P, B = ctx.split(PB)
        U = ctx.empty(8)
        ctx.prim_to_cons(P, B, U)
        return U, PB, P, B

    U, PB, P, B = fresh()
    dt0 = ctx.cfl_dt(P, B)

    # ---- 1-step error against the oracle (rank 0, N = 1 only) ----
    err = None
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        dt1 = 0.5 * dt0
        ctx.step(U, P, B, dt1)
        Ug, Pg = ctx.to_host(U, N1), ctx.to_host(PB, N1)
        cpu, err = cpu_leg(cfg, P0, dt1, Ug, Pg)
        U, PB, P, B = fresh()

    # ---- warm-up ----
    dt = dt0
    for _ in range(args.warmup):
        dt, _ = ctx.step(U, P, B, 0.5 * dt)
    # ---- timed region ----
    ctx.profile(True)
    sampler = ClockSampler(local)
    stream = torch.cuda.current_stream(dev)
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
    prof = ctx.profile_read()
    ctx.profile(False)
    t_max = ms
    if dist:
        t = torch.tensor([ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_max = float(t.item())
    value = nz * args.steps * world / (t_max * 1e-3)

    # ---- end to end through the C ABI with host buffers ----
    e2e = None
    if not args.no_e2e:
        hU = torch.empty(U.shape, dtype=torch.float64, pin_memory=True)
        hPB = torch.empty(PB.shape, dtype=torch.float64, pin_memory=True)
        hU.copy_(U)
        hPB.copy_(PB)
        torch.cuda.synchronize(dev)
        if dist:
            dist.barrier()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.steps):
            U.copy_(hU, non_blocking=True)
            PB.copy_(hPB, non_blocking=True)
            dt, _ = ctx.step(U, P, B, 0.5 * dt)
            hU.copy_(U, non_blocking=True)
            hPB.copy_(PB, non_blocking=True)
        f1.record(stream)
        torch.cuda.synchronize(dev)
        ems = f0.elapsed_time(f1)
        if dist:
            t = torch.tensor([ems], device=dev, dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ems = float(t.item())
        nbytes = (U.numel() + PB.numel()) * 8
        e2e = {"value": nz * args.steps * world / (ems * 1e-3), "unit": UNIT, "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": nbytes}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    # ---- roofline of the dominant kernel group ----
    hbm, hbm_kind, sm_max = peaks()
    groups = {k: v for k, v in prof.items() if v[1] > 0}
    top = max(groups, key=lambda k: groups[k][0])
    top_ms, top_n = groups[top]
    avg_ms = top_ms / top_n
    share = {k: round(v[0] / sum(x[0] for x in groups.values()), 4) for k, v in groups.items()}
    fp64_peak = fp64_peak_tflops(sm_max)
    flops_zone = FP64_FLOPS_PER_ZONE.get(top)
    achieved = (flops_zone * nz / (avg_ms * 1e-3) / 1e12) if flops_zone else None
    roofline = {
        "bound": "alu", "kernel": top, "achieved": achieved, "peak": round(fp64_peak, 4), "unit": "TFLOP/s",
        "frac": (achieved / fp64_peak) if achieved else None, "traffic": TRAFFIC_PER_LAUNCH.get(top),
        "peak_source": "FP64 from unit counts: 152 SMs x 4 flop/clk x max SM clock (measured probe 1.20 TFLOP/s)",
        "avg_launch_ms": avg_ms, "flops_per_zone": flops_zone,
    }
    hbm_step = {"algorithmic_bytes_per_zone_cycle": ALG_BYTES_PER_ZONE_CYCLE,
                "achieved_gbs": ALG_BYTES_PER_ZONE_CYCLE * value / world / 1e9,
                "peak_gbs": hbm, "peak_kind": hbm_kind}
    hbm_step["frac"] = hbm_step["achieved_gbs"] / hbm
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(cfg), "precision": "fp64", "zones": nz,
                   "l2": "inputs larger than L2 (~1 GB resident), no flush",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "roofline": roofline, "hbm_step": hbm_step,
        "kernel_share": share,
        "cpu_baseline": cpu, "err_vs_oracle": err, "e2e": e2e, "gpu_launches": launches,
        "clocks": clocks, "nfail_timed": nfail,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


# FP64 floating-point operations per zone of each kernel group, counted from
# ncu's executed DFMA/DADD/DMUL instruction totals (2 flops per FMA) on the
# torus workload, divided by the zones a launch processes.
FP64_FLOPS_PER_ZONE: dict = {}
# dram read + write bytes per launch of each group from one ncu capture
TRAFFIC_PER_LAUNCH: dict = {}


def cpu_leg(cfg, P0, dt, Ug, Pg):
    """The oracle as it stands on the host cores: one full step of the same
    workload from the same state (bounded sample: one step), plus the GPU
    path's 1-step error against it."""
    import numpy as np

    import oracle
    from paper_2408_01361_gb300 import inputs

    oracle.build()
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    U0 = oracle.prim_to_cons(cfg, P0)
    t0 = time.perf_counter()
    Uo, Po, dto, st = oracle.step(cfg, U0, P0, dt)
    el = time.perf_counter() - t0
    nz = cfg["n1"] * cfg["n2"] * cfg["n3"]
    sl = (slice(None),) + inputs.interior(cfg)
    errs = {}
    for name, a, b in (("U", Ug[sl], Uo[sl]), ("P", Pg[sl], Po[sl])):
        e = []
        for v in range(8):
            den = np.abs(b[v]).sum()
            e.append(float(np.abs(a[v] - b[v]).sum() / den) if den > 0 else float(np.abs(a[v]).sum()))
        errs[name] = e
    cpu = {"value": nz / el, "unit": UNIT, "cores": oracle.get_threads(), "kind": "oracle",
           "sample": f"1 two-stage step of the full {cfg['n1']}x{cfg['n2']}x{cfg['n3']} torus ({el:.1f} s)"}
    err = {"rel_l1_per_var": errs, "max": max(max(errs["U"]), max(errs["P"])),
           "how": "1 step from the same state and dt, GPU FP64 path vs FP64 oracle"}
    return cpu, err


def main():
    args = parse()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, world, rank)
    return run_kh(args, world, rank, local)


if __name__ == "__main__":
    sys.exit(main())
