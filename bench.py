#!/usr/bin/env python
"""Benchmark of the Scheme II step (arXiv:1909.02894) on the GPU.

A bench step is one time step of the whole hot path (half-step U, x pass, y pass,
half-step U; consecutive U's merged) on the 4096^2 complex64 grid (m=0.5, 16 random
strain bumps, absorbing layer 128, dt=0.05), whose state and coefficient fields are
larger than L2, so no flush is needed between timed steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]
                    [--workload large-4096|large-2048|large-4096-c128|graphene-1024-c64|
                                graphene-1024-c128|plain-128-c128|batch-mix|serve]

Prints one JSON line. The path does not shard: with N > 1 each rank runs an
independent replica and `value` sums the ranks ("replicas only", weak scaling).
The reference arm times the FP64 CPU oracle on the host cores on a bounded sample.

At N = 1 the default line also carries, each with its error against the FP64 oracle:
`rel_l2_vs_oracle` of the 4096^2 grid itself (whole grid, a few steps); `batch`, the
256-instance uneven mix (128^2..1024^2) stepped 2000 times in complex64 beside the plain
complex128 single-instance path (their ratio, per-size rel-L2 of batched and plain
results); and `serving`, a short window of the 200 req/s strained-graphene stream through
the continuous-batching loop (p50/p99 latency, throughput, clocks, FP64 check).
"""
from __future__ import annotations

import argparse
import hashlib
import re
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1909_02894_gb300 import workloads as W  # noqa: E402

METRIC = "grid-point*steps/s"
UNIT = "grid-point*steps/s"
FALLBACK_HBM_GBS = 6800.0
L2_BYTES = 129 * 2 ** 20


def workload(name):
    """(Workload, precision name, algorithmic bytes per grid point per step)."""
    if name == "large-4096":
        return W.large_4096(), "c64", 88
    if name == "large-2048":
        return W.large_4096(n=2048), "c64", 88
    if name == "graphene-1024-c64":
        return W.graphene_strained(n=1024), "c64", 88
    if name == "graphene-1024-c128":
        return W.graphene_strained(n=1024), "c128", 176
    if name == "plain-128-c128":
        return W.plain_128(), "c128", 176
    if name == "large-4096-c128":
        return W.large_4096(), "c128", 176
    raise SystemExit(f"unknown workload {name}")


def kernel_name(w, prec_name):
    """The fused line-pass kernel the default launch shape runs for this grid."""
    if prec_name == "c64" and min(w.nx, w.ny) >= 1024:
        return "line_pass_persistent"
    return "line_pass_kernel"


def hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            for k in ("hbm_gbs", "hbm_GBps", "hbm"):
                if k in d and isinstance(d[k], (int, float)):
                    return float(d[k]), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


# FP64 rate of GB300 (nominal 1.25 TFLOP/s dense FP64: 2 FP64 FMAs per SM per clock on 152
# SMs at 2.07 GHz); the complex128 line pass is bound by it, not by HBM.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def fft_flops_per_point_step(nx, ny):
    """Algorithmic flops of one Scheme II step per grid point, by the 5 N log2 N convention
    for a complex FFT of N points: per direction two components, forward and inverse
    (4 x 5 log2 N per point), plus about 76 pointwise flops (k-space multiply, combine, U)."""
    return 20.0 * (np.log2(nx) + np.log2(ny)) + 76.0


KERNEL_SOURCES = ("line_pass.cuh", "persist_pass.cuh", "launch_impl.cuh", "common.cuh")


def kernel_hash():
    """Hash of the line-pass kernel sources with comments and spacing removed: the committed
    ncu counters (profiles/*traffic.txt) stay valid across comment edits, and any change of
    code voids them."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        src = open(os.path.join(ROOT, "paper_1909_02894_gb300", "csrc", f)).read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def batch_traffic(count, pts):
    """DRAM bytes per step of the whole batch mix from the committed ncu summary of one
    tick, if it was taken on the current kernel sources and the same mix; else None."""
    p = os.path.join(ROOT, "profiles", "batch_tick_traffic.txt")
    if not os.path.exists(p):
        return None
    kv = {}
    for line in open(p):
        if "=" in line and not line.startswith("#"):
            k, v = line.split("=", 1)
            kv[k.strip()] = v.strip()
    if (kv.get("kernel_hash") != kernel_hash() or kv.get("instances") != str(count)
            or kv.get("points_per_step") != str(pts)):
        return None
    try:
        return float(kv["dram_bytes_per_step"])
    except (KeyError, ValueError):
        return None


def ncu_traffic(workload_name, precision):
    """DRAM bytes per launch of the line pass from the committed ncu summary, if it was
    taken on the current kernel source, the same grid and the same precision; else None."""
    p = os.path.join(ROOT, "profiles", "line_pass_traffic.txt")
    if not os.path.exists(p):
        return None
    kv = {}
    for line in open(p):
        if "=" in line and not line.startswith("#"):
            k, v = line.split("=", 1)
            kv[k.strip()] = v.strip()
    if (kv.get("kernel_hash") != kernel_hash() or kv.get("workload") != workload_name
            or kv.get("precision") != precision):
        return None
    try:
        return float(kv["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        for line in (self.out or "").strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


class ProfileRegion:
    """cudaProfilerStart/Stop around a timed region when --profile-region is given, so an
    `ncu --profile-from-start off` capture covers exactly the timed launches."""

    def __init__(self, on):
        self.on = on

    def __enter__(self):
        if self.on:
            import torch

            torch.cuda.synchronize()
            torch.cuda.cudart().cudaProfilerStart()
        return self

    def __exit__(self, *a):
        if self.on:
            import torch

            torch.cuda.synchronize()
            torch.cuda.cudart().cudaProfilerStop()


def alu_peaks():
    """Measured FMA throughput of the device (TFLOP/s): FP64, FP32, packed FP32 pairs."""
    import paper_1909_02894_gb300 as D

    return {"fp64_tflops": D.dirac_measure_alu_peak(D.ALU_FP64),
            "fp32_tflops": D.dirac_measure_alu_peak(D.ALU_FP32),
            "fp32x2_tflops": D.dirac_measure_alu_peak(D.ALU_FP32X2),
            "how": "dirac_measure_alu_peak: 8 x 256-thread blocks per SM, 8 independent FMA "
                   "chains per thread, CUDA events over one >= 2 ms launch after a warm-up"}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(ms, world, device=None):
    """The slowest rank's time: all_reduce(MAX) over the process group (NCCL with CUDA
    tensors, gloo with CPU ones); a single process returns its own."""
    if world <= 1:
        return float(ms)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(points_per_rank, steps, world, ms):
    """Grid-point steps per second of the whole job: every rank runs an independent
    replica of `points_per_rank` points for `steps` steps, over the slowest rank's time."""
    return points_per_rank * steps * world / (ms * 1e-3)


def run_reference(args, wl_name):
    """The FP64 CPU oracle, as it stands, timed on the host cores as the reference arm.
    Each of the K timed steps is one oracle time step on a bounded sample of the
    workload: the same recipe on the largest grid whose K + W steps fit about two
    minutes (estimated from a one-step probe)."""
    world, rank, _ = dist_setup(args)
    if rank != 0:
        return 0
    import oracle

    oracle.build()
    w_full, prec, _ = workload(wl_name)
    recipe = {"large-4096": lambda n: W.large_4096(n=n, steps=1),
              "large-2048": lambda n: W.large_4096(n=n, steps=1),
              "graphene-1024-c64": lambda n: W.graphene_strained(n=n, steps=1),
              "graphene-1024-c128": lambda n: W.graphene_strained(n=n, steps=1),
              "plain-128-c128": lambda n: W.plain_128(n=n, steps=1),
              "large-4096-c128": lambda n: W.large_4096(n=n, steps=1)}[wl_name]
    steps, warm = max(1, args.steps), max(0, args.warmup)
    budget_s = 120.0
    n = 256 if w_full.nx >= 256 else w_full.nx
    probe = recipe(n)
    pp = oracle.Problem.from_workload(probe)
    t0 = time.perf_counter()
    oracle.run(pp, probe.psi0, probe.dt, 1)
    per_pt = (time.perf_counter() - t0) / probe.points
    while n * 2 <= w_full.nx and per_pt * (2 * n) ** 2 * 1.15 * (steps + warm) <= budget_s:
        n *= 2
    w = recipe(n)
    prob = oracle.Problem.from_workload(w)
    psi = oracle.run(prob, w.psi0, w.dt, warm) if warm else w.psi0
    t0 = time.perf_counter()
    oracle.run(prob, psi, w.dt, steps)
    elapsed = time.perf_counter() - t0
    value = w.points * steps / elapsed
    sample = f"{steps} oracle steps on the {n}^2 grid of the {w_full.name} recipe"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": steps, "warmup": warm, "ms_per_step": elapsed / steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": w_full.name, "precision": "f64 oracle",
                                        "sample_grid": [n, n]},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def cpu_baseline(w, scheme="printed", degree=8, check_steps=0):
    """Oracle timing on a bounded sample of the same workload (about 10-30 s of CPU): the
    difference of a k-step and a 1-step run on all host cores, k = max(2,
    check_steps), and the same on one core (on the 1024^2 grid of the recipe when the
    workload is larger). Also returns the oracle's state after max(2, check_steps) steps
    from psi0 (for the rel-L2 of the GPU result)."""
    import oracle

    oracle.build()

    def runner(wl):
        prob = oracle.Problem.from_workload(wl)

        def run(n):
            if scheme == "cn":
                return oracle.run_cn(prob, wl.psi0, wl.dt, n, tol=1e-14)[0]
            if scheme in ("taylor", "chebyshev"):
                fam = oracle.POLY_TAYLOR if scheme == "taylor" else oracle.POLY_CHEBYSHEV
                return oracle.run_poly(prob, wl.psi0, wl.dt, n, fam, degree)
            return oracle.run(prob, wl.psi0, wl.dt, n, scheme=1 if scheme == "symmetric" else 0)
        return run

    def timed(run, n):
        t0 = time.perf_counter()
        out = run(n)
        return time.perf_counter() - t0, out

    def per_step(run, k, tk, t1, min_diff=2.0, max_rounds=4):
        """Seconds per step from the difference of a k-step and a 1-step run; on a grid so
        small that the difference is under min_diff seconds (timer noise and the fixed
        set-up of a run would dominate), longer runs until it is not."""
        for _ in range(max_rounds):
            if tk - t1 >= min_diff:
                break
            diff = tk - t1
            k = int(k * min(64.0, max(2.0, 1.5 * min_diff / diff))) if diff > 0.01 else k * 64
            tk, _ = timed(run, k)
        return max(tk - t1, 1e-9) / (k - 1), k

    k = max(2, check_steps)
    run = runner(w)
    t1, _ = timed(run, 1)
    tk, state = timed(run, k)
    sec, m = per_step(run, k, tk, t1)
    cores = oracle.threads()
    rec = {"value": w.nx * w.ny / sec, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"difference of {m}-step and 1-step FP64 oracle runs on {w.name}, "
                     f"divided by {m - 1}"}
    # one core, on a smaller grid of the same recipe when the full grid is large
    small = w
    if w.nx * w.ny > 1024 * 1024 and w.name.startswith("large-"):
        small = W.large_4096(n=1024, steps=1)
    try:
        oracle.set_threads(1)
        run1 = runner(small)
        t1, _ = timed(run1, 1)
        t2, _ = timed(run1, 2)
        sec, m = per_step(run1, 2, t2, t1, min_diff=1.0)
        rec["single_thread"] = {
            "value": small.nx * small.ny / sec, "unit": UNIT, "cores": 1,
            "sample": f"difference of {m}-step and 1-step runs on {small.name}, divided by {m - 1}"}
    finally:
        oracle.set_threads(cores)
    return rec, state


def plain_c128_rate(w, stream, steps=50):
    """Point-steps/s of the plain complex128 single-instance path on one workload (3
    untimed steps, then `steps` steps timed with CUDA events on the context's stream)."""
    import torch

    import paper_1909_02894_gb300 as D

    with D.Simulation(w, precision=D.DIRAC_C128, stream=stream.cuda_stream) as s:
        s.set_state(w.psi0)
        s.step(3, w.dt)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step(steps, w.dt)
        e1.record(stream)
        torch.cuda.synchronize()
        return w.points * steps / (e0.elapsed_time(e1) * 1e-3)


# Steps of the per-size oracle check of batched results: as many as keep the oracle's
# share of the bench to about 15 s on the host cores.
BATCH_CHECK_STEPS = {128: 1000, 256: 500, 512: 200, 1024: 100}


def batch_record(args, stream, steps, world=1, check=True):
    """Batched uneven mix (256 instances, 128^2..1024^2 with weights 0.4/0.3/0.2/0.1),
    each stepped `steps` times in one batch of graph-captured ticks, complex64; beside it
    the plain complex128 single-instance path on one instance of each size (each alone),
    and, per size, the rel-L2 of a batched result and of the plain complex128 result
    against the FP64 oracle."""
    import torch

    import paper_1909_02894_gb300 as D

    count = args.batch_count
    ws = W.batch_mix(count=count, steps=steps)
    sims = [D.Simulation(w, precision=D.DIRAC_C64, stream=stream.cuda_stream) for w in ws]
    budget = sum(D.dirac_footprint_bytes(w.nx, w.ny) for w in ws) + (1 << 20)
    batch = D.dirac_batch_create(budget, D.DIRAC_C64, steps_per_tick=args.tick,
                                 stream=stream.cuda_stream)
    pts = sum(w.points for w in ws)
    try:
        def run(n_steps, tune=False, profile=False):
            slots = []
            for s, w in zip(sims, ws):
                s.set_state(w.psi0)
                slots.append(D.dirac_batch_submit(batch, s.ctx, n_steps, w.dt))
            torch.cuda.synchronize()
            if tune:  # CTA shapes of every class timed on its contexts (outside the timing)
                D.dirac_batch_autotune(batch, 5)
            if world > 1:
                torch.distributed.barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            with ProfileRegion(profile):
                e0.record(stream)
                ticks = 0
                while D.dirac_batch_active(batch):
                    D.dirac_batch_run(batch, 1)
                    ticks += 1
                e1.record(stream)
                D.dirac_batch_synchronize(batch)
            torch.cuda.synchronize()
            for sl in slots:
                D.dirac_batch_release(batch, sl)
            return max_over_ranks(e0.elapsed_time(e1), world, device="cuda"), ticks

        warm = max(3, args.warmup)
        run(warm, tune=True)
        shapes = {str(n): list(D.dirac_batch_launch_shape(batch, n, n)) for n in W.BATCH_SIZES
                  if any(w.nx == n for w in ws)}
        l0 = D.dirac_batch_launch_count(batch)
        with Clocks(torch.cuda.current_device()) as clk:
            ms, ticks = run(steps, profile=getattr(args, "profile_region", False))
        launches = int(D.dirac_batch_launch_count(batch) - l0)
        value = whole_job_value(pts, steps, world, ms)
        # plain complex128 path, each instance alone, one instance of each size, scaled by
        # the mix's point counts
        sample, seen = [], set()
        for w in ws:
            if w.nx not in seen:
                seen.add(w.nx)
                sample.append(w)
        rates = {w.nx: plain_c128_rate(w, stream) for w in sample}
        t_plain = sum(x.points / rates[x.nx] for x in ws)
        plain = pts / t_plain
        peak, peak_kind = hbm_peak()
        gbs = 88.0 * pts / (ms * 1e-3 / steps) / 1e9
        rec = {
            "workload": f"batch-mix-{count}", "value": value, "unit": UNIT, "steps": steps,
            "warmup": warm, "ms_per_step": ms / steps, "dtype": "f32",
            "precision": "c64 batched, FP64 tables and reductions",
            "sizes": {str(n): sum(1 for w in ws if w.nx == n) for n in W.BATCH_SIZES},
            "points_per_step": pts, "steps_per_tick": args.tick, "ticks": ticks,
            "gpu_launches": launches, "launches_per_tick": launches / max(1, ticks),
            "autotuned_threads_xy": shapes,
            "l2": "working set larger than L2 (no flush)",
            "plain_c128_single_instance": {
                "value": plain, "unit": UNIT,
                "per_size": {str(k): v for k, v in sorted(rates.items())},
                "sample": "one instance of each size alone, 50 steps, weighted by the mix's "
                          "point counts"},
            "batched_over_plain_c128": value / world / plain,
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                         "frac": gbs / peak, "traffic": batch_traffic(count, pts),
                         "peak_source": peak_kind,
                         "kernel": "whole tick (every class's x and y passes)",
                         "algorithmic_bytes_per_point_step": 88,
                         "traffic_unit": "DRAM bytes per step of the whole mix"},
            "clocks": clk.summary(),
        }
        if check:
            rec["rel_l2_vs_oracle"] = batch_oracle_check(batch, sims, ws, sample, stream)
        return rec
    finally:
        D.dirac_batch_destroy(batch)
        for s in sims:
            s.close()


def batch_oracle_check(batch, sims, ws, sample, stream):
    """Per size: one instance stepped in the batch (complex64) and alone in complex128,
    both against the FP64 oracle after BATCH_CHECK_STEPS[n] steps."""
    import torch

    import oracle
    import paper_1909_02894_gb300 as D

    oracle.build()
    idx = {w.nx: ws.index(w) for w in sample}
    slots = {}
    for n, i in idx.items():
        sims[i].set_state(ws[i].psi0)
        slots[n] = D.dirac_batch_submit(batch, sims[i].ctx, BATCH_CHECK_STEPS[n], ws[i].dt)
    while D.dirac_batch_active(batch):
        D.dirac_batch_run(batch, 1)
    D.dirac_batch_synchronize(batch)
    torch.cuda.synchronize()
    out = {}
    for n, i in sorted(idx.items()):
        D.dirac_batch_release(batch, slots[n])
        w, k = ws[i], BATCH_CHECK_STEPS[n]
        got64 = sims[i].get_state()
        with D.Simulation(w, precision=D.DIRAC_C128, stream=stream.cuda_stream) as s:
            s.set_state(w.psi0)
            s.step(k, w.dt)
            got128 = s.get_state()
        ref = oracle.run(oracle.Problem.from_workload(w), w.psi0, w.dt, k)
        out[str(n)] = {"steps": k, "c64_batched": W.rel_l2(got64, ref),
                       "c128_plain": W.rel_l2(got128, ref),
                       "kept_norm": float(np.linalg.norm(ref) / np.linalg.norm(w.psi0))}
    out["max_c64_batched"] = max(v["c64_batched"] for v in out.values())
    return out


def run_batch(args):
    """The batch-mix record as a line of its own (--workload batch-mix): `--steps` steps
    per instance (2000 in the configuration)."""
    import torch

    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    if world > 1:  # independent replicas of the whole mix, one per rank
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local))
    stream = torch.cuda.Stream()
    rec = batch_record(args, stream, args.steps, world, check=(world == 1))
    line = {
        "metric": METRIC, "value": rec["value"], "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": rec["warmup"], "ms_per_step": rec["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": rec["workload"], "precision": "c64 batched",
                   "sizes": rec["sizes"], "points_per_step": rec["points_per_step"],
                   "steps_per_tick": args.tick, "autotuned_threads_xy":
                   rec["autotuned_threads_xy"], "l2": rec["l2"]},
        "plain_c128_single_instance": rec["plain_c128_single_instance"],
        "batched_over_plain_c128": rec["batched_over_plain_c128"],
        "roofline": rec["roofline"], "clocks": rec["clocks"],
        "gpu_launches": rec["gpu_launches"], "launches_per_tick": rec["launches_per_tick"],
    }
    if "rel_l2_vs_oracle" in rec:
        line["rel_l2_vs_oracle"] = rec["rel_l2_vs_oracle"]
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def oracle_reference(max_n):
    """A reference(workload, steps) callable for the serving check: the FP64 CPU oracle on
    grids up to max_n^2 (None above, where the check falls back to the complex128 path)."""
    import oracle

    oracle.build()

    def ref(w, steps):
        if w.nx > max_n:
            return None
        return oracle.run(oracle.Problem.from_workload(w), w.psi0, w.dt, steps)
    return ref


def serve_record(args, stream, rate, window, check=True, plain_rates=None):
    """The strained-graphene request stream through the continuous-batching loop: Poisson
    arrivals at `rate` over `window` seconds, grids {256,512,1024,2048}^2, steps
    U{500..5000}, complex64; latency p50/p99, throughput, clocks, and the FP64 check of 1%
    of the requests (at least one)."""
    import torch

    from paper_1909_02894_gb300 import serve as S

    free, total = torch.cuda.mem_get_info()
    budget = int(0.8 * free)
    reqs = S.graphene_requests(rate=rate, duration=window, seed=1914)
    if check and reqs and not any(r.check for r in reqs):
        reqs[0].check = True
    work = sum(r.nx * r.ny * r.steps for r in reqs)
    srv = S.Server(budget, steps_per_tick=args.tick, stream=stream.cuda_stream,
                   policy=args.serve_policy, max_active_points=args.serve_cap_points)
    try:
        for r in reqs:
            srv.submit(r)
        with Clocks(torch.cuda.current_device()) as clk:
            t0 = time.perf_counter()
            results = srv.run(t0=t0)
            elapsed = time.perf_counter() - t0
    finally:
        srv.close()
    summ = S.latency_summary(results)
    summ.update({"rate_per_s": rate, "window_s": window, "throughput": work / elapsed,
                 "unit": UNIT, "elapsed_s": elapsed, "max_active": srv.max_active,
                 "admitted_while_busy": srv.admitted_while_busy, "ticks": srv.ticks,
                 "budget_bytes": budget, "clocks": clk.summary(), "dtype": "f32",
                 "policy": args.serve_policy,
                 "max_active_points": args.serve_cap_points if args.serve_policy == "sjf" else None})
    if plain_rates:
        # the same requests, each alone on the plain complex128 path
        t_plain = sum(r.nx * r.ny * r.steps / plain_rates[r.nx] for r in reqs
                      if r.nx in plain_rates)
        summ["served_over_plain_c128"] = (t_plain / elapsed
                                          if all(r.nx in plain_rates for r in reqs) else None)
    if check:
        checks = S.fp64_check(results, stream=stream.cuda_stream, short_steps=200,
                              reference=oracle_reference(512))
        summ["fp64_check"] = {
            "requests": len(checks),
            "max_short_rel_l2": max((c["short_rel_l2"] for c in checks), default=None),
            "max_rel_l2": max((c["rel_l2"] for c in checks), default=None),
            "max_err_vs_initial_norm": max((c["err_vs_initial_norm"] for c in checks),
                                           default=None),
            "min_kept_norm": min((c["kept_norm"] for c in checks), default=None),
            "checks": [{k: c[k] for k in ("n", "steps", "rel_l2", "err_vs_initial_norm",
                                          "kept_norm", "short_steps", "short_rel_l2",
                                          "short_kept_norm", "short_reference")}
                       for c in checks]}
    return summ


def run_serve(args):
    """The serving record as a line of its own (--workload serve): the configured rate
    (200/s) over --serve-seconds and a sustainable rate over --sustainable-seconds."""
    import torch

    world, rank, local = dist_setup(args)
    if rank != 0:  # one request stream, served by rank 0's GPU; other ranks have no work
        return 0
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    out = {"configured": serve_record(args, stream, 200.0, args.serve_seconds),
           "sustainable": serve_record(args, stream, args.sustainable_rate,
                                       args.sustainable_seconds)}
    line = {
        "metric": "p50/p99 solve ms and grid-point*steps/s (serving)",
        "value": out["configured"]["throughput"], "unit": UNIT, "n_gpus": 1,
        "steps": None, "warmup": 0, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "serve-graphene", "arrivals": "Poisson",
                   "sizes": list(W.SERVE_SIZES), "steps": [500, 5000],
                   "steps_per_tick": args.tick},
        "clocks": out["configured"]["clocks"],
        "serving": out,
    }
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="large-4096")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-solves", type=int, default=3)
    ap.add_argument("--batch-count", type=int, default=256)
    ap.add_argument("--tick", type=int, default=32)
    ap.add_argument("--serve-seconds", type=float, default=2.0)
    ap.add_argument("--batch-steps", type=int, default=2000,
                    help="steps per instance of the default line's batch-mix record")
    ap.add_argument("--record-serve-seconds", type=float, default=0.5,
                    help="arrival window of the default line's serving record")
    ap.add_argument("--no-records", action="store_true",
                    help="default line without its batch-mix and serving records")
    ap.add_argument("--profile-region", action="store_true",
                    help="cudaProfilerStart/Stop around the timed region (for ncu "
                         "--profile-from-start off)")
    ap.add_argument("--check-steps", type=int, default=5,
                    help="steps of the default line's rel-L2 check against the oracle")
    ap.add_argument("--serve-policy", default="sjf", choices=["fifo", "sjf"],
                    help="admission order of the serving loop: arrival order, or the least "
                         "work first under a cap on the active grid points")
    ap.add_argument("--serve-cap-points", type=int, default=16 << 20,
                    help="sjf: most grid points of the requests running at once")
    ap.add_argument("--sustainable-rate", type=float, default=4.0)
    ap.add_argument("--sustainable-seconds", type=float, default=20.0)
    ap.add_argument("--scheme", default="printed",
                    choices=["printed", "symmetric", "taylor", "chebyshev", "cn"],
                    help="Scheme II (printed x, y or symmetric x/2, y, x/2 order), the "
                         "polynomial scheme with a Taylor or Chebyshev middle step, or "
                         "Scheme I (Crank-Nicolson, GMRES)")
    ap.add_argument("--poly-degree", type=int, default=8)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args, args.workload)
    if args.workload == "batch-mix":
        return run_batch(args)
    if args.workload == "serve":
        return run_serve(args)

    import torch

    import paper_1909_02894_gb300 as D

    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    w, prec_name, bytes_pt = workload(args.workload)
    prec = D.DIRAC_C64 if prec_name == "c64" else D.DIRAC_C128
    symmetric = args.scheme == "symmetric"
    poly = args.scheme in ("taylor", "chebyshev")
    cn = args.scheme == "cn"
    passes = 3 if symmetric else 2
    scheme_id = {"printed": D.DIRAC_SCHEME_II, "symmetric": D.DIRAC_SCHEME_II_SYMMETRIC,
                 "taylor": D.DIRAC_SCHEME_POLY_TAYLOR,
                 "chebyshev": D.DIRAC_SCHEME_POLY_CHEBYSHEV,
                 "cn": D.DIRAC_SCHEME_CRANK_NICOLSON}[args.scheme]
    if symmetric:
        # three sweeps of psi, b - 1 read in each, U^2 once: 124 B (complex64)
        bytes_pt = bytes_pt // 88 * 124
    if poly:
        # per term: x-derivative pass, transpose, y-derivative pass (each a read and a write
        # of a state array), combine (dx, dy, FP64 a1 a2, previous term for Chebyshev,
        # output, accumulator read and write); per step: U^2 on the state, the first copy
        s = bytes_pt // 88 * 16  # bytes of one state point
        term = 6 * s + (2 * s + 16 + (s if args.scheme == "chebyshev" else 0) + s + 2 * s)
        bytes_pt = args.poly_degree * term + 2 * s + 16 + 2 * s
    # A dedicated stream: the default stream's handle is 0, which the ABI reads as
    # "create a private stream", and events must be recorded where the kernels run.
    stream = torch.cuda.Stream()
    sim = D.Simulation(w, precision=prec, stream=stream.cuda_stream, scheme=scheme_id,
                       poly_degree=args.poly_degree if poly else None)
    sim.set_state(w.psi0)
    pts = w.nx * w.ny
    warm = max(3, args.warmup)
    sim.step(warm, w.dt)
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # ---- device-resident timed region
    l0 = D.dirac_launch_count(sim.ctx)
    it0 = D.dirac_krylov_iterations(sim.ctx)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk, ProfileRegion(args.profile_region):
        barrier()
        ev0.record(stream)
        sim.step(args.steps, w.dt)
        ev1.record(stream)
        barrier()
    launches = D.dirac_launch_count(sim.ctx) - l0
    ms = max_over_ranks(ev0.elapsed_time(ev1), world, device="cuda")
    value = whole_job_value(pts, args.steps, world, ms)

    # ---- roofline of the dominant kernel (the fused line pass, 2 launches per step, 3 in
    # the symmetric order; the timed region holds nothing else, so its average launch
    # duration is ms/launches)
    peak, peak_kind = hbm_peak()
    per_launch_s = ms * 1e-3 / max(1, launches)
    alg_bytes_launch = bytes_pt * pts / float(passes)
    achieved = alg_bytes_launch / per_launch_s / 1e9
    if poly:  # many kernels per step: the whole step against the roofline
        achieved = bytes_pt * pts / (ms * 1e-3 / args.steps) / 1e9
    krylov = None
    if cn:  # bytes of the operator applications and Krylov vector work actually done
        s_ = bytes_pt // 88 * 16
        iters = D.dirac_krylov_iterations(sim.ctx) - it0
        apply_b = 6 * s_ + 2 * s_ + 16 + 2 * s_  # passes, combine (dx, dy, a, prev, out)
        per_iter = apply_b + 4 * 3 * s_ + 2 * s_  # G v, two Gram-Schmidt sweeps, norm
        bytes_pt = (iters * per_iter + args.steps * (3 * apply_b + 2 * s_ + 16)) / args.steps
        achieved = bytes_pt * pts / (ms * 1e-3 / args.steps) / 1e9
        krylov = {"arnoldi_steps_per_step": iters / args.steps}
    traffic = None if (symmetric or poly or cn) else ncu_traffic(w.name, prec_name)

    # ---- rel-L2 of the GPU result against the FP64 oracle (full grid, a few steps), and
    # the oracle's own rate on the host cores from the same runs
    check = None
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        k = max(2, args.check_steps)
        cpu, ref = cpu_baseline(w, scheme=args.scheme, degree=args.poly_degree, check_steps=k)
        sim.set_state(w.psi0)
        sim.step(k, w.dt)
        got = sim.get_state()
        check = {"value": W.rel_l2(got, ref), "steps": k, "grid": [w.nx, w.ny],
                 "tolerance": 1e-5 if prec == D.DIRAC_C64 else 1e-11,
                 "against": "FP64 CPU oracle, whole grid, same launch configuration"}

    # ---- end to end through the public API with pinned host buffers
    e2e = None
    if args.e2e_solves > 0:
        host_in = torch.empty((2, w.ny, w.nx), dtype=torch.complex128, pin_memory=True)
        host_in.numpy()[...] = w.psi0
        host_out = torch.empty_like(host_in).pin_memory()
        solve_steps = min(args.steps, w.steps)
        # one untimed solve first, like the warm-up steps of the device-timed region (the
        # GPU has been idle during the host-side oracle run before this)
        D.lib().dirac_set_state(sim.ctx, host_in.data_ptr(), 0)
        sim.step(min(solve_steps, max(args.warmup, 20)), w.dt)
        D.lib().dirac_get_state(sim.ctx, host_out.data_ptr(), 0)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_solves):
            D.lib().dirac_set_state(sim.ctx, host_in.data_ptr(), 0)
            sim.step(solve_steps, w.dt)
            D.lib().dirac_get_state(sim.ctx, host_out.data_ptr(), 0)
        barrier()
        ms_e2e = max_over_ranks((time.perf_counter() - t0) * 1e3, world, device="cuda")
        # each solve copies its initial state in and its final state out once; per time
        # step that is the solve's bytes over its steps
        e2e = {"value": whole_job_value(pts, solve_steps * args.e2e_solves, world, ms_e2e),
               "unit": UNIT,
               "h2d_bytes_per_step": host_in.numel() * 16 / solve_steps,
               "d2h_bytes_per_step": host_out.numel() * 16 / solve_steps,
               "h2d_bytes_per_solve": host_in.numel() * 16,
               "d2h_bytes_per_solve": host_out.numel() * 16,
               "solves": args.e2e_solves, "steps_per_solve": solve_steps,
               "solve": f"set_state(pinned host) + {solve_steps} steps + get_state(pinned host)",
               "warmup": "one untimed solve"}

    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "peak_source": peak_kind,
                "kernel": "whole step (derivative passes, transposes, combines)"
                if (poly or cn) else kernel_name(w, prec_name),
                "algorithmic_bytes_per_point_step": bytes_pt}
    peaks = alu_peaks() if rank == 0 else None
    if prec == D.DIRAC_C128 and not (poly or cn):
        # FP64-bound: algorithmic flops per launch over the average launch duration, against
        # the FP64 FMA rate measured on this device
        fl_pt = fft_flops_per_point_step(w.nx, w.ny)
        tflops = fl_pt * pts / float(passes) / per_launch_s / 1e12
        p64 = peaks["fp64_tflops"] if peaks else FP64_PEAK_TFLOPS
        roofline = {"bound": "alu", "achieved": tflops, "peak": p64,
                    "unit": "TFLOP/s", "frac": tflops / p64, "traffic": None,
                    "peak_source": "measured FP64 FMA rate (dirac_measure_alu_peak)" if peaks
                    else "nominal FP64 (2 FMA per SM per clock, 152 SMs, 2.07 GHz)",
                    "kernel": kernel_name(w, prec_name),
                    "algorithmic_flops_per_point_step": fl_pt,
                    "hbm_frac": achieved / peak}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": warm, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if prec == D.DIRAC_C64 else "f64", "data": "synthetic",
            "config": {"workload": w.name, "precision": prec_name, "grid": [w.nx, w.ny],
                       "scheme": {"printed": "Scheme II (x, y)",
                                  "symmetric": "Scheme II, symmetric x/2-y-x/2",
                                  "taylor": f"polynomial, Taylor degree {args.poly_degree}",
                                  "chebyshev": f"polynomial, Chebyshev degree {args.poly_degree}",
                                  "cn": "Scheme I (Crank-Nicolson, restarted GMRES)",
                                  }[args.scheme],
                       "dt": w.dt, "absorber": w.pml_width_x, "parallelism": "replicas",
                       "l2": "inputs larger than L2 (no flush)"
                       if bytes_pt * pts > L2_BYTES else "working set fits L2"},
            "roofline": roofline,
            "clocks": clk.summary(),
            "gpu_launches": int(launches),
            "e2e": e2e,
            "alu_peaks": peaks,
        }
        if krylov:
            line["krylov"] = krylov
        if check is not None:
            line["rel_l2_vs_oracle"] = check
        if cpu is not None:
            line["cpu_baseline"] = cpu
    sim.close()
    if (rank == 0 and world == 1 and not args.no_records and args.scheme == "printed"
            and args.workload == "large-4096"):
        # the batched/served complex64 throughput against the plain complex128 path, each
        # with its error against the FP64 oracle (a failure is recorded, not fatal)
        try:
            line["batch"] = batch_record(args, stream, args.batch_steps)
        except Exception as e:  # noqa: BLE001
            line["batch"] = {"error": f"{type(e).__name__}: {e}"}
        try:
            rates = dict((int(k), v) for k, v in line["batch"].get(
                "plain_c128_single_instance", {}).get("per_size", {}).items())
            for n in W.SERVE_SIZES:
                if n not in rates:
                    rates[n] = plain_c128_rate(W.serve_instance(n, 100, 1), stream)
            line["serving"] = serve_record(args, stream, 200.0, args.record_serve_seconds,
                                           plain_rates=rates)
        except Exception as e:  # noqa: BLE001
            line["serving"] = {"error": f"{type(e).__name__}: {e}"}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
