#!/usr/bin/env python
"""Throughput of the ray-shooting hot path (GLAMER Part I, arXiv:1312.1128).

Workload (the headline configuration): 1e6 smoothed particles sampled from an
NFW profile (r_s = 0.1, r < 1, equal masses, total 1), smoothing length = 3D
distance to the 32nd neighbour, truncated-Gaussian kernel with q = 3; rays on
a 2048 x 2048 cell-centred grid over [-1, 1]^2; FP32 tree at theta = 0.3.

One step = the whole hot path for one lens: tree build (stage, Morton sort,
topology, moments, big lists) + ray grouping + tree walk for every ray,
producing alpha1, alpha2, kappa, gamma1, gamma2.  `value` is rays per second
over the whole job with inputs resident in HBM; `e2e` is the same through
the public API with host buffers (pinned H2D of particles and rays, D2H of
the five outputs inside the timed region).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Multi-GPU: one process per GPU (torchrun); each rank builds its own lens and
shoots its own full grid (independent problems, no data-path collective):
weak scaling.  --impl reference times the FP64 CPU oracle instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import lensgen  # noqa: E402

METRIC = "rays/sec (alpha+kappa+gamma) and FP32 interaction-roofline fraction at stated error"
UNIT = "rays/s"
WORKLOAD = "nfw_sph_1e6_2048sq"
THETA = 0.3

# FP32 flops per interaction as the kernels write them (FADD/FMUL = 1,
# FFMA = 2, MUFU = 1), frozen before tuning.
FLOPS = {"far_cells": 50, "near_point": 22, "near_full": 33, "big_corrections": 38}


def useful_flops_per_ray(theta: float) -> float:
    """Paper-tree (per-ray MAC, leaf < 5) interaction counts of this workload
    (tests/golden/useful_counts.json, written from the oracle) x FLOPS."""
    with open(os.path.join(ROOT, "tests", "golden", "useful_counts.json")) as f:
        c = json.load(f)[WORKLOAD][str(theta)]
    return sum(FLOPS[k] * c[k] for k in FLOPS)


def walk_traffic():
    """DRAM bytes per walk launch from the committed ncu capture, if the walk
    source is unchanged since it was taken."""
    p = os.path.join(ROOT, "profiles", "walk_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    src = os.path.join(ROOT, "paper_1312_1128_gb300", "csrc", "walk.cu")
    with open(src, "rb") as f:
        h = hashlib.sha256(f.read()).hexdigest()[:16]
    return d.get("bytes_per_launch") if d.get("walk_cu_sha256_16") == h else None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    def __init__(self, index: int):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-i", str(index), "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        out, _ = self.p.communicate(timeout=10)
        rows = [r.split(",") for r in out.strip().splitlines() if r.strip()]
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for k, name in enumerate(names):
                if len(r) > 5 + k and r[5 + k].strip().lower() == "active":
                    reasons.add(name)
        load = [s for s in sm if s > 0.5 * max(sm)] if sm else []
        return {"sm_mhz": statistics.median(load) if load else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(backend: str):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group(backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, v: float, device=None) -> float:
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------ CPU oracle

def bench_config(ws: int) -> dict:
    return {"workload": WORKLOAD, "n_particles": 1_000_000, "grid": 2048, "theta": THETA,
            "kernel": "gauss q=3, r_sm = 32nd 3D neighbour", "leaf_max": 5,
            "l2": "flushed between timed steps (256 MB write)",
            "parallelism": f"independent replicas x{ws}"}


def oracle_rays_per_sec(w, budget_s: float, seed: int = 7):
    """FP64 direct sum over all particles (the oracle as it stands) on a
    time-bounded random sample of the grid rays."""
    import oracle
    p = w["gauss"].astype(np.float64)
    comps = oracle.make_components(oracle.GAUSS, p[:, 0], p[:, 1], p[:, 2], p[:, 3], w["q"])
    g = lensgen.rng(seed)
    order = g.permutation(w["rx"].size)
    done, t0, chunk = 0, time.perf_counter(), 64
    while time.perf_counter() - t0 < budget_s and done < order.size:
        idx = order[done:done + chunk]
        oracle.direct_sum(comps, w["rx"][idx].astype(np.float64), w["ry"][idx].astype(np.float64))
        done += idx.size
    dt = time.perf_counter() - t0
    return done / dt, done, dt, oracle.max_threads()


def run_reference(args, ws, rank):
    if rank != 0:
        return
    w = lensgen.workload_nfw_sph()
    n_rays = w["rx"].size
    per_step = 2.0  # seconds of oracle work per step
    for _ in range(args.warmup):
        oracle_rays_per_sec(w, 0.5)
    rates, samples = [], 0
    cores = None
    t_all = 0.0
    for k in range(args.steps):
        r, done, dt, cores = oracle_rays_per_sec(w, per_step, seed=100 + k)
        rates.append(r)
        samples += done
        t_all += dt
    value = samples / t_all
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * n_rays / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": bench_config(ws),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{samples} random grid rays of the workload, FP64 direct "
                                       f"sum over all 1e6 particles (the tree's theta -> 0 limit), "
                                       f"{per_step:.0f} s per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------- GPU path

def run_gpu(args, ws, rank, local):
    import torch

    import paper_1312_1128_gb300 as L
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = lensgen.workload_nfw_sph()
    n_rays = w["rx"].size
    parts = torch.from_numpy(w["gauss"]).to(dev)
    rx = torch.from_numpy(w["rx"]).to(dev)
    ry = torch.from_numpy(w["ry"]).to(dev)
    outs = [torch.empty(n_rays, dtype=torch.float32, device=dev) for _ in range(5)]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2
    species = [L.Species.gauss(parts, w["q"])]
    lib = L.lib()

    tuned = {"group_rays": 32}

    def step(flags=L.TIMING):
        lens = L.Lens(species, theta=THETA, group_rays=tuned["group_rays"])
        lens.shoot(rx, ry, flags=flags, out=outs)
        return lens

    # autotune the ray-group size once on this lens and these rays (warm-up)
    lens = L.Lens(species, theta=THETA)
    tuned["group_rays"] = lens.autotune(rx, ry)
    lens.close()
    for _ in range(args.warmup):
        step().close()
    torch.cuda.synchronize()
    # interaction counters of one step (outside the timed region)
    lens = step(L.COUNT)
    lens.sync()
    cnt = lens.counters()
    lens.close()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    walk_ms, group_ms = [], []
    clocks = ClockSampler(local)
    launches0 = lib.lens_kernel_launches()
    for k in range(args.steps):
        flush.fill_(k & 0xff)  # evict L2 between timed steps
        torch.cuda.synchronize()
        barrier(ws)
        ev[k][0].record()
        lens = step()
        ev[k][1].record()
        torch.cuda.synchronize()
        g_ms, w_ms = lens.last_timing()
        group_ms.append(g_ms)
        walk_ms.append(w_ms)
        build_phases = [round(x, 3) for x in lens.info()["build_ms"][0]]
        lens.close()
    barrier(ws)
    launches = lib.lens_kernel_launches() - launches0
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = max_over_ranks(ws, float(np.mean(step_ms)), dev)
    value = ws * n_rays / (ms * 1e-3)

    # end to end through the public API with host buffers
    h_parts = torch.from_numpy(w["gauss"]).pin_memory()
    h_rx = torch.from_numpy(w["rx"]).pin_memory()
    h_ry = torch.from_numpy(w["ry"]).pin_memory()
    h_out = [torch.empty(n_rays, dtype=torch.float32).pin_memory() for _ in range(5)]
    d_parts = torch.empty_like(parts)
    d_rx, d_ry = torch.empty_like(rx), torch.empty_like(ry)
    e2e_ms = []
    for k in range(max(3, args.steps // 2)):
        flush.fill_(k & 0xff)
        torch.cuda.synchronize()
        barrier(ws)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        d_parts.copy_(h_parts, non_blocking=True)
        d_rx.copy_(h_rx, non_blocking=True)
        d_ry.copy_(h_ry, non_blocking=True)
        lens = L.Lens([L.Species.gauss(d_parts, w["q"])], theta=THETA)
        lens.shoot(d_rx, d_ry, out=outs)
        for h, o in zip(h_out, outs):
            h.copy_(o, non_blocking=True)
        b.record()
        torch.cuda.synchronize()
        e2e_ms.append(a.elapsed_time(b))
        lens.close()
    e2e = max_over_ranks(ws, float(np.mean(e2e_ms)), dev)
    h2d = h_parts.numel() * 4 + 2 * n_rays * 4
    d2h = 5 * n_rays * 4

    # roofline of the dominant kernel (the walk): useful flops / its duration
    fpr = useful_flops_per_ray(THETA)
    w_ms = float(np.mean(walk_ms))
    achieved = fpr * n_rays / (w_ms * 1e-3) / 1e12
    props = torch.cuda.get_device_properties(dev)
    sm_max = clk.get("sm_max_mhz") or 2070.0
    peak = props.multi_processor_count * 128 * 2 * sm_max * 1e6 / 1e12
    measured_peak = L.fp32_peak(20000) / 1e12

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": bench_config(ws), "tuning": {"group_rays": tuned["group_rays"]},
            "e2e": {"value": ws * n_rays / (e2e * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": walk_traffic(),
                         "peak_basis": f"{props.multi_processor_count} SMs x 128 FP32 lanes x 2 x "
                                       f"{sm_max:.0f} MHz (max SM clock)",
                         "fp32_ffma_measured": measured_peak,
                         "useful_flops_per_ray": fpr, "walk_ms": w_ms,
                         "group_ms": float(np.mean(group_ms))},
            "build_ms_phases": build_phases,
            "interactions": {k: cnt[k] for k in ["groups", "visited", "cells", "leaf_particles",
                                                 "big_scanned", "big_kept", "ray_interactions"]},
            "clocks": clk, "gpu_launches": int(launches)}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        r, done, dt, cores = oracle_rays_per_sec(w, args.cpu_seconds)
        line["cpu_baseline"] = {"value": r, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"{done} random grid rays of the workload, FP64 direct sum "
                                          f"over all 1e6 particles, {dt:.1f} s"}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_once(args):
    """One build + shoot of the workload (profiling: `ncu ... python bench.py --once`)."""
    import torch

    import paper_1312_1128_gb300 as L
    w = lensgen.workload_nfw_sph(n_grid=args.grid)
    parts = torch.from_numpy(w["gauss"]).cuda()
    rx, ry = torch.from_numpy(w["rx"]).cuda(), torch.from_numpy(w["ry"]).cuda()
    lens = L.Lens([L.Species.gauss(parts, w["q"])], theta=THETA, group_rays=64)
    lens.shoot(rx, ry, flags=L.TIMING | L.COUNT)
    lens.sync()
    print(json.dumps({"grid": args.grid, "timing_ms": lens.last_timing(), "counters": lens.counters(),
                      "build_ms": lens.info()["build_ms"][0]}))
    lens.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--grid", type=int, default=2048,
                    help="ray grid side (profiling runs use a smaller grid; the metric is quoted at 2048)")
    ap.add_argument("--once", action="store_true",
                    help="one build + shoot of the workload and exit (for profiler captures)")
    args = ap.parse_args()
    if args.once:
        run_once(args)
        return
    if args.warmup < 3 and args.impl == "gpu":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        ws, rank, _ = dist_setup("gloo")
        run_reference(args, ws, rank)
    else:
        ws, rank, local = dist_setup("nccl")
        run_gpu(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
