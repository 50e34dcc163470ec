#!/usr/bin/env python
"""Throughput of the ray-shooting hot path (GLAMER Part I, arXiv:1312.1128).

Workload (the headline configuration): 1e6 smoothed particles sampled from an
NFW profile (r_s = 0.1, r < 1, equal masses, total 1), smoothing length = 3D
distance to the 32nd neighbour, truncated-Gaussian kernel with q = 3; rays on
a 2048 x 2048 cell-centred grid over [-1, 1]^2; FP32 tree at theta = 0.3.

One step = the whole hot path for one lens: tree build (stage, Morton sort,
topology, moments, big lists) + ray grouping + tree walk for every ray,
producing alpha1, alpha2, kappa, gamma1, gamma2; the shoot is issued on a
second stream, so the ray grouping runs beside the end of the build and the
walk waits for the build on the device.  `value` is rays per second over the
whole job with inputs resident in HBM; `e2e` is the same through the public
API with host buffers (pinned H2D of particles and rays, D2H of the five
outputs inside the timed region).

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

# FP32 flops per interaction as the kernels evaluate them now (FADD/FMUL =
# 1, FFMA = 2, MUFU = 1; comparisons and selects 0; a packed FFMA2 counts as
# its two FFMAs), term by term:
#   far cell (cell_terms): w 2, r^2 3, 1/r^2 1, u = 1/w 2, u^2 5, u^3 6,
#     alpha 12, u^4 5, 3 Q2 2, gamma 12 = 50 (alpha only: 31);
#   leaf point (point_terms + radial): w 2, r^2 3, 1/r^2, kb, D 3, radial 14
#     = 22 (alpha only: 11);
#   leaf Gaussian inside its support (gauss_terms + radial): w 2, r^2 3, u 1,
#     1/r^2 1, e^-u 2, h1 and g 4, m c / N_q 2, kb, kappa, D 4, radial 14 = 33
#     (alpha only: 19);
#   big-list correction (gauss_correction_x2, per entry and ray): w 2, w_y^2
#     1, r^2 2, t 1, 2^-t 1, 1/r^2 1, -dkb 3, alpha 4, kappa 2, P 2, gamma1 3,
#     w_x w_y 1, gamma2 2 = 26 (alpha only: 15).
FLOPS = {"far_cells": 50, "near_point": 22, "near_full": 33, "big_corrections": 26}
# the same interactions when only alpha is accumulated (LENS_ALPHA_ONLY)
FLOPS_ALPHA = {"far_cells": 31, "near_point": 11, "near_full": 19, "big_corrections": 15}
# the adjoint's per-interaction work for alpha gradients, as backward.cu
# writes it: a far cell's dL/dM, dL/dQ2, dL/dz_cm over the group's rays (w 2,
# 1/r^2 4, u 2, u^2 5, u^3 6, u^4 5, dL/dM 4, dL/dQ2 8, dL/dz_cm 20 = 56);
# a particle term's forward value plus its gradient update (term_grad: G.w
# 3, c2 s2 5, gamma 2, m 2, size 2, position 10 = 24): point 8 + 24,
# Gaussian 19 + 24, big-list correction 14 + 24
FLOPS_ADJOINT = {"far_cells": 56, "near_point": 32, "near_full": 43, "big_corrections": 38}
# the survey's nominal table (written before the kernels existed), reported
# beside the kernel's own counts for the headline workload
FLOPS_NOMINAL = {"far_cells": 46, "near_point": 20, "near_full": 32, "big_corrections": 35}


# the potential walk's interactions (psi.cu, potential.cuh) counted the same
# way: a far cell's M ln|w| - Re(Q2/2w^2) with its deflection (46), a
# point's m ln r with its deflection (15), a truncated Gaussian's potential
# inside its support with the Ein series as a 20-term Horner polynomial (68),
# a big-list entry's (full - softened point) with Ein as u p(u - 9/4), p of
# degree 9 (q <= 3) (56; 77 with the 20-term series it replaced)
FLOPS_PSI = {"far_cells": 46, "near_point": 15, "near_full": 68, "big_corrections": 56}


WALK_SOURCES = ("walk.cu", "walk_dev.cuh", "profiles.cuh")


def side_stream(wl):
    """A second stream for a workload's shooting call, ordered after the work
    already queued on the current stream (the L2 flush, the inputs).  Taken
    before the build, it lets the shoot's ray grouping run beside the end of
    the build, which stays on the current stream; the walk waits for the
    build on the device."""
    import torch
    if not getattr(wl, "overlap", True):
        return torch.cuda.current_stream()
    side = wl.__dict__.setdefault("side", torch.cuda.Stream())
    side.wait_stream(torch.cuda.current_stream())
    return side


def join(side):
    import torch
    torch.cuda.current_stream().wait_stream(side)


def rays_h2d(torch, side, dst, src):
    """Copy the rays to the device on a second stream, beside the particles'
    copy and the build on the current stream."""
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for d, h in zip(dst, src):
            d.copy_(h, non_blocking=True)


def walk_traffic():
    """DRAM bytes per walk launch from the committed ncu capture, if the walk
    source is unchanged since it was taken."""
    p = os.path.join(ROOT, "profiles", "walk_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    return d.get("bytes_per_launch") if d.get("walk_src_sha256_16") == walk_src_hash() else None


def walk_src_hash(names=None):
    """First 16 hex digits of the SHA-256 of a kernel's sources (default: the
    walk's)."""
    h = hashlib.sha256()
    for name in names or WALK_SOURCES:
        with open(os.path.join(ROOT, "paper_1312_1128_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


PSI_SOURCES = ("psi.cu", "potential.cuh", "walk_dev.cuh", "profiles.cuh")


def psi_traffic():
    """DRAM bytes per potential-walk launch from the committed ncu capture, if
    its sources are unchanged since it was taken."""
    p = os.path.join(ROOT, "profiles", "psi_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    return d.get("bytes_per_launch") if d.get("psi_src_sha256_16") == walk_src_hash(PSI_SOURCES) else None


def refine_traffic():
    """DRAM bytes per refinement step (the k_refine launch) from the committed ncu
    capture, if refine.cu is unchanged since it was taken."""
    p = os.path.join(ROOT, "profiles", "refine_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    return d.get("bytes_per_step") if d.get("refine_src_sha256_16") == walk_src_hash(("refine.cu",)) else None


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
        # wait (5 s at most) for the first sample: nvidia-smi's start-up,
        # which loads the management library and queries the driver, would
        # otherwise land in the timed region and delay the host side of
        # short steps
        self.first = []
        if self.p is not None:
            import select
            ready, _, _ = select.select([self.p.stdout], [], [], 5.0)
            if ready:
                line = self.p.stdout.readline()
                if line:
                    self.first.append(line)

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        out, _ = self.p.communicate(timeout=10)
        out = "".join(self.first) + out
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


def replica_rate(ws, units_per_rank: int, ms_local: float, device=None):
    """Whole-job rate of independent replicas: every rank processes
    units_per_rank units; the job takes as long as the slowest rank.
    Returns (max ms over ranks, units of all ranks per second)."""
    ms = max_over_ranks(ws, ms_local, device)
    return ms, ws * units_per_rank / (ms * 1e-3)


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


def run_reference(args, ws, rank):
    if rank != 0:
        return
    wl = WORKLOADS[args.workload]()
    n_rays = wl.n_rays
    unit = getattr(wl, "unit", UNIT)
    per_step = 2.0  # seconds of oracle work per step
    for _ in range(args.warmup):
        wl.oracle_rate(0.5)
    samples, t_all, cores = 0, 0.0, None
    for k in range(args.steps):
        r, done, dt, cores = wl.oracle_rate(per_step, seed=100 + k)
        samples += done
        t_all += dt
    value = samples / t_all
    line = {"impl": "reference", "metric": getattr(wl, "metric", METRIC), "value": value,
            "unit": unit, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * n_rays / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": wl.config(ws),
            "cpu_baseline": {"value": value, "unit": unit, "cores": cores, "kind": "oracle",
                             "sample": f"{samples} " + getattr(wl, "oracle_desc",
                                       "random rays of the workload, FP64 direct sum over every lens "
                                       "component (the tree's theta -> 0 limit)") + f", {per_step:.0f} s per step"},
            "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------- workloads

class Workload:
    """One benchmark workload: inputs, one timed step, its end-to-end form."""
    name = ""
    theta = THETA
    dtype = "f32"
    graph = False
    tile = "default"

    def extra(self):
        return {}

    def flops_per_ray(self):
        with open(os.path.join(ROOT, "tests", "golden", "useful_counts.json")) as f:
            c = json.load(f)[self.name][str(self.theta)]
        return sum(self.FLOPS[k] * c[k] for k in self.FLOPS)


class NfwSph(Workload):
    """Headline: 1e6 smoothed NFW particles, 2048^2 grid, theta 0.3; step =
    tree build + ray grouping + walk."""
    name = WORKLOAD
    FLOPS = FLOPS
    FLOPS_NOMINAL = FLOPS_NOMINAL

    def __init__(self, grid=2048):
        self.w = lensgen.workload_nfw_sph(n_grid=grid)
        self.n_rays = self.w["rx"].size

    def config(self, ws):
        return bench_config(ws)

    def prepare(self, L, torch, dev):
        w = self.w
        self.L = L
        self.parts = torch.from_numpy(w["gauss"]).to(dev)
        self.rx, self.ry = torch.from_numpy(w["rx"]).to(dev), torch.from_numpy(w["ry"]).to(dev)
        self.outs = [torch.empty(self.n_rays, dtype=torch.float32, device=dev) for _ in range(5)]
        self.group = 32
        self.walk = "default"
        # pinned host buffers of the end-to-end form, allocated outside any timing
        self.h = [torch.from_numpy(w["gauss"]).pin_memory(), torch.from_numpy(w["rx"]).pin_memory(),
                  torch.from_numpy(w["ry"]).pin_memory()]
        self.d = [torch.empty_like(x, device=dev) for x in self.h]
        self.hout = [torch.empty(self.n_rays, dtype=torch.float32).pin_memory() for _ in range(5)]

    def tune(self):
        lens = self.L.Lens([self.L.Species.gauss(self.parts, self.w["q"])], theta=self.theta)
        self.group = lens.autotune(self.rx, self.ry)
        self.walk = lens.info()["walk"]
        self.tile = lens.info()["tile"]
        lens.close()

    def step(self, flags):
        side = side_stream(self)
        lens = self.L.Lens([self.L.Species.gauss(self.parts, self.w["q"])], theta=self.theta,
                           group_rays=self.group, walk=self.walk, tile=self.tile)
        lens.shoot(self.rx, self.ry, flags=flags, out=self.outs, stream=side)
        join(side)
        return lens

    def e2e(self, torch, dev):
        """Host buffers: H2D of the particles, and of the rays on a second
        stream beside the build, where the shoot follows (its grouping
        beside the end of the build); the walk writes the five outputs
        straight into page-locked host memory (they cross to the host inside
        the timed region)."""
        w, L = self.w, self.L
        side = self.__dict__.setdefault("side", torch.cuda.Stream())
        rays_h2d(torch, side, self.d[1:], self.h[1:])
        self.d[0].copy_(self.h[0], non_blocking=True)
        lens = L.Lens([L.Species.gauss(self.d[0], w["q"])], theta=self.theta, group_rays=self.group,
                      walk=self.walk, tile=self.tile)
        lens.shoot(self.d[1], self.d[2], out=self.hout, stream=side)
        join(side)
        return lens, sum(x.numel() * 4 for x in self.h), 5 * self.n_rays * 4

    def oracle_rate(self, budget, seed=7):
        import oracle
        w = self.w
        p = w["gauss"].astype(np.float64)
        comps = oracle.make_components(oracle.GAUSS, p[:, 0], p[:, 1], p[:, 2], p[:, 3], w["q"])
        return _oracle_loop(oracle, comps, w["rx"], w["ry"], None, budget, seed)

    def direct_forms(self, torch, dev, fp64_peak):
        """The plain direct-sum forms of this lens on the GPU, FP64 and FP32,
        on 4,096 sampled grid rays (every particle for every ray, the tree's
        theta -> 0 limit): rays/s beside the tree's, and the FP64 form's
        fraction of the measured FP64 peak.  Direct flops per ray: a
        Gaussian inside its support 33, a point mass outside 22 (the walk's
        table), with the support count per ray from the paper tree's big-list
        corrections (every particle whose support covers the ray)."""
        L, w = self.L, self.w
        idx = lensgen.sample_indices(lensgen.rng(4246), self.n_rays, 4096)
        with open(os.path.join(ROOT, "tests", "golden", "useful_counts.json")) as f:
            inside = json.load(f)[WORKLOAD][str(self.theta)]["big_corrections"]
        n = w["gauss"].shape[0]
        fpr = inside * FLOPS["near_full"] + (n - inside) * FLOPS["near_point"]
        out = {}
        for prec, dt in (("fp64", torch.float64), ("fp32", torch.float32)):
            lens = L.Lens([L.Species.gauss(self.parts.to(dt), w["q"])], theta=self.theta, precision=prec)
            dx = torch.from_numpy(w["rx"][idx]).to(dev).to(dt)
            dy = torch.from_numpy(w["ry"][idx]).to(dev).to(dt)
            ms = []
            for _ in range(4):
                lens.shoot(dx, dy, flags=L.DIRECT | L.TIMING)
                ms.append(lens.last_timing()[1])
            lens.close()
            t = float(np.median(ms[1:]))
            peak = fp64_peak if prec == "fp64" else None
            out[prec] = {"rays_per_s": 4096 / (t * 1e-3), "walk_ms": t, "rays": 4096,
                         "interactions_per_s": 4096 * n / (t * 1e-3),
                         "achieved_tflops": fpr * 4096 / (t * 1e-3) / 1e12,
                         **({"fp64_peak_tflops": peak / 1e12, "frac_of_fp64_peak": fpr * 4096 / (t * 1e-3) / peak}
                            if peak else {}),
                         "error": "exact sum: FP64 within 1e-12, FP32 within 1e-5 or 8 roundings of sum |term|"}
        out["flops_per_ray"] = fpr
        return out

    def cpu_other(self, budget=4.0):
        """The oracle's direct sum on one core, and the oracle's paper tree
        (Sec. 3.2, per-ray walk, OpenMP) on all cores, on bounded samples."""
        import oracle
        w = self.w
        p = w["gauss"].astype(np.float64)
        comps = oracle.make_components(oracle.GAUSS, p[:, 0], p[:, 1], p[:, 2], p[:, 3], w["q"])
        r1, n1, dt1, _ = _oracle_loop(oracle, comps, w["rx"], w["ry"], None, budget, 11, nthreads=1)
        t0 = time.perf_counter()
        tree = oracle.PaperTree(comps, 5, self.theta)
        tb = time.perf_counter() - t0
        idx = lensgen.rng(12).permutation(w["rx"].size)[:max(64, int(budget * 1500))]
        t0 = time.perf_counter()
        tree.eval(w["rx"][idx].astype(np.float64), w["ry"][idx].astype(np.float64))
        te = time.perf_counter() - t0
        return {"oracle_direct_1core": {"value": r1, "unit": UNIT, "cores": 1,
                                        "sample": f"{n1} random rays, {dt1:.1f} s"},
                "oracle_paper_tree": {"value": idx.size / te, "unit": UNIT, "cores": oracle.max_threads(),
                                      "build_s": tb, "theta": self.theta,
                                      "sample": f"{idx.size} random rays, {te:.1f} s (build excluded)"}}


class Potential(NfwSph):
    """The headline's lens (1e6 smoothed NFW particles, 2048^2 grid, theta
    0.3) shooting the lensing potential with the deflection (Eq. alpha, Eq.
    timedelay); step = tree build + ray grouping + potential walk."""
    name = "potential_nfw_sph_1e6_2048sq"
    FLOPS = FLOPS_PSI
    metric = "rays/sec (psi + alpha) at stated error"
    oracle_desc = ("random rays of the workload, FP64 direct potential and deflection over every lens "
                   "component (the tree's theta -> 0 limit)")

    def flops_per_ray(self):
        # the potential walk visits the same cells, leaves and big lists as
        # the headline's walk over the same tree
        with open(os.path.join(ROOT, "tests", "golden", "useful_counts.json")) as f:
            c = json.load(f)[WORKLOAD][str(self.theta)]
        return sum(self.FLOPS[k] * c[k] for k in self.FLOPS)

    def config(self, ws):
        return {**bench_config(ws), "workload": self.name, "outputs": "psi, alpha1, alpha2"}

    def prepare(self, L, torch, dev):
        super().prepare(L, torch, dev)
        self.outs = self.outs[:3]
        self.hout = self.hout[:3]

    def tune(self):
        """Group size by the potential walk's own time (32 or 64 rays)."""
        best = None
        for g in (32, 64):
            lens = self.L.Lens([self.L.Species.gauss(self.parts, self.w["q"])], theta=self.theta, group_rays=g)
            t = []
            for _ in range(3):
                lens.potential(self.rx, self.ry, flags=self.L.TIMING, out=self.outs)
                t.append(lens.last_timing()[1])
            lens.close()
            if best is None or min(t) < best[0]:
                best = (min(t), g)
        self.group = best[1]
        self.walk = "warp"

    def step(self, flags):
        side = side_stream(self)
        lens = self.L.Lens([self.L.Species.gauss(self.parts, self.w["q"])], theta=self.theta,
                           group_rays=self.group)
        lens.potential(self.rx, self.ry, flags=flags, out=self.outs, stream=side)
        join(side)
        return lens

    def e2e(self, torch, dev):
        """Host buffers: H2D of the particles, and of the rays on a second
        stream beside the build; psi, alpha1, alpha2 written straight into
        page-locked host memory."""
        w, L = self.w, self.L
        side = self.__dict__.setdefault("side", torch.cuda.Stream())
        rays_h2d(torch, side, self.d[1:], self.h[1:])
        self.d[0].copy_(self.h[0], non_blocking=True)
        lens = L.Lens([L.Species.gauss(self.d[0], w["q"])], theta=self.theta, group_rays=self.group)
        lens.potential(self.d[1], self.d[2], out=self.hout, stream=side)
        join(side)
        return lens, sum(x.numel() * 4 for x in self.h), 3 * self.n_rays * 4

    def oracle_rate(self, budget, seed=7):
        import oracle
        w = self.w
        p = w["gauss"].astype(np.float64)
        comps = oracle.make_components(oracle.GAUSS, p[:, 0], p[:, 1], p[:, 2], p[:, 3], w["q"])
        return _oracle_loop(oracle, comps, w["rx"], w["ry"], None, budget, seed, potential=True)

    def cpu_other(self, budget=4.0):
        return {}


class MixedBatches(Workload):
    """1,000 NFW halos + 1e6 stars; 256 uneven refinement batches (3.7e7
    rays) in one persistent launch replayed as a CUDA graph; the lens is
    built once (an adaptive-refinement loop reuses it), so a step is one
    pass over all batches."""
    name = "mixed_batches_256"
    # NFW leaf inside R_max (nfw_terms: F, f, g with sqrt, log, log1p counted
    # as one operation each, 29, + w, r^2 5 + radial 14 = 48); an NFW big-list
    # correction (the same minus the softened point: 52)
    FLOPS = {"far_cells": 50, "near_point": 22, "near_full": 48, "big_corrections": 52}

    def __init__(self):
        self.w = lensgen.workload_mixed_batches()
        self.n_rays = int(self.w["offsets"][-1])

    def config(self, ws):
        return {"workload": self.name, "n_halos": 1000, "n_stars": 1_000_000, "n_batches": 256,
                "rays": self.n_rays, "theta": self.theta, "leaf_max": 5,
                "l2": "flushed between timed steps (256 MB write)", "graph": "CUDA graph replay",
                "parallelism": f"independent replicas x{ws}"}

    def prepare(self, L, torch, dev):
        w = self.w
        self.L = L
        self.sp = [torch.from_numpy(w["points"]).to(dev), torch.from_numpy(w["nfw"]).to(dev)]
        self.dx, self.dy = torch.from_numpy(w["dx"]).to(dev), torch.from_numpy(w["dy"]).to(dev)
        self.outs = [torch.empty(self.n_rays, dtype=torch.float32, device=dev) for _ in range(5)]
        self.lens = L.Lens([L.Species.points(self.sp[0]), L.Species.nfw(self.sp[1], w["conc"])],
                           theta=self.theta)
        self.lens.reserve(self.n_rays, 256)
        self.group = 32
        self.walk = "default"
        self.h = [torch.from_numpy(w["dx"]).pin_memory(), torch.from_numpy(w["dy"]).pin_memory()]
        self.hout = [torch.empty(self.n_rays, dtype=torch.float32).pin_memory() for _ in range(5)]

    graph = True  # timed by the caller's events (a replayed graph records no internal events)

    def tune(self):
        """Group size and walk form by the time of one replay of all 256
        batches (lens_autotune times one batch, which does not represent
        uneven batches in one launch)."""
        import torch
        L, w = self.L, self.w
        best = None
        for g, walk, tile in [(32, "warp", "standard"), (64, "warp", "standard"), (32, "pairs", "standard"),
                              (64, "pairs", "standard"), (64, "trios", "standard"), (32, "warp", "large"),
                              (64, "warp", "large"), (128, "warp", "standard")]:
            lens = L.Lens([L.Species.points(self.sp[0]), L.Species.nfw(self.sp[1], w["conc"])], theta=self.theta,
                          group_rays=g, walk=walk, tile=tile)
            lens.reserve(self.n_rays, 256)
            t = []
            for _ in range(3):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                lens.shoot_batches(w["offsets"], w["origins"], self.dx, self.dy, flags=L.USE_GRAPH, out=self.outs)
                b.record()
                torch.cuda.synchronize()
                t.append(a.elapsed_time(b))
            lens.close()
            if best is None or min(t[1:]) < best[0]:
                best = (min(t[1:]), g, walk, tile)
        _, self.group, self.walk, self.tile = best
        self.lens.close()
        self.lens = L.Lens([L.Species.points(self.sp[0]), L.Species.nfw(self.sp[1], w["conc"])], theta=self.theta,
                           group_rays=self.group, walk=self.walk, tile=self.tile)
        self.lens.reserve(self.n_rays, 256)

    def step(self, flags):
        # LENS_TIMING does not combine with graph replay; COUNT does (own graph)
        self.lens.shoot_batches(self.w["offsets"], self.w["origins"], self.dx, self.dy,
                                flags=(flags & ~self.L.TIMING) | self.L.USE_GRAPH, out=self.outs)
        return None

    def e2e(self, torch, dev):
        w = self.w
        self.dx.copy_(self.h[0], non_blocking=True)
        self.dy.copy_(self.h[1], non_blocking=True)
        # (device outputs and one copy each: written straight into host
        # memory, the 780 MB of the 256 batches made this step slower)
        self.lens.shoot_batches(w["offsets"], w["origins"], self.dx, self.dy, flags=self.L.USE_GRAPH,
                                out=self.outs)
        for h, o in zip(self.hout, self.outs):
            h.copy_(o, non_blocking=True)
        return None, 2 * self.n_rays * 4, 5 * self.n_rays * 4

    def oracle_rate(self, budget, seed=7):
        import oracle
        w = self.w
        s, h = w["points"].astype(np.float64), w["nfw"].astype(np.float64)
        comps = oracle.concat(oracle.make_components(oracle.POINT, s[:, 0], s[:, 1], s[:, 2]),
                              oracle.make_components(oracle.NFW, h[:, 0], h[:, 1], h[:, 2], h[:, 3],
                                                     w["conc"] * h[:, 3]))
        b = np.repeat(np.arange(len(w["offsets"]) - 1), np.diff(w["offsets"]))
        rx = w["origins"][b, 0] + w["dx"].astype(np.float64)
        ry = w["origins"][b, 1] + w["dy"].astype(np.float64)
        return _oracle_loop(oracle, comps, rx, ry, None, budget, seed)


class Microlensing(Workload):
    """1e7 stars + SIS; 4096^2 rays over a 1e-6 patch at (0.5, 0) as FP64
    origin + FP32 offsets; theta 0.1; step = build + grouping + walk."""
    name = "microlensing_1e7_4096sq"
    theta = 0.1
    FLOPS = {"far_cells": 50, "near_point": 22}
    SIS_FLOPS = 23  # w 2, r^2 3, sqrt 1, kb 1, kappa 1, D 1, radial 14

    def __init__(self):
        self.w = lensgen.workload_microlensing()
        self.n_rays = self.w["dx"].size

    def flops_per_ray(self):
        return super().flops_per_ray() + self.SIS_FLOPS

    def config(self, ws):
        return {"workload": self.name, "n_stars": 10_000_000, "sis_r_e": 0.5, "grid": 4096,
                "patch": "1e-6 at (0.5, 0)", "theta": self.theta, "leaf_max": 5,
                "l2": "flushed between timed steps (256 MB write)",
                "parallelism": f"independent replicas x{ws}"}

    def prepare(self, L, torch, dev):
        w = self.w
        self.L = L
        self.sp = torch.from_numpy(w["points"]).to(dev)
        self.dx, self.dy = torch.from_numpy(w["dx"]).to(dev), torch.from_numpy(w["dy"]).to(dev)
        self.outs = [torch.empty(self.n_rays, dtype=torch.float32, device=dev) for _ in range(5)]
        self.group = 32
        self.walk = "default"
        self.h = [torch.from_numpy(w["points"]).pin_memory(), torch.from_numpy(w["dx"]).pin_memory(),
                  torch.from_numpy(w["dy"]).pin_memory()]
        self.d = [torch.empty_like(x, device=dev) for x in self.h]
        self.hout = [torch.empty(self.n_rays, dtype=torch.float32).pin_memory() for _ in range(5)]

    def tune(self):
        lens = self.L.Lens([self.L.Species.points(self.sp)], [self.L.Halo.sis(0.0, 0.0, self.w["sis_re"])],
                           theta=self.theta)
        self.group = lens.autotune(self.dx, self.dy, origin=self.w["origin"])
        self.walk = lens.info()["walk"]
        self.tile = lens.info()["tile"]
        lens.close()

    def step(self, flags):
        L = self.L
        side = side_stream(self)
        lens = L.Lens([L.Species.points(self.sp)], [L.Halo.sis(0.0, 0.0, self.w["sis_re"])], theta=self.theta,
                      group_rays=self.group, walk=self.walk, tile=self.tile)
        lens.shoot(self.dx, self.dy, origin=self.w["origin"], flags=flags, out=self.outs, stream=side)
        join(side)
        return lens

    def e2e(self, torch, dev):
        """As the headline's: the rays' copy beside the build, the outputs
        written straight into page-locked host memory."""
        w, L = self.w, self.L
        side = self.__dict__.setdefault("side", torch.cuda.Stream())
        rays_h2d(torch, side, self.d[1:], self.h[1:])
        self.d[0].copy_(self.h[0], non_blocking=True)
        lens = L.Lens([L.Species.points(self.d[0])], [L.Halo.sis(0.0, 0.0, w["sis_re"])], theta=self.theta,
                      group_rays=self.group, walk=self.walk, tile=self.tile)
        lens.shoot(self.d[1], self.d[2], origin=w["origin"], out=self.hout, stream=side)
        join(side)
        return lens, sum(x.numel() * 4 for x in self.h), 5 * self.n_rays * 4

    def oracle_rate(self, budget, seed=7):
        import oracle
        w = self.w
        s = w["points"].astype(np.float64)
        comps = oracle.concat(oracle.make_components(oracle.POINT, s[:, 0], s[:, 1], s[:, 2]),
                              oracle.make_components(oracle.SIS, 0.0, 0.0, 0.0, w["sis_re"]))
        rx = w["origin"][0] + w["dx"].astype(np.float64)
        ry = w["origin"][1] + w["dy"].astype(np.float64)
        return _oracle_loop(oracle, comps, rx, ry, None, budget, seed)


class Fit(Workload):
    """Lens fit: 1e5 Gaussians (r_sm 0.01), 1000^2 grid, theta 0.3; step =
    build + forward alpha (keeping its interaction lists) + adjoint of
    L = sum |alpha - alpha_t|^2 (replaying them).  The adjoint is the
    dominant kernel: the line's roofline describes it, the forward walk's is
    reported beside it."""
    name = "fit_1e5_1000sq"
    FLOPS = FLOPS_ALPHA

    def adjoint_flops_per_ray(self):
        with open(os.path.join(ROOT, "tests", "golden", "useful_counts.json")) as f:
            c = json.load(f)[self.name][str(self.theta)]
        return sum(FLOPS_ADJOINT[k] * c[k] for k in FLOPS_ADJOINT)

    def __init__(self):
        self.w = lensgen.workload_fit()
        self.n_rays = self.w["rx"].size

    def config(self, ws):
        return {"workload": self.name, "n_particles": 100_000, "grid": 1000, "theta": self.theta,
                "loss": "sum |alpha - alpha_t|^2, target masses m exp(0.05 N(0,1))",
                "l2": "flushed between timed steps (256 MB write)",
                "parallelism": f"independent replicas x{ws}"}

    def prepare(self, L, torch, dev):
        w = self.w
        self.L = L
        self.torch = torch
        self.parts = torch.from_numpy(w["gauss"]).to(dev)
        self.rx, self.ry = torch.from_numpy(w["rx"]).to(dev), torch.from_numpy(w["ry"]).to(dev)
        tl = L.Lens([L.Species.gauss(torch.from_numpy(w["target"]).to(dev), w["q"])], theta=self.theta)
        at = tl.shoot(self.rx, self.ry, flags=L.ALPHA_ONLY)
        self.at = [a.clone() for a in at[:2]]
        tl.close()
        self.outs = [torch.empty(self.n_rays, dtype=torch.float32, device=dev) for _ in range(5)]
        self.grad = torch.zeros(self.parts.shape[0], 4, dtype=torch.float32, device=dev)
        self.group = 32
        self.walk = "default"
        self.h = [torch.from_numpy(w["gauss"]).pin_memory(), torch.from_numpy(w["rx"]).pin_memory(),
                  torch.from_numpy(w["ry"]).pin_memory()]
        self.d = [torch.empty_like(x, device=dev) for x in self.h]
        self.hgrad = torch.empty(self.parts.shape[0], 4, dtype=torch.float32).pin_memory()
        self.hloss = torch.empty(1, dtype=torch.float32).pin_memory()
        self.back_ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))

    def tune(self):
        lens = self.L.Lens([self.L.Species.gauss(self.parts, self.w["q"])], theta=self.theta)
        self.group = lens.autotune(self.rx, self.ry)
        self.walk = lens.info()["walk"]
        self.tile = lens.info()["tile"]
        lens.close()

    def step(self, flags):
        L = self.L
        # (one stream: the grouping beside this small build saves less than
        # the cross-stream hand-overs cost)
        lens = L.Lens([L.Species.gauss(self.parts, self.w["q"])], theta=self.theta, group_rays=self.group,
                      walk=self.walk, tile=self.tile)
        lens.shoot(self.rx, self.ry, flags=flags | L.ALPHA_ONLY | L.KEEP_LISTS, out=self.outs)
        g1 = 2 * (self.outs[0] - self.at[0])
        g2 = 2 * (self.outs[1] - self.at[1])
        self.grad.zero_()
        self.back_ev[0].record()
        lens.backward(self.rx, self.ry, g1, g2, grads=[self.grad], flags=L.KEEP_LISTS)
        self.back_ev[1].record()
        return lens

    def extra(self):
        return {"backward_ms": self.back_ev[0].elapsed_time(self.back_ev[1])}

    def e2e(self, torch, dev):
        w, L = self.w, self.L
        for d, h in zip(self.d, self.h):
            d.copy_(h, non_blocking=True)
        lens = L.Lens([L.Species.gauss(self.d[0], w["q"])], theta=self.theta, group_rays=self.group,
                      walk=self.walk, tile=self.tile)
        lens.shoot(self.d[1], self.d[2], flags=L.ALPHA_ONLY | L.KEEP_LISTS, out=self.outs)
        r1, r2 = self.outs[0] - self.at[0], self.outs[1] - self.at[1]
        self.grad.zero_()
        lens.backward(self.d[1], self.d[2], (2 * r1).contiguous(), (2 * r2).contiguous(), grads=[self.grad],
                      flags=L.KEEP_LISTS)
        self.hloss.copy_((r1 * r1 + r2 * r2).sum().reshape(1), non_blocking=True)
        self.hgrad.copy_(self.grad, non_blocking=True)
        return lens, sum(x.numel() * 4 for x in self.h), self.hgrad.numel() * 4 + 4

    def oracle_rate(self, budget, seed=7):
        import oracle
        w = self.w
        p = w["gauss"].astype(np.float64)
        comps = oracle.make_components(oracle.GAUSS, p[:, 0], p[:, 1], p[:, 2], p[:, 3], w["q"])
        return _oracle_loop(oracle, comps, w["rx"], w["ry"], None, budget, seed)

    def cpu_other(self, budget=4.0):
        """The oracle's direct sum on one core, and the oracle's paper tree
        (Sec. 3.2, per-ray walk, OpenMP) on all cores, on bounded samples."""
        import oracle
        w = self.w
        p = w["gauss"].astype(np.float64)
        comps = oracle.make_components(oracle.GAUSS, p[:, 0], p[:, 1], p[:, 2], p[:, 3], w["q"])
        r1, n1, dt1, _ = _oracle_loop(oracle, comps, w["rx"], w["ry"], None, budget, 11, nthreads=1)
        t0 = time.perf_counter()
        tree = oracle.PaperTree(comps, 5, self.theta)
        tb = time.perf_counter() - t0
        idx = lensgen.rng(12).permutation(w["rx"].size)[:max(64, int(budget * 1500))]
        t0 = time.perf_counter()
        tree.eval(w["rx"][idx].astype(np.float64), w["ry"][idx].astype(np.float64))
        te = time.perf_counter() - t0
        return {"oracle_direct_1core": {"value": r1, "unit": UNIT, "cores": 1,
                                        "sample": f"{n1} random rays, {dt1:.1f} s"},
                "oracle_paper_tree": {"value": idx.size / te, "unit": UNIT, "cores": oracle.max_threads(),
                                      "build_s": tb, "theta": self.theta,
                                      "sample": f"{idx.size} random rays, {te:.1f} s (build excluded)"}}


class Refine:
    """Sec. 3.4 cell refinement: the 2048^2 grid of a lens of 1,000 NFW halos
    (the batched workload's halo field, smooth at the cell scale away from
    the halo centres) is shot once; a step refines every interior cell into
    3x3 sub-cells with the kappa/gamma uniformity test (tol 1e-4, Eq.
    magmatrix) = lens_refine_cells."""
    name = "refine_2048sq_k3"
    metric = "refined sub-cell rays/sec (Sec. 3.4 linear lens equation)"
    k, tol = 3, 1e-4
    # algorithmic bytes per cell: kappa, gamma1, gamma2, alpha1, alpha2 (FP32,
    # each grid value read once) and the outputs: the flag, A (4 floats) and
    # k^2 source positions (2 doubles each); every interior cell, so the
    # cell list is implicit
    BYTES_PER_CELL = 5 * 4 + 1 + 16 + 3 * 3 * 16

    def __init__(self, grid=2048):
        self.w = lensgen.workload_refine(n_grid=grid)
        self.n = grid
        self.h = self.w["h"]
        self.x0, self.y0 = self.w["x0"], self.w["y0"]
        self.n_cells = (grid - 2) ** 2
        self.n_rays = self.n_cells * self.k * self.k  # sub-cell rays produced per step

    def config(self, ws):
        return {"workload": self.name, "grid": self.n, "cells": self.n_cells, "k": self.k, "tol": self.tol,
                "mode": "kappa/gamma", "patch": "0.03 x 0.03 at (0.3, 0.2)",
                "lens": "1,000 NFW halos (batched workload's field), tree theta 0.3",
                "l2": "flushed between timed steps (256 MB write)",
                "parallelism": f"independent replicas x{ws}"}

    def prepare(self, L, torch, dev):
        w = self.w
        self.L, self.torch = L, torch
        halos = torch.from_numpy(w["nfw"]).to(dev)
        dx, dy = torch.from_numpy(w["dx"]).to(dev), torch.from_numpy(w["dy"]).to(dev)
        lens = L.Lens([L.Species.nfw(halos, w["conc"])], theta=THETA, group_rays=64)
        self.grid = lens.shoot(dx, dy, origin=tuple(w["origin"]))
        lens.sync()
        lens.close()
        j, i = torch.meshgrid(torch.arange(1, self.n - 1, device=dev), torch.arange(1, self.n - 1, device=dev),
                              indexing="ij")
        self.cells = (i + self.n * j).reshape(-1).to(torch.int64).contiguous()
        self.out = (torch.empty(self.n_cells, dtype=torch.uint8, device=dev),
                    torch.empty(self.n_cells, 4, dtype=torch.float32, device=dev),
                    torch.empty(self.n_cells, self.k, self.k, 2, dtype=torch.float64, device=dev))
        self.h_grid = [g.cpu().pin_memory() for g in self.grid]
        self.d_grid = [torch.empty_like(g) for g in self.grid]
        self.h_y = torch.empty(self.out[2].shape, dtype=torch.float64).pin_memory()
        self.h_u = torch.empty(self.n_cells, dtype=torch.uint8).pin_memory()

    def step(self, grid=None):
        g = grid if grid is not None else self.grid
        self.L.refine_cells(self.x0, self.y0, self.h, self.n, self.n, g[0], g[1], g[2], g[3], g[4],
                            cells=None, k=self.k, tol=self.tol, out=self.out)

    def e2e(self):
        for d, hg in zip(self.d_grid, self.h_grid):
            d.copy_(hg, non_blocking=True)
        self.step(self.d_grid)
        self.h_u.copy_(self.out[0], non_blocking=True)
        self.h_y.copy_(self.out[2], non_blocking=True)
        return 5 * self.n * self.n * 4, self.n_cells * (1 + self.k * self.k * 16)

    def oracle_rate(self, budget, seed=7):
        """The refinement oracle (numpy, FP64) on 256 random cells, repeated
        for `budget` seconds; its grid inputs at those cells and their
        neighbours come from the oracle's own direct sum of the lens (input
        preparation, not timed)."""
        import oracle
        import oracle.refine as R
        w = self.w
        n = self.n
        if getattr(self, "_oracle_inputs", None) is None:
            g = lensgen.rng(seed)
            i = g.integers(1, n - 1, 256)
            j = g.integers(1, n - 1, 256)
            cells = (i + n * j).astype(np.int64)
            need = np.unique(np.concatenate([cells, cells + 1, cells - 1, cells + n, cells - n]))
            p = w["nfw"].astype(np.float64)
            comps = oracle.make_components(oracle.NFW, p[:, 0], p[:, 1], p[:, 2], p[:, 3], w["conc"] * p[:, 3])
            vals = oracle.direct_sum(comps, w["origin"][0] + w["dx"][need], w["origin"][1] + w["dy"][need])
            grid = [np.full(n * n, np.nan, np.float32) for _ in range(5)]
            for q in range(5):
                grid[q][need] = vals[:, q]
            self._oracle_inputs = (cells, grid)
        cells, grid = self._oracle_inputs
        done, t0 = 0, time.perf_counter()
        while time.perf_counter() - t0 < budget:
            R.refine_cells(self.x0, self.y0, self.h, n, n, *grid, cells, self.k, self.tol, R.KAPPA_GAMMA)
            done += cells.size
        dt = time.perf_counter() - t0
        return done * self.k * self.k / dt, done * self.k * self.k, dt, 1

    oracle_desc = ("sub-cell rays of 256 random cells (repeated), FP64 numpy refinement oracle on "
                   "oracle-computed grid values")


class Knn:
    """Sec. 3.1 smoothing lengths: the 3D distance to the 32nd nearest
    neighbour of each of the headline's 1e6 NFW particles (the input
    preparation of the smoothed-particle lens, on the device); step =
    lens_smoothing_lengths."""
    name = "smoothing_1e6_k32"
    metric = "smoothing lengths/sec (Sec. 3.1, 3D k = 32 nearest neighbour)"
    unit = "particles/s"
    k = 32
    # algorithmic bytes per particle of this sort-based search: positions in
    # (12) and lengths out (4), keys and indices written (12), 8 radix passes
    # over (key, index) read and written (24 each), the sorted copy (16 in,
    # 16 out)
    BYTES_PER_PARTICLE = 12 + 4 + 12 + 8 * 24 + 32

    def __init__(self, n=1_000_000):
        self.xyz = lensgen.nfw_positions_3d(n, 2)
        self.n_rays = n  # units of the line: particles

    def config(self, ws):
        return {"workload": self.name, "n_particles": self.n_rays, "k": self.k,
                "particles": "3D NFW, r_s = 0.1, r < 1 (the headline's, seed 2)",
                "l2": "flushed between timed steps (256 MB write)",
                "parallelism": f"independent replicas x{ws}"}

    def prepare(self, L, torch, dev):
        self.L = L
        self.d_xyz = torch.from_numpy(self.xyz).to(dev)
        self.r = torch.empty(self.n_rays, dtype=torch.float32, device=dev)
        self.h_xyz = torch.from_numpy(self.xyz).pin_memory()
        self.d2 = torch.empty_like(self.d_xyz)
        self.h_r = torch.empty(self.n_rays, dtype=torch.float32).pin_memory()

    def step(self):
        self.L.smoothing_lengths(self.d_xyz, self.k, out=self.r)

    def e2e(self):
        self.d2.copy_(self.h_xyz, non_blocking=True)
        self.L.smoothing_lengths(self.d2, self.k, out=self.r)
        self.h_r.copy_(self.r, non_blocking=True)
        return self.xyz.nbytes, self.n_rays * 4

    oracle_desc = "particles (every particle of the workload), the oracle's k-d tree search on all host cores"

    def oracle_rate(self, budget, seed=7):
        from oracle import knn
        t0 = time.perf_counter()
        knn.kth_neighbour_distance_tree(self.xyz, self.k)
        dt = time.perf_counter() - t0
        import os as _os
        return self.n_rays / dt, self.n_rays, dt, _os.cpu_count()


class Images:
    """Sec. 4 / Sec. 5.2 image finding: the paper's SIS test -- an SIS of
    r_e = 1, a 64 x 64 initial grid over 20 r_e x 20 r_e, mu_min = 0.01,
    uniform circular sources of radius 0.1, 0.01 and 1e-4 r_e with their
    centres at 0, 0.1, ..., 2 r_e (62 sources: the smallest from 0.1 r_e),
    all images of every source refined until their largest border cell is
    5e-4 of their area; step = one lens_find_images call for all sources."""
    name = "images_sis_62src"
    metric = "sources/sec (all images and magnifications of uniform sources, Sec. 4; SIS test of Sec. 5.2)"
    unit = "sources/s"
    # algorithmic bytes per cell of one image-labelling pass (the dominant
    # kernels): neighbours (leaf fields 21 in, 4 neighbour keys 32, 16 out),
    # union-find (init 9, unite 41, roots 12), the rank scan (8), labels (13),
    # borders (37)
    BYTES_PER_LABEL_CELL = 69 + 9 + 41 + 12 + 8 + 13 + 37
    GRID = dict(x0=-10.0, y0=-10.0, side=20.0, n=64, l_max=12, mu_min=0.01, f_area=5e-4, n_min=50)

    def __init__(self):
        src = []
        for R in (0.1, 0.01, 1e-4):
            for b in np.round(np.linspace(0.0, 2.0, 21), 6):
                if R < 1e-3 and b == 0.0:
                    continue
                src.append((float(b), 0.0, R))
        self.src = np.array(src)
        self.n_rays = len(src)  # units of the line: sources

    def config(self, ws):
        return {"workload": self.name, "lens": "SIS, r_e = 1", "sources": self.n_rays,
                "radii": [0.1, 0.01, 1e-4], "centres": "0 .. 2 r_e in steps of 0.1 (R = 1e-4 from 0.1)",
                "grid": "64 x 64 over 20 r_e x 20 r_e", "mu_min": 0.01, "f_area": 5e-4, "n_min": 50,
                "l_max": 12, "precision": "fp64 deflections",
                "l2": "flushed between timed steps (256 MB write)",
                "parallelism": f"independent replicas x{ws}"}

    def prepare(self, L, torch, dev):
        self.L = L
        self.lens = L.Lens([], [L.Halo.sis(0.0, 0.0, 1.0)], theta=0.3, precision="fp64")
        self.stats = None

    def step(self):
        imgs, self.stats = self.lens.find_images(self.src, max_cells=1 << 26, max_images=1024, **self.GRID)
        self.n_images = len(imgs)
        return imgs

    oracle_desc = ("sources of the workload (R = 0.1 at 1.1, 1.5 and 1.9 r_e, the oracle's fastest: one image "
                   "each), the oracle's pure-Python grid refinement with FP64 deflections from its C direct sum, "
                   "one core")

    def oracle_rate(self, budget, seed=7):
        import oracle
        from oracle import images as I
        comps = oracle.make_components(oracle.SIS, 0.0, 0.0, 0.0, 1.0)

        def alpha(x, y):
            o = oracle.direct_sum(comps, x, y, nthreads=1)
            return o[:, 0], o[:, 1]
        prm = I.AmrParams(**{k: v for k, v in self.GRID.items()})
        sample = [(1.1, 0.0, 0.1), (1.5, 0.0, 0.1), (1.9, 0.0, 0.1)]
        t0 = time.perf_counter()
        done = 0
        while done < 1 or time.perf_counter() - t0 < budget:
            I.find_images(alpha, [sample[done % len(sample)]], prm)
            done += 1
            if done >= 3 * len(sample):
                break
        dt = time.perf_counter() - t0
        return done / dt, done, dt, 1


def run_gpu_images(args, ws, rank, local):
    """The image-finding workload: same timing rules as run_gpu."""
    import torch

    import paper_1312_1128_gb300 as L
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = Images()
    wl.prepare(L, torch, dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    lib = L.lib()
    for _ in range(args.warmup):
        wl.step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    clocks = ClockSampler(local)
    launches0 = lib.lens_kernel_launches()
    label_ms, label_cells, shoot_ms, wall = [], [], [], []
    for k in range(args.steps):
        flush.fill_(k & 0xff)
        torch.cuda.synchronize()
        barrier(ws)
        t0 = time.perf_counter()
        ev[k][0].record()
        wl.step()
        ev[k][1].record()
        torch.cuda.synchronize()
        wall.append(1e3 * (time.perf_counter() - t0))
        label_ms.append(wl.stats["label_ms"])
        label_cells.append(wl.stats["label_cells"])
        shoot_ms.append(wl.stats["shoot_ms"])
    barrier(ws)
    launches = lib.lens_kernel_launches() - launches0
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms, value = replica_rate(ws, wl.n_rays, float(np.mean(step_ms)), dev)
    # the call takes host sources and returns host images: its wall time is
    # the end-to-end figure
    e2e, e2e_value = replica_rate(ws, wl.n_rays, float(np.mean(wall)), dev)
    peak, basis = measured_hbm_gbs()
    achieved = wl.BYTES_PER_LABEL_CELL * float(np.mean(label_cells)) / (float(np.mean(label_ms)) * 1e-3) / 1e9
    st = wl.stats
    line = {"metric": wl.metric, "value": value, "unit": wl.unit, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": wl.config(ws),
            "e2e": {"value": e2e_value, "unit": wl.unit, "h2d_bytes_per_step": int(wl.src.nbytes),
                    "d2h_bytes_per_step": int(wl.n_images * 32)},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "peak_basis": basis,
                         "algorithmic_bytes_per_cell": wl.BYTES_PER_LABEL_CELL,
                         "kernel": "image labelling pass (neighbours, union-find, labels, borders), timed per "
                                   "pass with CUDA events inside the call",
                         "label_ms_per_step": float(np.mean(label_ms)),
                         "label_cells_per_step": float(np.mean(label_cells))},
            "shooting": {"ms_per_step": float(np.mean(shoot_ms)), "rays_per_step": int(st["rays"]),
                         "rays_per_s": st["rays"] / (float(np.mean(shoot_ms)) * 1e-3)},
            "images": wl.n_images, "final_cells": int(st["cells"]), "rounds": int(st["rounds"]),
            "clocks": clk, "gpu_launches": int(launches)}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        r, done_n, dt, cores = wl.oracle_rate(args.cpu_seconds)
        line["cpu_baseline"] = {"value": r, "unit": wl.unit, "cores": cores, "kind": "oracle",
                                "sample": f"{done_n} {wl.oracle_desc}, {dt:.1f} s"}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_gpu_knn(args, ws, rank, local):
    """The smoothing-length workload: same timing rules as run_gpu."""
    import torch

    import paper_1312_1128_gb300 as L
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = Knn()
    wl.prepare(L, torch, dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    lib = L.lib()
    for _ in range(args.warmup):
        wl.step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    clocks = ClockSampler(local)
    launches0 = lib.lens_kernel_launches()
    for k in range(args.steps):
        flush.fill_(k & 0xff)
        torch.cuda.synchronize()
        barrier(ws)
        ev[k][0].record()
        wl.step()
        ev[k][1].record()
        torch.cuda.synchronize()
    barrier(ws)
    launches = lib.lens_kernel_launches() - launches0
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms, value = replica_rate(ws, wl.n_rays, float(np.mean(step_ms)), dev)
    wl.e2e()  # one untimed call first, like the warm-up steps
    torch.cuda.synchronize()
    e2e_ms = []
    for k in range(max(3, args.steps // 2)):
        flush.fill_(k & 0xff)
        torch.cuda.synchronize()
        barrier(ws)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        h2d, d2h = wl.e2e()
        b.record()
        torch.cuda.synchronize()
        e2e_ms.append(a.elapsed_time(b))
    e2e, e2e_value = replica_rate(ws, wl.n_rays, float(np.mean(e2e_ms)), dev)
    peak, basis = measured_hbm_gbs()
    achieved = wl.BYTES_PER_PARTICLE * wl.n_rays / (float(np.mean(step_ms)) * 1e-3) / 1e9
    line = {"metric": wl.metric, "value": value, "unit": "particles/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": wl.config(ws),
            "e2e": {"value": e2e_value, "unit": "particles/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "peak_basis": basis,
                         "algorithmic_bytes_per_particle": wl.BYTES_PER_PARTICLE,
                         "kernels": "bbox, keys, radix sort, gather, query (one call per step)"},
            "clocks": clk, "gpu_launches": int(launches)}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        r, done_n, dt, cores = wl.oracle_rate(args.cpu_seconds)
        line["cpu_baseline"] = {"value": r, "unit": "particles/s", "cores": cores, "kind": "oracle",
                                "sample": f"{done_n} {wl.oracle_desc}, {dt:.1f} s"}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_gpu_refine(args, ws, rank, local):
    """The refinement workload: same timing rules as run_gpu (warm-up, L2
    flush between timed steps, CUDA events, max over ranks, clocks)."""
    import torch

    import paper_1312_1128_gb300 as L
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = Refine()
    wl.prepare(L, torch, dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    lib = L.lib()
    for _ in range(args.warmup):
        wl.step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    clocks = ClockSampler(local)
    launches0 = lib.lens_kernel_launches()
    for k in range(args.steps):
        flush.fill_(k & 0xff)
        torch.cuda.synchronize()
        barrier(ws)
        ev[k][0].record()
        wl.step()
        ev[k][1].record()
        torch.cuda.synchronize()
    barrier(ws)
    launches = lib.lens_kernel_launches() - launches0
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms, value = replica_rate(ws, wl.n_rays, float(np.mean(step_ms)), dev)
    wl.e2e()  # one untimed call first, like the warm-up steps
    torch.cuda.synchronize()
    e2e_ms = []
    for k in range(max(3, args.steps // 2)):
        flush.fill_(k & 0xff)
        torch.cuda.synchronize()
        barrier(ws)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        h2d, d2h = wl.e2e()
        b.record()
        torch.cuda.synchronize()
        e2e_ms.append(a.elapsed_time(b))
    e2e, e2e_value = replica_rate(ws, wl.n_rays, float(np.mean(e2e_ms)), dev)
    peak, basis = measured_hbm_gbs()
    nbytes = wl.BYTES_PER_CELL * wl.n_cells
    achieved = nbytes / (float(np.mean(step_ms)) * 1e-3) / 1e9
    uni = wl.out[0]
    line = {"metric": wl.metric, "value": value,
            "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": wl.config(ws),
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": refine_traffic(), "peak_basis": basis,
                         "algorithmic_bytes_per_cell": wl.BYTES_PER_CELL,
                         "kernels": "k_refine (one launch per step)"},
            "uniform_fraction": float((uni == 1).float().mean().item()),
            "clocks": clk, "gpu_launches": int(launches)}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        r, done_n, dt, cores = wl.oracle_rate(min(args.cpu_seconds, 10.0))
        line["cpu_baseline"] = {"value": r, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"{done_n} {wl.oracle_desc}, {dt:.1f} s"}
    if rank == 0:
        print(json.dumps(line), flush=True)


class PointDiskFp64:
    """The FP64 form (Sec. 5.1's direct-summation comparison; alpha kept in
    higher precision, Sec. 3.4): 2,000 equal point masses in the unit disk,
    a 64 x 64 FP64 grid over [-1.2, 1.2]^2; step = FP64 tree build + the FP64
    direct sum + the FP64 tree walk at theta = 0.1, both for every ray."""
    name = "point_disk_2000_64sq_fp64"
    metric = "rays/sec (alpha+kappa+gamma), FP64 direct sum and FP64 tree at theta = 0.1"
    unit = "rays/s"
    theta = 0.1
    FLOPS_DIRECT = 22     # a point mass's alpha + kappa + gamma (the FP32 table's count)
    FLOPS = {"far_cells": 50, "near_point": 22}

    def __init__(self):
        self.w = lensgen.workload_point_disk()
        self.n_rays = self.w["rx"].size
        self.n = self.w["points"].shape[0]

    def config(self, ws):
        return {"workload": self.name, "n_points": self.n, "grid": 64, "extent": "[-1.2, 1.2]^2",
                "theta": self.theta, "leaf_max": 5, "precision": "fp64 throughout",
                "error": "direct sum within 1e-12 of the FP64 oracle; tree median alpha error <= 1e-4",
                "l2": "flushed between timed steps (256 MB write)",
                "parallelism": f"independent replicas x{ws}"}

    def tree_flops_per_ray(self):
        with open(os.path.join(ROOT, "tests", "golden", "useful_counts.json")) as f:
            c = json.load(f)["point_disk_2000_64sq"][str(self.theta)]
        return sum(self.FLOPS[k] * c[k] for k in self.FLOPS)

    def prepare(self, L, torch, dev):
        w = self.w
        self.L = L
        self.parts = torch.from_numpy(w["points"]).to(dev)
        self.rx, self.ry = torch.from_numpy(w["rx"]).to(dev), torch.from_numpy(w["ry"]).to(dev)
        self.od = [torch.empty(self.n_rays, dtype=torch.float64, device=dev) for _ in range(5)]
        self.ot = [torch.empty(self.n_rays, dtype=torch.float64, device=dev) for _ in range(5)]
        self.h = [torch.from_numpy(w["points"]).pin_memory(), torch.from_numpy(w["rx"]).pin_memory(),
                  torch.from_numpy(w["ry"]).pin_memory()]
        self.d = [torch.empty_like(x, device=dev) for x in self.h]
        self.hout = [torch.empty(self.n_rays, dtype=torch.float64).pin_memory() for _ in range(10)]

    def step(self, flags=0, inputs=None):
        L = self.L
        parts, rx, ry = inputs if inputs is not None else (self.parts, self.rx, self.ry)
        lens = L.Lens([L.Species.points(parts)], theta=self.theta, precision="fp64")
        lens.shoot(rx, ry, flags=flags | L.DIRECT, out=self.od)
        t_direct = lens.last_timing()[1] if flags & L.TIMING else None
        lens.shoot(rx, ry, flags=flags, out=self.ot)
        t_tree = lens.last_timing()[1] if flags & L.TIMING else None
        return lens, t_direct, t_tree

    def e2e(self):
        for d, h in zip(self.d, self.h):
            d.copy_(h, non_blocking=True)
        lens, _, _ = self.step(0, self.d)
        for h, o in zip(self.hout, self.od + self.ot):
            h.copy_(o, non_blocking=True)
        return lens, sum(x.numel() * 8 for x in self.h), 10 * self.n_rays * 8

    oracle_desc = "rays of the grid, FP64 direct sum over every point mass (the oracle), all host cores"

    def oracle_rate(self, budget, seed=7):
        import oracle
        p = self.w["points"]
        comps = oracle.make_components(oracle.POINT, p[:, 0], p[:, 1], p[:, 2])
        return _oracle_loop(oracle, comps, self.w["rx"], self.w["ry"], None, budget, seed)


def run_gpu_fp64(args, ws, rank, local):
    """The FP64 workload: same timing rules as run_gpu (warm-up, L2 flush
    between timed steps, CUDA events, max over ranks, clocks)."""
    import torch

    import paper_1312_1128_gb300 as L
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = PointDiskFp64()
    wl.prepare(L, torch, dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    lib = L.lib()
    for _ in range(args.warmup):
        wl.step(L.TIMING)[0].close()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    clocks = ClockSampler(local)
    launches0 = lib.lens_kernel_launches()
    t_dir, t_tree = [], []
    for k in range(args.steps):
        flush.fill_(k & 0xff)
        torch.cuda.synchronize()
        barrier(ws)
        ev[k][0].record()
        lens, a, b = wl.step(L.TIMING)
        ev[k][1].record()
        torch.cuda.synchronize()
        t_dir.append(a)
        t_tree.append(b)
        lens.close()
    barrier(ws)
    launches = lib.lens_kernel_launches() - launches0
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms, value = replica_rate(ws, wl.n_rays, float(np.mean(step_ms)), dev)
    wl.e2e()[0].close()  # one untimed call first, like the warm-up steps
    torch.cuda.synchronize()
    e2e_ms = []
    for k in range(max(3, args.steps // 2)):
        flush.fill_(k & 0xff)
        torch.cuda.synchronize()
        barrier(ws)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        lens, h2d, d2h = wl.e2e()
        b.record()
        torch.cuda.synchronize()
        lens.close()
        e2e_ms.append(a.elapsed_time(b))
    e2e, e2e_value = replica_rate(ws, wl.n_rays, float(np.mean(e2e_ms)), dev)
    peak64 = L.fp64_peak(256)
    d_ms, tr_ms = float(np.median(t_dir)), float(np.median(t_tree))
    d_flops = wl.n_rays * wl.n * wl.FLOPS_DIRECT
    achieved = d_flops / (d_ms * 1e-3) / 1e12
    tree_fpr = wl.tree_flops_per_ray()
    line = {"metric": wl.metric, "value": value, "unit": wl.unit, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": wl.config(ws),
            "e2e": {"value": e2e_value, "unit": wl.unit, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak64 / 1e12, "unit": "TFLOP/s",
                         "frac": achieved * 1e12 / peak64, "traffic": None,
                         "peak_basis": "measured FP64 DFMA rate (lens_fp64_peak, every SM)",
                         "kernel": "FP64 direct sum (walk_kernel, LENS_DIRECT), CUDA events on its stream",
                         "useful_flops": d_flops, "direct_ms": d_ms},
            "direct": {"ms": d_ms, "rays_per_s": wl.n_rays / (d_ms * 1e-3),
                       "interactions_per_s": wl.n_rays * wl.n / (d_ms * 1e-3)},
            "tree": {"ms": tr_ms, "rays_per_s": wl.n_rays / (tr_ms * 1e-3), "theta": wl.theta,
                     "useful_flops_per_ray": tree_fpr,
                     "achieved_tflops": tree_fpr * wl.n_rays / (tr_ms * 1e-3) / 1e12,
                     "frac_of_fp64_peak": tree_fpr * wl.n_rays / (tr_ms * 1e-3) / peak64},
            "clocks": clk, "gpu_launches": int(launches)}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        r, done_n, dt, cores = wl.oracle_rate(min(args.cpu_seconds, 10.0))
        line["cpu_baseline"] = {"value": r, "unit": wl.unit, "cores": cores, "kind": "oracle",
                                "sample": f"{done_n} {wl.oracle_desc}, {dt:.1f} s"}
    if rank == 0:
        print(json.dumps(line), flush=True)


WORKLOADS = {"nfw_sph": NfwSph, "mixed_batches": MixedBatches, "microlensing": Microlensing, "fit": Fit,
             "refine": Refine, "knn": Knn, "potential": Potential, "images": Images, "point_disk_fp64": PointDiskFp64}


def _oracle_loop(oracle, comps, rx, ry, _, budget_s, seed, nthreads=0, potential=False):
    """The oracle's FP64 direct sum (as it stands) over a time-bounded random
    sample of the workload's rays (nthreads = 0: all host cores); with
    potential, its direct potential and the direct deflection."""
    g = lensgen.rng(seed)
    order = g.permutation(rx.size)
    done, t0, chunk = 0, time.perf_counter(), 64 if nthreads != 1 else 8
    while time.perf_counter() - t0 < budget_s and done < order.size:
        idx = order[done:done + chunk]
        x, y = np.asarray(rx[idx], np.float64), np.asarray(ry[idx], np.float64)
        oracle.direct_sum(comps, x, y, nthreads=nthreads)
        if potential:
            oracle.direct_potential(comps, x, y, nthreads=nthreads)
        done += idx.size
    dt = time.perf_counter() - t0
    return done / dt, done, dt, (oracle.max_threads() if nthreads == 0 else nthreads)


def measured_hbm_gbs():
    """(peak GB/s, basis) from MEASURED_PEAKS.json, else the recipe's fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured copy bandwidth (MEASURED_PEAKS.json)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback 6.8 TB/s"


def grouping_roofline(n_rays, group_ms):
    """Achieved bandwidth of the ray grouping (bounding box, Morton keys, a
    4-pass radix sort of 32-bit keys, group records) against its algorithmic
    bytes per ray: 8 B read for the box, 8 B read + 12 B written for the
    keys, 24 B per sort pass, 12 B read + 12 B written for the sorted rays."""
    nbytes = n_rays * (8 + 20 + 24 * 4 + 24)
    peak, basis = measured_hbm_gbs()
    gbs = nbytes / (group_ms * 1e-3) / 1e9
    return {"ms": group_ms, "algorithmic_bytes": nbytes, "achieved_gbs": gbs, "peak_gbs": peak,
            "frac": gbs / peak, "peak_basis": basis}


def build_roofline(n, n_nodes, phases):
    """Achieved bandwidth of the tree build against the algorithmic bytes:
    per particle 16 B read + 16 B written, 24 B per radix pass (key and index
    read and written; 6 passes of 8 bits over the 48-bit keys), and 48 B per
    node; and of its first phase (staging 32 B, Morton keys 28 B, the six
    sort passes 144 B, the gather 36 B per particle)."""
    build_ms = sum(phases)
    nbytes = n * (32 + 24 * 6) + n_nodes * 48
    sort_bytes = n * (32 + 28 + 24 * 6 + 36)
    peak, basis = measured_hbm_gbs()
    gbs = nbytes / (build_ms * 1e-3) / 1e9
    sgbs = sort_bytes / (phases[0] * 1e-3) / 1e9 if phases[0] > 0 else None
    return {"ms": build_ms, "algorithmic_bytes": nbytes, "achieved_gbs": gbs, "peak_gbs": peak,
            "frac": gbs / peak, "peak_basis": basis,
            "stage_sort": {"ms": phases[0], "algorithmic_bytes": sort_bytes, "achieved_gbs": sgbs,
                           "frac": sgbs / peak if sgbs else None},
            "note": "device time of the build phases (CUDA events on the build's stream), in steps "
                    "that shoot on the build's stream (no grouping beside the build)"}


# ------------------------------------------------------------- GPU path

def run_gpu(args, ws, rank, local):
    import torch

    import paper_1312_1128_gb300 as L
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = WORKLOADS[args.workload]()
    wl.prepare(L, torch, dev)
    n_rays = wl.n_rays
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2
    lib = L.lib()

    def done(lens):
        if lens is not None:
            lens.close()

    wl.tune()   # autotune the ray-group size once (warm-up)
    for _ in range(args.warmup):
        done(wl.step(L.TIMING))
    torch.cuda.synchronize()
    # interaction counters of one step (outside the timed region)
    lens = wl.step(L.COUNT)
    tgt = lens if lens is not None else getattr(wl, "lens", None)
    tgt.sync()
    cnt = tgt.counters()
    done(lens)

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    walk_ms, group_ms, build_phases, build_sizes, extras = [], [], None, None, []
    clocks = ClockSampler(local)
    launches0 = lib.lens_kernel_launches()
    for k in range(args.steps):
        flush.fill_(k & 0xff)  # evict L2 between timed steps
        torch.cuda.synchronize()
        barrier(ws)
        ev[k][0].record()
        lens = wl.step(L.TIMING)
        ev[k][1].record()
        torch.cuda.synchronize()
        if wl.graph:
            g_ms, w_ms = 0.0, ev[k][0].elapsed_time(ev[k][1])  # grouping + walk, one graph
        else:
            g_ms, w_ms = lens.last_timing()
        group_ms.append(g_ms)
        walk_ms.append(w_ms)
        extras.append(wl.extra())
        if lens is not None:
            info = lens.info()
            build_phases = [round(x, 3) for x in info["build_ms"][0]]
            build_sizes = (info["n_particles"][0], info["n_nodes"][0])
        done(lens)
    barrier(ws)
    launches = lib.lens_kernel_launches() - launches0
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms, value = replica_rate(ws, n_rays, float(np.mean(step_ms)), dev)

    # the build's own device time: in the timed steps the shoot's grouping
    # runs beside the build's end, which stretches the build's phases, so
    # take them from steps with the shoot on the build's stream (untimed)
    overlapped_phases = build_phases
    if build_phases is not None:
        wl.overlap = False
        for k in range(3):
            flush.fill_(k & 0xff)
            torch.cuda.synchronize()
            lens = wl.step(L.TIMING)
            torch.cuda.synchronize()
            info = lens.info()
            build_phases = [round(x, 3) for x in info["build_ms"][0]]
            done(lens)
        wl.overlap = True

    # end to end through the public API with host buffers (one untimed call
    # first, like the warm-up steps)
    lens, _, _ = wl.e2e(torch, dev)
    torch.cuda.synchronize()
    done(lens)
    e2e_ms = []
    for k in range(max(3, args.steps // 2)):
        flush.fill_(k & 0xff)
        torch.cuda.synchronize()
        barrier(ws)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        lens, h2d, d2h = wl.e2e(torch, dev)
        b.record()
        torch.cuda.synchronize()
        e2e_ms.append(a.elapsed_time(b))
        done(lens)
    e2e, e2e_value = replica_rate(ws, n_rays, float(np.mean(e2e_ms)), dev)

    direct = None
    if hasattr(wl, "direct_forms"):
        direct = wl.direct_forms(torch, dev, L.fp64_peak(256))

    # roofline of the dominant kernel (the forward walk): useful flops / its duration
    fpr = wl.flops_per_ray()
    nominal_fpr = None
    if getattr(wl, "FLOPS_NOMINAL", None):
        saved = wl.FLOPS
        wl.FLOPS = wl.FLOPS_NOMINAL
        nominal_fpr = wl.flops_per_ray()
        wl.FLOPS = saved
    w_ms = float(np.mean(walk_ms))
    achieved = fpr * n_rays / (w_ms * 1e-3) / 1e12
    props = torch.cuda.get_device_properties(dev)
    sm_max = clk.get("sm_max_mhz") or 2070.0
    peak = props.multi_processor_count * 128 * 2 * sm_max * 1e6 / 1e12
    measured_peak = L.fp32_peak(20000) / 1e12

    line = {"metric": getattr(wl, "metric", METRIC), "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": wl.dtype, "data": "synthetic",
            "config": wl.config(ws), "tuning": {"group_rays": wl.group, "walk": wl.walk, "tile": getattr(wl, "tile", "default")},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak,
                         "traffic": {"nfw_sph": walk_traffic, "potential": psi_traffic}.get(
                             args.workload, lambda: None)(),
                         "peak_basis": f"{props.multi_processor_count} SMs x 128 FP32 lanes x 2 x "
                                       f"{sm_max:.0f} MHz (max SM clock)",
                         "fp32_ffma_measured": measured_peak,
                         "useful_flops_per_ray": fpr, "walk_ms": w_ms,
                         **({"frac_nominal_table": nominal_fpr * n_rays / (w_ms * 1e-3) / 1e12 / peak,
                             "useful_flops_per_ray_nominal_table": nominal_fpr} if nominal_fpr else {}),
                         "group_ms": float(np.mean(group_ms))},
            "build_ms_phases": build_phases,
            "build_ms_phases_beside_grouping": overlapped_phases,
            **({"build": build_roofline(build_sizes[0], build_sizes[1], build_phases)}
               if build_phases and build_sizes else {}),
            "walk_interactions_per_s": cnt["ray_interactions"] / (w_ms * 1e-3),
            **({"grouping": grouping_roofline(n_rays, float(np.mean(group_ms)))}
               if not wl.graph and float(np.mean(group_ms)) > 0 else {}),
            **({k: float(np.mean([e[k] for e in extras])) for k in extras[0]} if extras and extras[0] else {}),
            "interactions": {k: cnt[k] for k in ["groups", "visited", "cells", "leaf_particles",
                                                 "big_scanned", "big_kept", "ray_interactions"]},
            **({"direct_sum_forms": direct} if direct else {}),
            "clocks": clk, "gpu_launches": int(launches)}
    if hasattr(wl, "adjoint_flops_per_ray"):
        # the adjoint dominates this step: its roofline is the line's
        b_ms = line["backward_ms"]
        afpr = wl.adjoint_flops_per_ray()
        a_ach = afpr * n_rays / (b_ms * 1e-3) / 1e12
        line["roofline_forward"] = line["roofline"]
        line["roofline"] = {"bound": "alu", "achieved": a_ach, "peak": peak, "unit": "TFLOP/s",
                            "frac": a_ach / peak, "traffic": None,
                            "peak_basis": line["roofline_forward"]["peak_basis"],
                            "kernel": "lens_shoot_rays_backward (back_kernel + push-down + leaf gradients), "
                                      "timed as a whole",
                            "useful_flops_per_ray": afpr, "backward_ms": b_ms}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        r, done_n, dt, cores = wl.oracle_rate(args.cpu_seconds)
        line["cpu_baseline"] = {"value": r, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"{done_n} " + getattr(wl, "oracle_desc",
                                          "random rays of the workload, FP64 direct sum over every lens "
                                          "component") + f", {dt:.1f} s"}
        if hasattr(wl, "cpu_other") and wl.cpu_other is not None:
            other = wl.cpu_other()
            if other:
                line["cpu_other"] = other
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_once(args):
    """One build + shoot of the headline's lens (profiling: `ncu ... python
    bench.py --once`); with --workload potential, one potential shot; with
    --workload microlensing, one build of the 1e7-star tree (inputs larger
    than L2) and a shot of a --grid^2 patch; with --workload fit, one step of
    the lens fit (build, forward keeping its lists, adjoint replaying them)."""
    import torch

    import paper_1312_1128_gb300 as L
    if args.workload == "fit":
        w = lensgen.workload_fit()
        rx, ry = torch.from_numpy(w["rx"]).cuda(), torch.from_numpy(w["ry"]).cuda()
        tl = L.Lens([L.Species.gauss(torch.from_numpy(w["target"]).cuda(), w["q"])], theta=0.3)
        at = [a.clone() for a in tl.shoot(rx, ry, flags=L.ALPHA_ONLY)[:2]]
        tl.close()
        lens = L.Lens([L.Species.gauss(torch.from_numpy(w["gauss"]).cuda(), w["q"])], theta=0.3, group_rays=32,
                      walk="pairs")
        out = lens.shoot(rx, ry, flags=L.ALPHA_ONLY | L.KEEP_LISTS | L.TIMING)
        lens.sync()
        timing = lens.last_timing()
        ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        ev[0].record()
        lens.backward(rx, ry, (2 * (out[0] - at[0])).contiguous(), (2 * (out[1] - at[1])).contiguous(),
                      flags=L.KEEP_LISTS)
        ev[1].record()
        lens.sync()
        print(json.dumps({"workload": "fit", "timing_ms": timing, "backward_ms": ev[0].elapsed_time(ev[1]),
                          "split_groups": lens.info()["split_groups"]}))
        lens.close()
        return
    if args.workload == "microlensing":
        w = lensgen.workload_microlensing(n_grid=args.grid)
        stars = torch.from_numpy(w["points"]).cuda()
        dx, dy = torch.from_numpy(w["dx"]).cuda(), torch.from_numpy(w["dy"]).cuda()
        lens = L.Lens([L.Species.points(stars)], [L.Halo.sis(0.0, 0.0, w["sis_re"])], theta=0.1, group_rays=64)
        lens.shoot(dx, dy, origin=w["origin"], flags=L.TIMING)
        lens.sync()
        print(json.dumps({"grid": args.grid, "timing_ms": lens.last_timing(), "build_ms": lens.info()["build_ms"][0]}))
        lens.close()
        return
    w = lensgen.workload_nfw_sph(n_grid=args.grid)
    parts = torch.from_numpy(w["gauss"]).cuda()
    rx, ry = torch.from_numpy(w["rx"]).cuda(), torch.from_numpy(w["ry"]).cuda()
    lens = L.Lens([L.Species.gauss(parts, w["q"])], theta=THETA, group_rays=64, walk=args.walk)
    if args.workload == "potential":
        lens.potential(rx, ry, flags=L.TIMING | L.COUNT)
    else:
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
    ap.add_argument("--workload", choices=["nfw_sph", "mixed_batches", "microlensing", "fit", "refine", "knn",
                                           "potential", "images", "point_disk_fp64"],
                    default="nfw_sph",
                    help="nfw_sph (default) is the headline; the others measure the batched, "
                         "microlensing and differentiable paths")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--grid", type=int, default=2048,
                    help="ray grid side (profiling runs use a smaller grid; the metric is quoted at 2048)")
    ap.add_argument("--once", action="store_true",
                    help="one build + shoot of the workload and exit (for profiler captures)")
    ap.add_argument("--walk", choices=["warp", "pairs", "trios"], default="warp",
                    help="walk form of --once (the headline's autotuned choice is warp)")
    ap.add_argument("--print-walk-hash", action="store_true",
                    help="print the hash of the walk sources that profiles/walk_traffic.json is keyed by "
                         "(with --workload potential: of the potential walk's, profiles/psi_traffic.json)")
    args = ap.parse_args()
    if args.print_walk_hash:
        print(walk_src_hash(PSI_SOURCES if args.workload == "potential" else None))
        return
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
        if args.workload == "refine":
            run_gpu_refine(args, ws, rank, local)
        elif args.workload == "knn":
            run_gpu_knn(args, ws, rank, local)
        elif args.workload == "images":
            run_gpu_images(args, ws, rank, local)
        elif args.workload == "point_disk_fp64":
            run_gpu_fp64(args, ws, rank, local)
        else:
            run_gpu(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
