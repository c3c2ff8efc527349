#!/usr/bin/env python
"""Benchmark of the path-calculation hot path on GB300.

One step = the whole hot path over one batch of synthetic input, for each
grid of the workload:
  trace_rays (locate, exit-wall walk, neighbor search, tau, crossing count),
  <N_cross> reduction, emission (scan + fill of cell ids and segment lengths),
  grid density at uniform points with Delta-rho, optical depth along
  uniform-endpoint paths with Delta-tau, and the adjoint scatter.
Grids are built and uploaded before timing; the true densities and optical
depths of the analytic model (the reference values of Delta-rho and
Delta-tau) are computed once before timing.

Default workload: the exponential disk at ~1e6 leaves, octree and k-d tree,
1e6 emission rays each (FP64).  ``value`` = emission rays traced through
both grids per second of whole-step time.

``--impl reference`` times the FP64 CPU oracle on a bounded sample of the
same workload (the comparison arm).  Under torchrun every rank traces its
own rays through replicated grids (weak scaling, no collective on the data
path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "rays/s and Gcell-crossings/s (octree vs k-d tree), % HBM roofline, vs FP64"
UNIT = "rays/s"
# algorithmic bytes of the trace kernel: per crossing 6 FP64 bounds + FP64 density + the exit
# wall's CSR range (2 x int64) + one neighbor id; per ray origin + direction in, tau + count + status out
BYTES_PER_CROSSING = {"fp64": 48 + 8 + 16 + 4, "fp32k": 48 + 4 + 16 + 4}
BYTES_PER_RAY = {"fp64": 48 + 8 + 4 + 1, "fp32k": 48 + 4 + 4 + 1}
# fused into the same walk: the emission staging (cell and ds per crossing, the first entry per ray)
STAGE_BYTES_PER_CROSSING = {"fp64": 4 + 8, "fp32k": 4 + 4}
STAGE_BYTES_PER_RAY = 4
L2_FLUSH_BYTES = 512 << 20
# what bounds the walk besides the copy bandwidth (see DESIGN, GB300-specific choices 1 and 4): random
# gathers of 96-byte records from a 2 GB array sustained 13.2 G records/s (~1.27 TB/s) in a separate probe,
# and FP64 add / fused multiply-add issued 16.5 G warp instructions/s (0.053 per cycle per SM) whether 32,
# 16 or 1 lane was active, i.e. 528 G lane operations/s at full warps; per crossing the walk issues 10 FP64
# instructions (3 wall times of 2 each, 2 fused exit-point coordinates, ds, the fused sum; under FP32-Kahan
# the sum leaves the FP64 pipe and the FP32 cast of ds joins it)
RANDOM_GATHER_GBS = 1.27e3
FP64_OPS_PER_S = 528e9
FP64_OPS_PER_CROSSING = {"fp64": 10, "fp32k": 10}


# ----------------------------------------------------------------------------- distributed plumbing

def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def dist_init(world: int, use_cuda: bool):
    if world <= 1:
        return None
    import torch.distributed as dist
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    dist.init_process_group(backend="nccl" if use_cuda else "gloo")
    return dist


def barrier(dist, device=None):
    if dist is not None:
        if device is not None:
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


def max_over_ranks(dist, x: float, device=None) -> float:
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(dist, x: float, device=None) -> float:
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def rank_seed(seed: int, rank: int) -> int:
    """Independent rays per rank (weak scaling): rank 0 keeps the workload's own seed."""
    return seed + 7919 * rank


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        # the samples go to HG_CLOCKS_DIR when set (to keep them), else to a temporary folder
        out_dir = os.environ.get("HG_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"hg_clocks_rank{gpu_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"], samples=0)
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["no samples"], samples=0)
        return dict(sm_mhz=statistics.median(sm), sm_max_mhz=max(smax), reasons=sorted(reasons), samples=len(sm))


# ----------------------------------------------------------------------------- workloads

def kernel_source_sha() -> str:
    h = hashlib.sha256()
    for f in ("walk.cuh", "trace.cu", "hg_internal.h"):
        h.update(open(os.path.join(ROOT, "paper_1311_0705_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(workload: str, precision: str):
    """DRAM bytes per launch of the trace kernel from the committed ncu summary, if it was
    taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", f"trace_kernel_{workload}_{precision}.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m_sha = re.search(r"kernel_source_sha:\s*([0-9a-f]+)", txt)
    m_b = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    if not m_sha or not m_b or m_sha.group(1) != kernel_source_sha():
        return None
    return float(m_b.group(1))


def make_disk_grids(hg, threads=0):
    grids = []
    for kind in (synth.TREE_OCTREE, synth.TREE_KD):
        model, bp, n_rays, seed = synth.workload_disk_1e6(kind)
        t0 = time.time()
        host = hg.build_grid(model, bp, threads=threads)
        tb = time.time() - t0
        grids.append(dict(name="octree" if kind == 0 else "kd", kind=kind, host=host, build_s=tb))
    return model, grids, n_rays, seed


def make_small_grids(hg, threads=0):
    model, bp, n_rays, seed = synth.workload_disk_small()
    grids = []
    for kind in (synth.TREE_OCTREE, synth.TREE_KD):
        bp.kind = kind
        t0 = time.time()
        host = hg.build_grid(model, bp, threads=threads)
        grids.append(dict(name="octree" if kind == 0 else "kd", kind=kind, host=host, build_s=time.time() - t0))
    return model, grids, n_rays, seed


def make_torus_grid(hg, threads=0):
    model, bp, n_rays, seed = synth.workload_torus_1e7()
    t0 = time.time()
    host = hg.build_grid(model, bp, threads=threads)
    return model, [dict(name="kd", kind=1, host=host, build_s=time.time() - t0)], n_rays, seed



WORKLOADS = {
    "disk-1e6": ("disk, octree (mass 1e-6, max level 12) and k-d tree (same threshold), 1e6 rays per grid",
                 make_disk_grids),
    "disk-1e4": ("disk, octree and k-d tree (mass 1e-4, max level 6), 1e4 rays per grid", make_small_grids),
    "torus-1e7": ("ring torus + 1000 clumps, k-d tree (mass 7e-7, tau 0.5, q 0.9, max level 10, ~9.8e6 leaves), "
                  "1e7 rays: FP32-Kahan and FP64 passes plus the adjoint", make_torus_grid),
    "batch-64": ("64 grids (octree/k-d, disk/ring/clumps, seeded), 1e5-1e7 rays each, one persistent launch",
                 None),
    "interact-1e6": ("disk, octree and k-d tree as disk-1e6; 1e6 photon packets per grid walked to their interaction "
                     "point (tau_int = -ln u), kappa 200 (face-on tau 12, edge-on ~100 at the centre)",
                     make_disk_grids),
    "build-1e6": ("disk-1e6's octree and k-d tree (mass 1e-6, max level 12) built on the GPU: Monte Carlo node "
                  "evaluation (100 draws per node), children and neighbor lists on the device", None),
}
# opacity of the interaction workload: the disk optically thick in its midplane
INTERACT_KAPPA = 200.0
# interaction search: the walk's bytes per crossing as the FP64 trace; per packet 48 B in, tau_int, then cell,
# t, count and status out
INTERACT_BYTES_PER_RAY = 48 + 8 + 4 + 8 + 4 + 1


def matched_kd(hg, model, grids, P, PA, PK, PL, RT, TT):
    """k-d tree with the octree's leaf count (within 5 %) by bisection of the mass threshold, and its
    Delta-rho / Delta-tau on the same points and paths as the timed step."""
    target = next(g for g in grids if g["kind"] == 0)["host"].n_leaves
    _, bp, _, _ = synth.workload_disk_1e6(1)
    lo, hi = math.log(bp.delta_max) - math.log(8.0), math.log(bp.delta_max)
    best = None
    t0 = time.time()
    for _ in range(12):
        dm = math.exp(0.5 * (lo + hi))
        _, bpi, _, _ = synth.workload_disk_1e6(1, delta_max=dm)
        H = hg.build_grid_gpu(model, bpi)
        r = H.n_leaves / target
        if best is None or abs(r - 1) < abs(best[2] - 1):
            best = (dm, H, r)
        if abs(r - 1) <= 0.05:
            break
        if r > 1:
            lo = math.log(dm)
        else:
            hi = math.log(dm)
    dm, H, r = best
    G = hg.load_grid(H)
    _, rg = hg.sample_density(G, P)
    ptau, _, _ = hg.trace_rays(G, PA, PK, PL, kappa=1.0, precision="fp64")
    drho = hg.diff_stats(RT, rg)
    dtau = hg.diff_stats(TT, ptau)
    return dict(delta_max=dm, leaves=H.n_leaves, leaves_over_octree=round(r, 4),
                delta_rho=float(drho[2].item()), delta_tau=float(dtau[2].item()),
                search_s=round(time.time() - t0, 1))


def kd_orientations(hg, torch, model, O, K, P, PA, PK, PL, RT, TT, flush, stream):
    """The disk k-d tree at the step's mass threshold split on the cyclic axis and on the axis of the
    strongest density gradient (Sect. 2.2): leaves, Delta-rho and Delta-tau on the step's points and
    paths, and an optical-depth walk of the step's rays (median of 5, L2 flushed), outside the timed step."""
    res = {}
    for name, axis in (("cyclic", 0), ("gradient", 1)):
        _, bp, _, _ = synth.workload_disk_1e6(1)
        bp.split_axis = axis
        H = hg.build_grid_gpu(model, bp)
        G = hg.load_grid(H)
        _, rg = hg.sample_density(G, P)
        ptau, _, _ = hg.trace_rays(G, PA, PK, PL, kappa=1.0, precision="fp64")
        drho = hg.diff_stats(RT, rg)
        dtau = hg.diff_stats(TT, ptau)
        R = hg.prepare_rays(G, O, K)
        tau, nc, st = R.trace()
        ms = statistics.median(_timed_steps(torch, stream, 5, flush, lambda: R.trace(out=(tau, nc, st))))
        cr = int(nc.sum().item())
        R.free()
        res[name] = dict(leaves=H.n_leaves, delta_rho=float(drho[2].item()), delta_tau=float(dtau[2].item()),
                         walk_ms=ms, mean_ncross=cr / nc.numel(), gcross_per_s=cr / ms / 1e6)
    return res


# ----------------------------------------------------------------------------- our arm

def run_ours(args):
    import torch
    import paper_1311_0705_gb300 as hg

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = dist_init(world, True)
    desc, maker = WORKLOADS[args.workload]
    model, grids, n_rays, seed = maker(hg)
    n_pts = n_rays
    n_paths = max(1, n_rays // 10)
    prec = args.precision
    rs = rank_seed(seed, rank)
    o, k = synth.emission_rays(rs, n_rays)
    pts = synth.sample_points(rs + 1, n_pts)
    pa, pk, pl = synth.endpoint_paths(rs + 2, n_paths)
    w = synth.adjoint_weights(rs + 3, n_rays)
    O, K = torch.tensor(o, device=dev), torch.tensor(k, device=dev)
    P = torch.tensor(pts, device=dev)
    PA, PK, PL = torch.tensor(pa, device=dev), torch.tensor(pk, device=dev), torch.tensor(pl, device=dev)
    W = torch.tensor(w, device=dev)
    dm = hg.load_model(model)
    # reference values of the metrics (the analytic model), computed once
    RT = hg.model_density(dm, P)
    TT = hg.model_tau(dm, PA, PK, PL)
    for g in grids:
        t0 = time.time()
        g["grid"] = hg.load_grid(g["host"], validate=args.validate)
        torch.cuda.synchronize()
        g["load_s"] = time.time() - t0
        n = n_rays
        g["tau"] = torch.empty(n, dtype=torch.float64 if prec == "fp64" else torch.float32, device=dev)
        g["nc"] = torch.empty(n, dtype=torch.int32, device=dev)
        g["st"] = torch.empty(n, dtype=torch.uint8, device=dev)
        g["ptau"] = torch.empty(n_paths, dtype=torch.float64, device=dev)
        g["pnc"] = torch.empty(n_paths, dtype=torch.int32, device=dev)
        g["grad"] = torch.zeros(g["grid"].n_leaves, dtype=torch.float32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    launch = {"min_blocks": args.min_blocks} if args.min_blocks else {}
    kev = []  # (start, end) events around the dominant kernel
    cev = []  # (start, end) events around the emission copy with the adjoint scatter
    gstreams = [torch.cuda.Stream(device=dev) for _ in grids]

    def on_grid_streams(fn):
        # fn(g) for every grid, each on its own stream after the work queued so far; then join
        for gs, g in zip(gstreams, grids):
            gs.wait_stream(stream)
            with torch.cuda.stream(gs):
                fn(g)
        for gs in gstreams:
            stream.wait_stream(gs)

    IN = {"O": O, "K": K}  # the step's input rays (the end-to-end loop alternates two sets)

    def step(record=False, copy_out=None):
        # per grid: one setup (first leaf, work-ordered queue, path segments) for the emission rays;
        # one walk for the optical depth, counts and the staged emission; then the emission copy,
        # which also scatters the adjoint from the staged lengths, and the quality metrics.  The two
        # grids' setups run concurrently on their own streams, the two walks run alone one after
        # the other (so that their event times are theirs), and the rest of each grid runs
        # concurrently again.
        out = {}

        def prep(g):
            g["R"] = hg.prepare_rays(g["grid"], IN["O"], IN["K"], **launch)
            g["grad"].zero_()

        def rest(g):
            G, R = g["grid"], g["R"]
            ncs = hg.sum_i32(g["nc"])
            off = hg.scan_offsets(g["nc"])
            cap = g.get("cap")
            if cap is None:
                cap = g["cap"] = int(off[-1].item())
            gs = torch.cuda.current_stream()
            if record:
                c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                c0.record(gs)
            cell, ds, _ = R.emit_staged_gradient(off, W, kappa=1.0, grad=g["grad"], grad_precision="fp32",
                                                 capacity=cap, status=g["st"])
            g["off"], g["cell"], g["ds"] = off, cell, ds
            if copy_out is not None:
                copy_out(g)
            if record:
                c1.record(gs)
                cev.append((g["name"], c0, c1))
            _, rg = hg.sample_density(G, P)
            drho = hg.diff_stats(RT, rg)
            ptau, _, _ = hg.trace_rays(G, PA, PK, PL, kappa=1.0, precision="fp64", out=(g["ptau"], g["pnc"], None))
            dtau = hg.diff_stats(TT, ptau)
            R.free()
            g["R"] = None
            out[g["name"]] = (ncs, drho, dtau)

        on_grid_streams(prep)
        for g in grids:
            if record:
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
            g["R"].trace_stage(kappa=1.0, precision=prec, out=(g["tau"], g["nc"], g["st"]))
            if record:
                e1.record(stream)
                kev.append((g["name"], e0, e1))
        on_grid_streams(rest)
        return out

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # correctness of the timed configuration: no ray may end in an error state
    for g in grids:
        bits = int(hg.reduce_status(g["st"]).item())
        if bits:
            raise RuntimeError(f"ray status bits {bits} on {g['name']}")

    clocks = ClockSampler(local)
    clocks.start()
    launches0 = hg.launch_count()
    barrier(dist, dev)
    torch.cuda.synchronize()
    step_ms = []
    results = None
    for s in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        results = step(record=True)
        b.record(stream)
        step_ms.append((a, b))
    torch.cuda.synchronize()
    barrier(dist, dev)
    launches = hg.launch_count() - launches0
    clk = clocks.stop()
    times = [a.elapsed_time(b) for a, b in step_ms]
    local_ms = sum(times)
    tot_ms = max_over_ranks(dist, local_ms, dev)
    rays_per_step = n_rays * len(grids)
    all_rays = sum_over_ranks(dist, rays_per_step * args.steps, dev)
    value = all_rays / (tot_ms / 1e3)

    # dominant kernel: the walk for optical depth and staged emission; algorithmic bytes per launch /
    # mean launch time
    per, cper = {}, {}
    for name, e0, e1 in kev:
        per.setdefault(name, []).append(e0.elapsed_time(e1))
    for name, e0, e1 in cev:
        cper.setdefault(name, []).append(e0.elapsed_time(e1))
    kern = {}
    tot_bytes, tot_time = 0.0, 0.0
    for g in grids:
        cr = int(g["nc"].sum().item())
        ms = statistics.mean(per[g["name"]])
        byt = ((BYTES_PER_CROSSING[prec] + STAGE_BYTES_PER_CROSSING[prec]) * cr +
               (BYTES_PER_RAY[prec] + STAGE_BYTES_PER_RAY) * n_rays)
        kern[g["name"]] = dict(leaves=g["grid"].n_leaves, build_s=round(g["build_s"], 2), load_s=round(g["load_s"], 2),
                               mean_ncross=cr / n_rays, trace_ms=ms, trace_rays_per_s=n_rays / ms * 1e3,
                               copy_adjoint_ms=statistics.mean(cper[g["name"]]),
                               gcross_per_s=cr / ms / 1e6, algorithmic_bytes=byt,
                               delta_rho=float(results[g["name"]][1][2].item()),
                               delta_tau=float(results[g["name"]][2][2].item()))
        tot_bytes += byt
        tot_time += ms
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    achieved = tot_bytes / (tot_time / 1e3) / 1e9
    traffic = recorded_traffic(args.workload, prec)
    tot_cross = sum(int(g["nc"].sum().item()) for g in grids)
    byte_per_cross = tot_bytes / max(1, tot_cross)
    fp64_gcross = FP64_OPS_PER_S / FP64_OPS_PER_CROSSING[prec]
    roofline = dict(bound="hbm", achieved=round(achieved, 1), peak=peak, unit="GB/s", frac=round(achieved / peak, 4),
                    traffic=traffic, kernel="trace_kernel, one walk for optical depth and staged emission over "
                                            "prepared rays (hg_rays_trace_stage)",
                    peak_source="measured" if "hbm_gbs" in peaks else "fallback",
                    ceilings=dict(
                        achieved_gcross_per_s=round(tot_cross / tot_time / 1e6, 2),
                        fp64_issue_gcross_per_s=round(fp64_gcross / 1e9, 1),
                        fp64_issue_frac_of_peak=round(fp64_gcross * byte_per_cross / 1e9 / peak, 3),
                        random_gather_gbs=RANDOM_GATHER_GBS,
                        random_gather_frac_of_peak=round(RANDOM_GATHER_GBS / peak, 3),
                        note=f"{FP64_OPS_PER_CROSSING[prec]} FP64 instructions per crossing at the 528 G lane "
                             "operations/s this GPU issues with full warps bound the walk at fp64_issue_gcross_per_s, "
                             "i.e. fp64_issue_frac_of_peak "
                             "of the copy bandwidth in algorithmic bytes; random 96-byte record gathers from "
                             "beyond L2 sustain random_gather_gbs (separate probes); L2 serves part of the records"))

    # the emitted cell sequences of the last step, on the host (the navigation comparison reads a sample)
    for g in grids:
        g["seg_off_h"] = g["off"].cpu().numpy()
        g["seg_cell_h"] = g["cell"].cpu().numpy()

    # e2e: the same step through the public API with host buffers (pinned), copies inside the timed region:
    # rays in; tau, crossing counts, the emitted cells and lengths (the CSR) and the gradient out
    e2e = None
    if not args.no_e2e:
        ho = torch.tensor(o).pin_memory()
        hk = torch.tensor(k).pin_memory()
        hout = []
        for g in grids:
            hout.append([torch.empty(n_rays, dtype=g["tau"].dtype).pin_memory(),
                         torch.empty(n_rays, dtype=torch.int32).pin_memory(),
                         torch.empty(n_rays + 1, dtype=torch.int64).pin_memory(),
                         torch.empty(g["cap"], dtype=torch.int32).pin_memory(),
                         torch.empty(g["cap"], dtype=g["ds"].dtype).pin_memory(),
                         torch.empty(g["grid"].n_leaves, dtype=torch.float32).pin_memory()])
        # Each grid's results go out on a copy stream of its own as soon as its emission and gradient
        # are complete, so that the device-to-host copies (bound by the host link, ~190 GB/s, one copy
        # at a time) overlap the rest of the step and the next step's work.  Steps alternate between
        # two sets of the tau, count and gradient buffers, so that a step never waits for the copies
        # of the step before (a set is rewritten two steps later, after the event `small` of its
        # copies); the CSR arrays are new tensors every step, kept alive for the copy stream by
        # record_stream.
        cstreams = [torch.cuda.Stream(device=dev) for _ in grids]
        hidx = {g["name"]: i for i, g in enumerate(grids)}
        for g in grids:
            g["alt"] = dict(tau=torch.empty_like(g["tau"]), nc=torch.empty_like(g["nc"]),
                            grad=torch.zeros_like(g["grad"]))
        small = [[None, None] for _ in grids]  # per grid and buffer set: the end of its small copies
        cur = [0]

        def copy_out(g):
            i = hidx[g["name"]]
            cs = cstreams[i]
            cs.wait_stream(torch.cuda.current_stream())
            h = hout[i]
            with torch.cuda.stream(cs):
                for dst, src in ((h[0], g["tau"]), (h[1], g["nc"]), (h[5], g["grad"]), (h[2], g["off"])):
                    dst.copy_(src, non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(cs)
                small[i][cur[0]] = ev
                for dst, src in ((h[3], g["cell"]), (h[4], g["ds"])):
                    src.record_stream(cs)
                    dst.copy_(src[:dst.shape[0]], non_blocking=True)
            g["off"].record_stream(cs)

        # the inputs of the next step are copied in on a stream of their own while the current step
        # runs, into the other of two sets of ray buffers (once the step that last read it is done)
        Oset, Kset = [O, torch.empty_like(O)], [K, torch.empty_like(K)]
        h2d = torch.cuda.Stream(device=dev)
        ready, done = [None, None], [None, None]

        def copy_in(x):
            if done[x] is not None:
                h2d.wait_event(done[x])
            with torch.cuda.stream(h2d):
                Oset[x].copy_(ho, non_blocking=True)
                Kset[x].copy_(hk, non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(h2d)
                ready[x] = ev

        def e2e_steps(nsteps):
            # nsteps end-to-end steps; returns their span in ms (CUDA events on the main stream)
            for lst in [ready, done] + small:
                lst[0] = lst[1] = None
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            h2d.wait_stream(stream)
            copy_in(0)
            for s in range(nsteps):
                x = s % 2
                if s + 1 < nsteps:
                    copy_in(1 - x)
                flush.zero_()
                stream.wait_event(ready[x])
                IN["O"], IN["K"] = Oset[x], Kset[x]
                cur[0] = x
                for i, g in enumerate(grids):
                    for key in ("tau", "nc", "grad"):
                        g[key], g["alt"][key] = g["alt"][key], g[key]
                    if small[i][x] is not None:
                        stream.wait_event(small[i][x])
                step(copy_out=copy_out)
                ev = torch.cuda.Event()
                ev.record(stream)
                done[x] = ev
            for cs in cstreams:
                stream.wait_stream(cs)
            b.record(stream)
            IN["O"], IN["K"] = O, K
            torch.cuda.synchronize()
            return a.elapsed_time(b)

        e2e_steps(max(2, args.warmup))  # untimed: the allocator's pools settle for the alternating buffers
        barrier(dist, dev)
        torch.cuda.synchronize()
        span = e2e_steps(args.steps)
        barrier(dist, dev)
        # every step walks the same rays: the host copies of the last step must be the device results
        for h, g in zip(hout, grids):
            if not (torch.equal(h[1], g["nc"].cpu()) and torch.equal(h[2], g["off"].cpu()) and
                    torch.equal(h[3], g["cell"][:h[3].shape[0]].cpu()) and torch.equal(h[0], g["tau"].cpu())):
                raise RuntimeError(f"end-to-end host copies differ from the device results on {g['name']}")
        e_ms = max_over_ranks(dist, span, dev)
        h2d = 2 * n_rays * 3 * 8
        d2h = sum(sum(t.numel() * t.element_size() for t in h) for h in hout)
        e2e = dict(value=sum_over_ranks(dist, rays_per_step * args.steps, dev) / (e_ms / 1e3), unit=UNIT,
                   h2d_bytes_per_step=h2d, d2h_bytes_per_step=d2h,
                   copied="in: origins, directions; out per grid: tau, crossing counts, CSR offsets, "
                          "emitted cells and lengths, gradient",
                   timing="one interval over all steps, after warm-up steps of the same loop, L2 flushes "
                          "included; each grid's device-to-host "
                          "copies run on a stream of their own from the moment its emission is complete and "
                          "overlap the rest of the step and the next step's work (two alternating sets of "
                          "the tau, count and gradient buffers); each step's rays are copied in on their own "
                          "stream while the step before runs (two alternating sets of ray buffers)")

    # quality at equal cell counts (outside the timed region): a k-d tree whose mass threshold is bisected
    # until its leaf count is within 5 % of the octree's, with its Delta-rho and Delta-tau
    matched = None
    if world == 1 and not args.no_matched and args.workload == "disk-1e6":
        matched = matched_kd(hg, model, grids, P, PA, PK, PL, RT, TT)
    orient = None
    if world == 1 and args.kd_orientations and args.workload == "disk-1e6":
        orient = kd_orientations(hg, torch, model, O, K, P, PA, PK, PL, RT, TT, flush, stream)

    # the other configurations: the torus k-d tree, the 64-grid batch, navigation and interaction (one GPU)
    extras = {}
    torus_check = None
    if world == 1 and not args.no_extras and args.workload == "disk-1e6":
        for g in grids:
            g["R"] = None
        extras["torus_1e7"], torus_check = measure_torus(hg, torch, dev, flush, stream)
        torch.cuda.empty_cache()
        extras["batch_64"] = measure_batch(hg, torch, dev, flush, stream)
        torch.cuda.empty_cache()
        extras["navigation"] = measure_navigation(hg, torch, grids, O, K, flush, stream)
        extras["interaction"] = measure_interaction(hg, torch, grids, O, K, rs, flush, stream)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(model, grids, o, k, pts, pa, pk, pl, w, sample=args.cpu_sample)
        if torus_check is not None:
            extras["torus_1e7"]["vs_oracle"] = torus_oracle_check(*torus_check)

    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
                ms_per_step=tot_ms / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f64" if prec == "fp64" else "f32+f64", data="synthetic",
                config=dict(workload=args.workload, description=desc, rays_per_grid=n_rays, points=n_pts,
                            paths=n_paths, precision=prec, l2="flushed between steps (512 MB write)",
                            min_blocks=args.min_blocks or 4,
                            grids=kern, kd_matched_to_octree=matched,
                            **({"kd_orientations": orient} if orient else {}), **extras),
                roofline=roofline, cpu_baseline=cpu, e2e=e2e, gpu_launches=int(launches),
                clocks=dict(sm_mhz=clk["sm_mhz"], sm_max_mhz=clk["sm_max_mhz"], reasons=clk["reasons"]))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# ----------------------------------------------------------------------------- torus and batch workloads

def _timed_steps(torch, stream, steps, flush, fn):
    """Run ``steps`` calls of fn with an L2 flush before each; returns per-step ms (CUDA events)."""
    ev = []
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        ev.append((a, b))
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def _peak():
    try:
        pk = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ----------------------------------------------------------------------------- sub-workloads of the default line
# Measured after the timed disk step (outside it) and reported under config: the other configurations
# -- the ~1e7-leaf torus (FP32-Kahan against FP64), the 64-grid batch (one graph-replayed
# launch against 64 launches), the rope walk against the neighbor-list walk, the interaction search.

def _events_ms(torch, stream, reps, flush, fn):
    return statistics.median(_timed_steps(torch, stream, reps, flush, fn))


def measure_torus(hg, torch, dev, flush, stream, reps=3):
    """The ~1e7-leaf k-d tree of the ring torus with clumps, 1e7 rays: one-shot FP32-Kahan and FP64 passes,
    the FP32 adjoint; rays/s, crossings/s, roofline per pass, FP32K against FP64 tau."""
    model, bp, n_rays, seed = synth.workload_torus_1e7()
    t0 = time.time()
    H = hg.build_grid_gpu(model, bp)
    build_s = time.time() - t0
    G = hg.load_grid(H)
    o, k = synth.emission_rays(seed, n_rays)
    w = synth.adjoint_weights(seed + 3, n_rays)
    O, K, W = torch.tensor(o, device=dev), torch.tensor(k, device=dev), torch.tensor(w, device=dev)
    t32 = torch.empty(n_rays, dtype=torch.float32, device=dev)
    t64 = torch.empty(n_rays, dtype=torch.float64, device=dev)
    nc32 = torch.empty(n_rays, dtype=torch.int32, device=dev)
    nc = torch.empty(n_rays, dtype=torch.int32, device=dev)
    st = torch.empty(n_rays, dtype=torch.uint8, device=dev)
    grad = torch.zeros(G.n_leaves, dtype=torch.float32, device=dev)
    run = {"fp32k": lambda: hg.trace_rays(G, O, K, precision="fp32k", out=(t32, nc32, st)),
           "fp64": lambda: hg.trace_rays(G, O, K, precision="fp64", out=(t64, nc, st))}
    for f in run.values():
        f()
    bits = int(hg.reduce_status(st).item())
    peak, _ = _peak()
    cr = int(nc.sum().item())
    passes = {}
    for prec, f in run.items():
        ms = _events_ms(torch, stream, reps, flush, f)
        byt = BYTES_PER_CROSSING[prec] * cr + BYTES_PER_RAY[prec] * n_rays
        passes[prec] = dict(trace_ms=round(ms, 3), rays_per_s=n_rays / ms * 1e3, gcross_per_s=cr / ms / 1e6,
                            achieved_gbs=round(byt / (ms / 1e3) / 1e9, 1),
                            roofline_frac=round(byt / (ms / 1e3) / 1e9 / peak, 4))
    # the same rays prepared once (setup, queue, segments) and walked per precision: the walk alone
    prepared = {}
    R = hg.prepare_rays(G, O, K)
    prepared["prepare_ms"] = round(_events_ms(torch, stream, reps, flush, lambda: hg.prepare_rays(G, O, K).free()), 3)
    for prec, out_ in (("fp32k", (t32, nc32, st)), ("fp64", (t64, nc, st))):
        f = lambda: R.trace(kappa=1.0, precision=prec, out=out_)  # noqa: E731
        f()
        ms = _events_ms(torch, stream, reps, flush, f)
        byt = BYTES_PER_CROSSING[prec] * cr + BYTES_PER_RAY[prec] * n_rays
        prepared[prec] = dict(walk_ms=round(ms, 3), gcross_per_s=cr / ms / 1e6,
                              roofline_frac=round(byt / (ms / 1e3) / 1e9 / peak, 4))
    R.free()
    grad_ms = _events_ms(torch, stream, 1, flush, lambda: (grad.zero_(), hg.tau_gradient(
        G, O, K, W, grad=grad, grad_precision="fp32")))
    a32 = t32.double().cpu().numpy()
    a64 = t64.cpu().numpy()
    same_counts = bool(torch.equal(nc, nc32))
    # the same passes on the rope walk (records beyond L2: the walk is bound by record gathers)
    t0 = time.time()
    GR = hg.load_grid(H, nav="ropes")
    rope_load_s = time.time() - t0
    ropes = {}
    for prec, out_ in (("fp32k", (t32, nc32, st)), ("fp64", (t64, nc, st))):
        f = lambda: hg.trace_rays(GR, O, K, precision=prec, out=out_)  # noqa: E731
        f()
        ms = _events_ms(torch, stream, reps, flush, f)
        ropes[prec] = dict(trace_ms=round(ms, 3), rays_per_s=n_rays / ms * 1e3, gcross_per_s=cr / ms / 1e6)
    ropes["load_s"] = round(rope_load_s, 2)
    del GR
    pos = a64 > 0
    rel = np.abs(a32[pos] - a64[pos]) / a64[pos]
    out = dict(leaves=G.n_leaves, rays=n_rays, mean_ncross=cr / n_rays, build_gpu_s=round(build_s, 2),
               status_bits=bits, passes=passes, prepared_walks=prepared, adjoint_fp32_ms=round(grad_ms, 3),
               rope_walk=ropes,
               fp32k_over_fp64_speed=passes["fp64"]["trace_ms"] / passes["fp32k"]["trace_ms"],
               fp32k_vs_fp64=dict(max_rel=float(rel.max()), median_rel=float(np.median(rel)),
                                  identical_counts=same_counts),
               description="ring torus + 1000 clumps, k-d tree (mass 7e-7, tau 0.5, q 0.9, max level 10), "
                           "built on the GPU; 1e7 emission rays, one-shot hg_trace_rays per precision")
    del O, K, W, grad
    return out, (H, o, k, a64, a32)


def measure_batch(hg, torch, dev, flush, stream, reps=3):
    """64 grids of uneven size (octree / k-d, disk / ring / clumps), ~1.5e8 rays: the batched FP32-Kahan
    launch replayed from a CUDA graph against 64 separate FP64 launches (and FP32K, and batched FP64)."""
    specs = synth.batch_specs(64)
    grids, begins, leaves = [], [0], []
    t0 = time.time()
    for sp in specs:
        bp = synth.BuildParams(kind=sp["kind"], delta_max=2.0 / sp["target_leaves"], max_level=10, seed=sp["seed"])
        grids.append(hg.load_grid(hg.build_grid_gpu(sp["model"], bp)))
        leaves.append(grids[-1].n_leaves)
        begins.append(begins[-1] + sp["n_rays"])
    build_s = time.time() - t0
    total = begins[-1]
    gen = torch.Generator(device=dev)
    gen.manual_seed(synth.config_seed(4))
    O = torch.rand(total, 3, dtype=torch.float64, device=dev, generator=gen) * 2.0 - 1.0
    mu = torch.rand(total, dtype=torch.float64, device=dev, generator=gen) * 2.0 - 1.0
    phi = torch.rand(total, dtype=torch.float64, device=dev, generator=gen) * (2.0 * math.pi)
    sn = torch.sqrt(torch.clamp(1.0 - mu * mu, min=0.0))
    K = torch.stack([sn * torch.cos(phi), sn * torch.sin(phi), mu], dim=1).contiguous()
    del mu, phi, sn
    batch = hg.Batch(grids, begins)
    t32 = torch.empty(total, dtype=torch.float32, device=dev)
    t64 = torch.empty(total, dtype=torch.float64, device=dev)
    nc = torch.empty(total, dtype=torch.int32, device=dev)
    st = torch.empty(total, dtype=torch.uint8, device=dev)
    side = torch.cuda.Stream(device=dev)
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        batch.trace(O, K, precision="fp32k", out=(t32, nc, st))
    stream.wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        batch.trace(O, K, precision="fp32k", out=(t32, nc, st))
    graph.replay()
    torch.cuda.synchronize()
    bits = int(hg.reduce_status(st).item())
    cr = int(nc.sum().item())

    def sep(prec, out):
        for i, g in enumerate(grids):
            s_ = slice(begins[i], begins[i + 1])
            hg.trace_rays(g, O[s_], K[s_], precision=prec, out=(out[0][s_], out[1][s_], None))

    batched = _events_ms(torch, stream, reps, flush, graph.replay)
    sep64 = _events_ms(torch, stream, reps, flush, lambda: sep("fp64", (t64, nc)))
    sep32 = _events_ms(torch, stream, reps, flush, lambda: sep("fp32k", (t32, nc)))
    b64 = _events_ms(torch, stream, reps, flush, lambda: batch.trace(O, K, precision="fp64", out=(t64, nc, None)))
    peak, _ = _peak()
    byt = BYTES_PER_CROSSING["fp32k"] * cr + BYTES_PER_RAY["fp32k"] * total
    del graph, batch, O, K
    return dict(grids=len(grids), rays=total, leaves_total=int(sum(leaves)), leaves_min=int(min(leaves)),
                leaves_max=int(max(leaves)), build_gpu_s=round(build_s, 1), mean_ncross=cr / total, status_bits=bits,
                batched_fp32k_graph_ms=round(batched, 3), batched_fp32k_rays_per_s=total / batched * 1e3,
                separate_fp64_ms=round(sep64, 3), separate_fp64_rays_per_s=total / sep64 * 1e3,
                separate_fp32k_ms=round(sep32, 3), batched_fp64_ms=round(b64, 3),
                batched_fp32k_over_separate_fp64=sep64 / batched, batched_fp32k_over_separate_fp32k=sep32 / batched,
                roofline_frac_batched_fp32k=round(byt / (batched / 1e3) / 1e9 / peak, 4),
                rays_generated="on the device with a seeded torch generator",
                description="64 grids (octree/k-d, disk/ring/clumps, 1e4-1e6 leaves, built on the GPU), "
                            "1e5-1e7 rays each")


def _node_depths(H):
    depth = np.zeros(H.n_nodes, np.int32)
    nch = 8 if H.kind == 0 else 2
    internal = np.nonzero(H.child_first >= 0)[0]
    for nd in internal:  # breadth-first order: parents before children
        c = H.child_first[nd]
        depth[c:c + nch] = depth[nd] + 1
    return depth


def navigation_costs(H, ropes, seg_off, seg_cell, n_rays=20000):
    """Exact per-crossing costs of finding the next leaf, from the emitted cell sequences of n_rays rays:
    with neighbor lists, the position of the next leaf in the exit wall's list (records tested, tail ids
    read), or, for a list too long to store whose head misses, the descent below the wall's rope node;
    with ropes, the nodes visited below the rope and the records tested.  Bytes: 96 per record, 4 per tail id, 16 (k-d) or 32 (octree) per node.
    Crossings through an edge or corner (no unique shared wall) count as root descents for both."""
    node_b = 32 if H.kind == 0 else 16
    n = min(n_rays, seg_off.shape[0] - 1)
    cells = seg_cell[:seg_off[n]].astype(np.int64)
    ray_of = np.repeat(np.arange(n), np.diff(seg_off[:n + 1]))
    same = ray_of[1:] == ray_of[:-1]
    a, b = cells[:-1][same], cells[1:][same]
    lo, hi = H.node_lo[H.leaf_node], H.node_hi[H.leaf_node]
    depth = _node_depths(H)
    leaf_depth = depth[H.leaf_node]
    wall = np.full(a.shape[0], -1, np.int64)
    nwalls = np.zeros(a.shape[0], np.int64)
    for ax in range(3):
        t = [x for x in range(3) if x != ax]
        ov = np.ones(a.shape[0], bool)
        for x in t:
            ov &= np.minimum(hi[a, x], hi[b, x]) > np.maximum(lo[a, x], lo[b, x])
        up = ov & (hi[a, ax] == lo[b, ax])
        dn = ov & (lo[a, ax] == hi[b, ax])
        wall = np.where(up, 2 * ax + 1, np.where(dn, 2 * ax, wall))
        nwalls += up.astype(np.int64) + dn.astype(np.int64)
    face = (wall >= 0) & (nwalls == 1)
    # neighbor lists: position of b in list (a, wall)
    rec_l = np.zeros(a.shape[0], np.float64)
    tail_l = np.zeros(a.shape[0], np.float64)
    node_l = np.zeros(a.shape[0], np.float64)
    off = H.nbr_off
    wsafe = np.maximum(wall, 0)
    start = off[6 * a + wsafe]
    cnt = off[6 * a + wsafe + 1] - start
    head = face & (cnt > 0) & (H.nbr_id[np.minimum(start, H.nbr_id.shape[0] - 1)] == b)
    rec_l[head] = 1
    for i in np.nonzero(~head)[0]:
        if face[i]:
            lst = H.nbr_id[start[i]:start[i] + cnt[i]]
            stored = lst if cnt[i] <= 16 else lst[:1]
            hit = np.nonzero(stored == b[i])[0]
            if hit.size:
                p = int(hit[0])
                rec_l[i], tail_l[i] = p + 1, p
                continue
            rec_l[i], tail_l[i] = stored.size + 1, max(0, stored.size - 1)
            if cnt[i] > 16:  # the rope node kept in the tail slot, then the descent below it
                rn_i = -2 - int(ropes[a[i], wall[i]])
                tail_l[i] = 1
                node_l[i] = leaf_depth[b[i]] - depth[rn_i] if ropes[a[i], wall[i]] <= -2 else leaf_depth[b[i]]
                continue
        else:
            rec_l[i] = 2
        node_l[i] = leaf_depth[b[i]]
    # ropes
    r = ropes[a, wsafe]
    rec_r = np.zeros(a.shape[0], np.float64)
    node_r = np.zeros(a.shape[0], np.float64)
    to_leaf = face & (r >= 0)
    hit_leaf = to_leaf & (r == b)
    rec_r[hit_leaf] = 1
    internal = face & (r <= -2)
    rn = np.where(internal, -2 - r, 0)
    # b lies below the rope's node when the node's box contains b's box
    inside = internal.copy()
    for ax in range(3):
        inside &= (H.node_lo[rn, ax] <= lo[b, ax]) & (hi[b, ax] <= H.node_hi[rn, ax])
    rec_r[inside] = 1
    node_r[inside] = leaf_depth[b[inside]] - depth[rn[inside]]
    miss = ~(hit_leaf | inside)
    rec_r[miss] = 2
    node_r[miss] = leaf_depth[b[miss]] + np.where(internal[miss], leaf_depth[b[miss]] - depth[rn[miss]], 0)
    m = max(1, a.shape[0])
    lists = dict(records=float(rec_l.sum() / m), tail_ids=float(tail_l.sum() / m), nodes=float(node_l.sum() / m),
                 head_hit=float(head.sum() / m))
    lists["bytes"] = 96 * lists["records"] + 4 * lists["tail_ids"] + node_b * lists["nodes"]
    rope = dict(records=float(rec_r.sum() / m), nodes=float(node_r.sum() / m),
                rope_to_leaf=float(to_leaf.sum() / m), rope_to_leaf_hit=float(hit_leaf.sum() / m))
    rope["bytes"] = 96 * rope["records"] + node_b * rope["nodes"]
    return dict(transitions=int(a.shape[0]), edge_or_corner=float((~face).sum() / m), lists=lists, ropes=rope,
                bytes_note="next-leaf lookups only; every crossing also reads nothing else for navigation")


def measure_navigation(hg, torch, grids, O, K, flush, stream, reps=5):
    """The rope walk against the neighbor-list walk on the step's grids and rays: the prepared optical-depth
    walk (median of reps, L2 flushed), and the exact lookup costs from a sample of the emitted sequences."""
    out = {}
    for g in grids:
        H = g["host"]
        t0 = time.time()
        ropes = hg.build_ropes(H)
        rope_s = time.time() - t0
        GR = hg.load_grid(H, nav="ropes", ropes=ropes)
        res = {}
        for name, G in (("lists", g["grid"]), ("ropes", GR)):
            R = hg.prepare_rays(G, O, K)
            tau, nc, st = R.trace()
            ms = _events_ms(torch, stream, reps, flush, lambda: R.trace(out=(tau, nc, st)))
            cr = int(nc.sum().item())
            R.free()
            res[name] = dict(walk_ms=round(ms, 4), gcross_per_s=cr / ms / 1e6)
        costs = navigation_costs(H, ropes, g["seg_off_h"], g["seg_cell_h"])
        for name in ("lists", "ropes"):
            res[name].update(costs[name])
        res.update(transitions_sampled=costs["transitions"], edge_or_corner=costs["edge_or_corner"],
                   rope_build_s=round(rope_s, 2), device_bytes_lists=g["grid"].device_bytes,
                   device_bytes_ropes=GR.device_bytes)
        out[g["name"]] = res
        del GR
    return out


def measure_interaction(hg, torch, grids, O, K, seed, flush, stream, reps=3):
    """Interaction-point search on the step's grids and rays (kappa 200, tau_int = -ln u)."""
    n = O.shape[0]
    TI = torch.tensor(synth.interaction_depths(seed + 5, n), device=O.device)
    peak, _ = _peak()
    out = {}
    for g in grids:
        res = hg.find_interactions(g["grid"], O, K, TI, kappa=INTERACT_KAPPA)
        ms = _events_ms(torch, stream, reps, flush,
                        lambda: hg.find_interactions(g["grid"], O, K, TI, kappa=INTERACT_KAPPA, out=res))
        cr = int(res[2].sum().item())
        byt = BYTES_PER_CROSSING["fp64"] * cr + INTERACT_BYTES_PER_RAY * n
        out[g["name"]] = dict(walk_ms=round(ms, 4), packets_per_s=n / ms * 1e3, gcross_per_s=cr / ms / 1e6,
                              mean_ncross=cr / n, interacted=float((res[0] >= 0).float().mean().item()),
                              roofline_frac=round(byt / (ms / 1e3) / 1e9 / peak, 4))
    return out


def run_torus(args):
    import torch
    import paper_1311_0705_gb300 as hg

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = dist_init(world, True)
    desc, maker = WORKLOADS[args.workload]
    model, grids, n_rays, seed = maker(hg)
    if args.rays:
        n_rays = args.rays  # a smaller ray batch on the full grid (profiling)
    g = grids[0]
    t0 = time.time()
    G = hg.load_grid(g["host"], validate=args.validate)
    torch.cuda.synchronize()
    load_s = time.time() - t0
    rs = rank_seed(seed, rank)
    o, k = synth.emission_rays(rs, n_rays)
    w = synth.adjoint_weights(rs + 3, n_rays)
    O, K, W = torch.tensor(o, device=dev), torch.tensor(k, device=dev), torch.tensor(w, device=dev)
    t32 = torch.empty(n_rays, dtype=torch.float32, device=dev)
    t64 = torch.empty(n_rays, dtype=torch.float64, device=dev)
    nc = torch.empty(n_rays, dtype=torch.int32, device=dev)
    nc64 = torch.empty(n_rays, dtype=torch.int32, device=dev)
    st = torch.empty(n_rays, dtype=torch.uint8, device=dev)
    grad = torch.zeros(G.n_leaves, dtype=torch.float32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    kev = {"fp32k": [], "fp64": []}

    def step(record=False):
        for prec, out in (("fp32k", (t32, nc, st)), ("fp64", (t64, nc64, None))):
            if record:
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
            hg.trace_rays(G, O, K, precision=prec, out=out)
            if record:
                e1.record(stream)
                kev[prec].append((e0, e1))
        grad.zero_()
        hg.tau_gradient(G, O, K, W, grad=grad, grad_precision="fp32")

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    bits = int(hg.reduce_status(st).item())
    if bits:
        raise RuntimeError(f"ray status bits {bits}")
    clocks = ClockSampler(local)
    clocks.start()
    l0 = hg.launch_count()
    barrier(dist, dev)
    torch.cuda.synchronize()
    times = _timed_steps(torch, stream, args.steps, flush, lambda: step(True))
    barrier(dist, dev)
    launches = hg.launch_count() - l0
    clk = clocks.stop()
    tot_ms = max_over_ranks(dist, sum(times), dev)
    value = sum_over_ranks(dist, n_rays * args.steps, dev) / (tot_ms / 1e3)
    cr = int(nc.sum().item())
    peak, src = _peak()
    passes = {}
    for prec in ("fp32k", "fp64"):
        ms = statistics.mean(a.elapsed_time(b) for a, b in kev[prec])
        byt = BYTES_PER_CROSSING[prec] * cr + BYTES_PER_RAY[prec] * n_rays
        passes[prec] = dict(trace_ms=ms, rays_per_s=n_rays / ms * 1e3, gcross_per_s=cr / ms / 1e6,
                            achieved_gbs=byt / (ms / 1e3) / 1e9, algorithmic_bytes=byt)
    a32 = t32.double().cpu().numpy()
    a64 = t64.cpu().numpy()
    pos = a64 > 0
    rel = np.abs(a32[pos] - a64[pos]) / a64[pos]
    same_counts = bool(torch.equal(nc, nc64))
    ach = passes["fp32k"]["achieved_gbs"]
    roofline = dict(bound="hbm", achieved=round(ach, 1), peak=peak, unit="GB/s", frac=round(ach / peak, 4),
                    traffic=recorded_traffic(args.workload, "fp32k"), kernel="trace_kernel FP32K (hg_trace_rays)",
                    peak_source=src)
    e2e = None
    if not args.no_e2e:
        ho, hk = torch.tensor(o).pin_memory(), torch.tensor(k).pin_memory()
        h32 = torch.empty(n_rays, dtype=torch.float32).pin_memory()
        h64 = torch.empty(n_rays, dtype=torch.float64).pin_memory()
        hn = torch.empty(n_rays, dtype=torch.int32).pin_memory()

        def e2e_step():
            O.copy_(ho, non_blocking=True)
            K.copy_(hk, non_blocking=True)
            step()
            h32.copy_(t32, non_blocking=True)
            h64.copy_(t64, non_blocking=True)
            hn.copy_(nc, non_blocking=True)

        barrier(dist, dev)
        et = _timed_steps(torch, stream, args.steps, flush, e2e_step)
        barrier(dist, dev)
        e_ms = max_over_ranks(dist, sum(et), dev)
        e2e = dict(value=sum_over_ranks(dist, n_rays * args.steps, dev) / (e_ms / 1e3), unit=UNIT,
                   h2d_bytes_per_step=2 * n_rays * 24, d2h_bytes_per_step=n_rays * (4 + 8 + 4))
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        H = g["host"]
        T = oracle.wrap_tree(H.kind, H.node_lo, H.node_hi, H.child_first, H.node_leaf, H.leaf_rho)
        n = min(args.cpu_sample, n_rays)
        threads = os.cpu_count() or 1
        t0 = time.perf_counter()
        r = oracle.trace(T, o[:n], k[:n], emit=True, threads=threads)
        oracle.adjoint(T.n_leaves, r["seg_off"], r["seg_cell"], r["seg_ds"], w[:n].astype(np.float64))
        dt = time.perf_counter() - t0
        cpu = dict(value=n / dt, unit=UNIT, cores=threads, kind="oracle",
                   sample=f"{n} of the {n_rays} rays: FP64 trace with emission and adjoint accumulation")
    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
                ms_per_step=tot_ms / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f32+f64", data="synthetic",
                config=dict(workload=args.workload, description=desc, rays=n_rays, leaves=G.n_leaves,
                            build_s=round(g["build_s"], 1), load_s=round(load_s, 2), mean_ncross=cr / n_rays,
                            passes=passes, fp32k_vs_fp64=dict(max_rel=float(rel.max()), median_rel=float(np.median(rel)),
                                                              identical_counts=same_counts),
                            l2="flushed between steps (512 MB write); grid records exceed L2"),
                roofline=roofline, cpu_baseline=cpu, e2e=e2e, gpu_launches=int(launches),
                clocks=dict(sm_mhz=clk["sm_mhz"], sm_max_mhz=clk["sm_max_mhz"], reasons=clk["reasons"]))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_batch(args):
    import torch
    import paper_1311_0705_gb300 as hg

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = dist_init(world, True)
    specs = synth.batch_specs(64)
    grids, begins, leaves = [], [0], []
    t0 = time.time()
    for sp in specs:
        bp = synth.BuildParams(kind=sp["kind"], delta_max=2.0 / sp["target_leaves"], max_level=10, seed=sp["seed"])
        grids.append(hg.load_grid(hg.build_grid(sp["model"], bp)))
        leaves.append(grids[-1].n_leaves)
        begins.append(begins[-1] + sp["n_rays"])
    build_s = time.time() - t0
    total = begins[-1]
    gen = torch.Generator(device=dev)
    gen.manual_seed(synth.config_seed(4) + 7919 * rank)
    O = torch.rand(total, 3, dtype=torch.float64, device=dev, generator=gen) * 2.0 - 1.0
    mu = torch.rand(total, dtype=torch.float64, device=dev, generator=gen) * 2.0 - 1.0
    phi = torch.rand(total, dtype=torch.float64, device=dev, generator=gen) * (2.0 * math.pi)
    sn = torch.sqrt(torch.clamp(1.0 - mu * mu, min=0.0))
    K = torch.stack([sn * torch.cos(phi), sn * torch.sin(phi), mu], dim=1).contiguous()
    batch = hg.Batch(grids, begins)
    t32 = torch.empty(total, dtype=torch.float32, device=dev)
    t64 = torch.empty(total, dtype=torch.float64, device=dev)
    nc = torch.empty(total, dtype=torch.int32, device=dev)
    st = torch.empty(total, dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(args.warmup):
            batch.trace(O, K, precision="fp32k", out=(t32, nc, st))
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        batch.trace(O, K, precision="fp32k", out=(t32, nc, st))
    graph.replay()
    torch.cuda.synchronize()
    bits = int(hg.reduce_status(st).item())
    if bits:
        raise RuntimeError(f"ray status bits {bits}")
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(local)
    clocks.start()
    l0 = hg.launch_count()
    barrier(dist, dev)
    torch.cuda.synchronize()
    times = _timed_steps(torch, stream, args.steps, flush, graph.replay)
    barrier(dist, dev)
    clk = clocks.stop()
    # graph replays launch the library's kernels without passing through its launch counter
    launches = hg.launch_count() - l0 + 2 * args.steps
    tot_ms = max_over_ranks(dist, sum(times), dev)
    value = sum_over_ranks(dist, total * args.steps, dev) / (tot_ms / 1e3)
    cr = int(nc.sum().item())

    def sep(prec, out):
        for i, g in enumerate(grids):
            s = slice(begins[i], begins[i + 1])
            hg.trace_rays(g, O[s], K[s], precision=prec, out=(out[0][s], out[1][s], out[2][s]))

    sep("fp32k", (t32, nc, st))
    sep_ms = statistics.mean(_timed_steps(torch, stream, max(1, min(3, args.steps)), flush,
                                          lambda: sep("fp32k", (t32, nc, st))))
    nc64 = torch.empty_like(nc)
    b64_ms = statistics.mean(_timed_steps(torch, stream, max(1, min(3, args.steps)), flush,
                                          lambda: batch.trace(O, K, precision="fp64", out=(t64, nc64, None))))
    peak, src = _peak()
    ach = (BYTES_PER_CROSSING["fp32k"] * cr + BYTES_PER_RAY["fp32k"] * total) / (tot_ms / args.steps / 1e3) / 1e9
    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
                ms_per_step=tot_ms / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f32+f64", data="synthetic",
                config=dict(workload=args.workload, description=WORKLOADS[args.workload][0], grids=len(grids),
                            rays=total, leaves_total=int(sum(leaves)), leaves_min=int(min(leaves)),
                            leaves_max=int(max(leaves)), build_s=round(build_s, 1), mean_ncross=cr / total,
                            batched_fp32k_graph_ms=tot_ms / args.steps, separate_launches_fp32k_ms=sep_ms,
                            batched_fp64_ms=b64_ms, separate_over_batched=sep_ms / (tot_ms / args.steps),
                            rays_generated="on the device with a seeded torch generator",
                            l2="flushed between steps (512 MB write)"),
                roofline=dict(bound="hbm", achieved=round(ach, 1), peak=peak, unit="GB/s", frac=round(ach / peak, 4),
                              traffic=None, kernel="batch_kernel FP32K (hg_batch_trace), setup pass included",
                              peak_source=src),
                cpu_baseline=None, e2e=None, gpu_launches=int(launches),
                clocks=dict(sm_mhz=clk["sm_mhz"], sm_max_mhz=clk["sm_max_mhz"], reasons=clk["reasons"]))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# ----------------------------------------------------------------------------- CPU oracle arm

def oracle_step(oracle, model, trees, o, k, pts, pa, pk, pl, w, threads):
    """The oracle's version of one step on a sample: trace with emission (tau, counts,
    cell sequences, adjoint accumulation), grid density at points, Delta-tau paths."""
    for T in trees:
        r = oracle.trace(T, o, k, emit=True, threads=threads)
        oracle.adjoint(T.n_leaves, r["seg_off"], r["seg_cell"], r["seg_ds"], w.astype(np.float64))
        oracle.sample_density(T, pts)
        oracle.trace(T, pa, pk, smax=pl, threads=threads)


def _oracle_trees(oracle, grids):
    trees = []
    for g in grids:
        H = g["host"]
        trees.append(oracle.wrap_tree(H.kind, H.node_lo, H.node_hi, H.child_first, H.node_leaf, H.leaf_rho))
    return trees


def run_interact(args):
    import torch
    import paper_1311_0705_gb300 as hg

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = dist_init(world, True)
    desc, maker = WORKLOADS[args.workload]
    model, grids, n_rays, seed = maker(hg)
    rs = rank_seed(seed, rank)
    o, k = synth.emission_rays(rs, n_rays)
    ti = synth.interaction_depths(rs + 5, n_rays)
    O, K, TI = torch.tensor(o, device=dev), torch.tensor(k, device=dev), torch.tensor(ti, device=dev)
    for g in grids:
        g["grid"] = hg.load_grid(g["host"], validate=args.validate)
        g["out"] = (torch.empty(n_rays, dtype=torch.int32, device=dev), torch.empty(n_rays, dtype=torch.float64,
                                                                                 device=dev),
                    torch.empty(n_rays, dtype=torch.int32, device=dev), torch.empty(n_rays, dtype=torch.uint8,
                                                                                 device=dev))
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    kev = {g["name"]: [] for g in grids}

    def step(record=False):
        for g in grids:
            if record:
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
            hg.find_interactions(g["grid"], O, K, TI, kappa=INTERACT_KAPPA, out=g["out"])
            if record:
                e1.record(stream)
                kev[g["name"]].append((e0, e1))

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    for g in grids:
        bits = int(hg.reduce_status(g["out"][3]).item())
        if bits:
            raise RuntimeError(f"ray status bits {bits} on {g['name']}")
    clocks = ClockSampler(local)
    clocks.start()
    l0 = hg.launch_count()
    barrier(dist, dev)
    torch.cuda.synchronize()
    times = _timed_steps(torch, stream, args.steps, flush, lambda: step(True))
    barrier(dist, dev)
    launches = hg.launch_count() - l0
    clk = clocks.stop()
    tot_ms = max_over_ranks(dist, sum(times), dev)
    value = sum_over_ranks(dist, n_rays * len(grids) * args.steps, dev) / (tot_ms / 1e3)
    peak, src = _peak()
    kern, tb, tt = {}, 0.0, 0.0
    for g in grids:
        cell, t, nc, st = g["out"]
        cr = int(nc.sum().item())
        ms = statistics.mean(a.elapsed_time(b) for a, b in kev[g["name"]])
        byt = BYTES_PER_CROSSING["fp64"] * cr + INTERACT_BYTES_PER_RAY * n_rays
        kern[g["name"]] = dict(leaves=g["grid"].n_leaves, walk_ms=ms, packets_per_s=n_rays / ms * 1e3,
                               mean_ncross=cr / n_rays, gcross_per_s=cr / ms / 1e6,
                               interacted=float((cell >= 0).float().mean().item()), algorithmic_bytes=byt)
        tb += byt
        tt += ms
    ach = tb / (tt / 1e3) / 1e9
    roofline = dict(bound="hbm", achieved=round(ach, 1), peak=peak, unit="GB/s", frac=round(ach / peak, 4),
                    traffic=recorded_traffic(args.workload, "fp64"),
                    kernel="trace_kernel interaction search (hg_find_interactions)", peak_source=src)
    e2e = None
    if not args.no_e2e:
        ho, hk, hti = torch.tensor(o).pin_memory(), torch.tensor(k).pin_memory(), torch.tensor(ti).pin_memory()
        hc = [torch.empty(n_rays, dtype=torch.int32).pin_memory() for _ in grids]
        ht = [torch.empty(n_rays, dtype=torch.float64).pin_memory() for _ in grids]

        def e2e_step():
            O.copy_(ho, non_blocking=True)
            K.copy_(hk, non_blocking=True)
            TI.copy_(hti, non_blocking=True)
            step()
            for j, g in enumerate(grids):
                hc[j].copy_(g["out"][0], non_blocking=True)
                ht[j].copy_(g["out"][1], non_blocking=True)

        barrier(dist, dev)
        et = _timed_steps(torch, stream, args.steps, flush, e2e_step)
        barrier(dist, dev)
        e_ms = max_over_ranks(dist, sum(et), dev)
        e2e = dict(value=sum_over_ranks(dist, n_rays * len(grids) * args.steps, dev) / (e_ms / 1e3), unit=UNIT,
                   h2d_bytes_per_step=n_rays * (24 + 24 + 8), d2h_bytes_per_step=len(grids) * n_rays * (4 + 8))
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        trees = _oracle_trees(oracle, grids)
        threads = os.cpu_count() or 1
        n = min(args.cpu_sample, n_rays)
        t0 = time.perf_counter()
        for T in trees:
            oracle.interact(T, o[:n], k[:n], ti[:n], kappa=INTERACT_KAPPA, threads=threads)
        dt = time.perf_counter() - t0
        cpu = dict(value=n * len(trees) / dt, unit=UNIT, cores=threads, kind="oracle",
                   sample=f"{n} of the {n_rays} packets per grid through {len(trees)} grids: interaction search")
    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
                ms_per_step=tot_ms / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f64", data="synthetic",
                config=dict(workload=args.workload, description=desc, packets_per_grid=n_rays, kappa=INTERACT_KAPPA,
                            grids=kern,
                            l2="flushed between steps (512 MB write)"),
                roofline=roofline, cpu_baseline=cpu, e2e=e2e, gpu_launches=int(launches),
                clocks=dict(sm_mhz=clk["sm_mhz"], sm_max_mhz=clk["sm_max_mhz"], reasons=clk["reasons"]))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_build(args):
    """Tree construction on the GPU (hg_build_grid_gpu) of the disk-1e6 octree and k-d tree; value = nodes
    built per second.  The call takes a host model description and returns host arrays, so the timed
    step is end to end; the host builder (all cores) and the oracle's builder are timed beside it."""
    import torch
    import paper_1311_0705_gb300 as hg

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = dist_init(world, True)
    desc, _ = WORKLOADS[args.workload]
    specs = []
    for kind in (synth.TREE_OCTREE, synth.TREE_KD):
        model, bp, _, _ = synth.workload_disk_1e6(kind)
        specs.append(("octree" if kind == 0 else "kd", model, bp))
    stream = torch.cuda.current_stream()
    sizes = {}

    def step(record=None):
        for name, model, bp in specs:
            if record is not None:
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
            G = hg.build_grid_gpu(model, bp)
            if record is not None:
                e1.record(stream)
                record.append((name, e0, e1))
            sizes[name] = (G.n_nodes, G.n_leaves, int(G.nbr_off[-1]))

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    l0 = hg.launch_count()
    barrier(dist, dev)
    torch.cuda.synchronize()
    ev = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step(ev)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    barrier(dist, dev)
    launches = hg.launch_count() - l0
    clk = clocks.stop()
    per = {}
    for name, a, b in ev:
        per.setdefault(name, []).append(a.elapsed_time(b))
    tot_ms = max_over_ranks(dist, sum(sum(v) for v in per.values()), dev)
    nodes = sum(v[0] for v in sizes.values())
    value = sum_over_ranks(dist, nodes * args.steps, dev) / (tot_ms / 1e3)
    grids = {}
    for name, model, bp in specs:
        t = time.perf_counter()
        hg.build_grid(model, bp)
        host_s = time.perf_counter() - t
        n, nl, ne = sizes[name]
        ms = statistics.mean(per[name])
        grids[name] = dict(nodes=n, leaves=nl, list_entries=ne, gpu_build_ms=ms, host_build_ms=host_s * 1e3,
                           nodes_per_s=n / ms * 1e3)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        name, model, bp = specs[1]  # the k-d tree: 2.9e6 nodes, a few seconds single-threaded
        t = time.perf_counter()
        T = oracle.build_tree(model, bp)
        dt = time.perf_counter() - t
        cpu = dict(value=T.n_nodes / dt, unit="nodes/s", cores=1, kind="oracle",
                   sample=f"the oracle's builder on the k-d grid ({T.n_nodes} nodes, node list and statistics; "
                          "the oracle has no neighbor lists)")
    per_node_h2d = 3 * 4 + 3 * 8  # levels and indices of each node, uploaded level by level
    h2d = sum(v[0] * (per_node_h2d + 4 + 4 + 3 * 8) + v[1] * 8 for v in sizes.values())
    d2h = sum(v[0] * 48 + (6 * v[1] + 1) * 8 + v[2] * 4 for v in sizes.values())
    line = dict(metric=METRIC, value=value, unit="nodes/s", n_gpus=world, steps=args.steps, warmup=args.warmup,
                ms_per_step=tot_ms / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f64", data="synthetic",
                config=dict(workload=args.workload, description=desc, grids=grids,
                            wall_ms_per_step=wall / args.steps * 1e3,
                            timing="CUDA events on the builder's stream around each (synchronous) build call"),
                roofline=None, cpu_baseline=cpu,
                e2e=dict(value=value, unit="nodes/s", h2d_bytes_per_step=h2d, d2h_bytes_per_step=d2h,
                         note="the build call is host to host: the timed step already includes its copies"),
                gpu_launches=int(launches),
                clocks=dict(sm_mhz=clk["sm_mhz"], sm_max_mhz=clk["sm_max_mhz"], reasons=clk["reasons"]))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def cpu_baseline(model, grids, o, k, pts, pa, pk, pl, w, sample: int = 200_000):
    import oracle
    threads = os.cpu_count() or 1
    trees = _oracle_trees(oracle, grids)
    n = min(sample, o.shape[0])
    npth = max(1, n // 10)
    rt = oracle.rho_true(model, pts[:n])  # noqa: F841  (the truth the step compares against)
    t0 = time.perf_counter()
    oracle_step(oracle, model, trees, o[:n], k[:n], pts[:n], pa[:npth], pk[:npth], pl[:npth], w[:n], threads)
    dt = time.perf_counter() - t0
    return dict(value=n * len(trees) / dt, unit=UNIT, cores=threads, kind="oracle",
                sample=f"{n} of the emission rays per grid (+{n} points, {npth} paths) through "
                       f"{len(trees)} grids: trace with emission, adjoint accumulation, density, Delta-tau paths")


def torus_oracle_check(H, o, k, t64, t32, n: int = 20000):
    """The torus rays' tau from the GPU (FP64 and FP32-Kahan) against the FP64 oracle on a sample."""
    import oracle
    T = oracle.wrap_tree(H.kind, H.node_lo, H.node_hi, H.child_first, H.node_leaf, H.leaf_rho)
    ref = oracle.trace(T, o[:n], k[:n], threads=os.cpu_count() or 1)["tau"]
    pos = ref > 0
    r64 = np.abs(t64[:n][pos] - ref[pos]) / ref[pos]
    r32 = np.abs(t32[:n][pos] - ref[pos]) / ref[pos]
    return dict(rays=n, fp64_max_rel=float(r64.max()), fp32k_max_rel=float(r32.max()),
                fp32k_median_rel=float(np.median(r32)))


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    import oracle
    import paper_1311_0705_gb300 as hg  # the grid is the workload's input; only the oracle runs below
    desc, maker = WORKLOADS[args.workload]
    model, grids, n_rays, seed = maker(hg)
    threads = os.cpu_count() or 1
    trees = _oracle_trees(oracle, grids)
    o, k = synth.emission_rays(seed, n_rays)
    pts = synth.sample_points(seed + 1, n_rays)
    n_paths = max(1, n_rays // 10)
    pa, pk, pl = synth.endpoint_paths(seed + 2, n_paths)
    w = synth.adjoint_weights(seed + 3, n_rays)
    n = min(args.cpu_sample, n_rays)
    npth = max(1, n // 10)
    for _ in range(args.warmup):
        oracle_step(oracle, model, trees, o[:n], k[:n], pts[:n], pa[:npth], pk[:npth], pl[:npth], w[:n], threads)
    t0 = time.perf_counter()
    for s in range(args.steps):
        j = (s * n) % max(1, n_rays - n + 1)
        oracle_step(oracle, model, trees, o[j:j + n], k[j:j + n], pts[j:j + n], pa[:npth], pk[:npth], pl[:npth],
                    w[j:j + n], threads)
    dt = time.perf_counter() - t0
    value = n * len(trees) * args.steps / dt
    sample = (f"per step {n} of the {n_rays} emission rays per grid (+{n} points, {npth} paths) through "
              f"{len(trees)} grids: trace with emission, adjoint accumulation, density, Delta-tau paths")
    line = dict(impl="reference", metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps,
                warmup=args.warmup, ms_per_step=dt / args.steps * 1e3, higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f64", data="synthetic",
                config=dict(workload=args.workload, description=desc, rays_per_grid=n_rays, precision="fp64"),
                cpu_baseline=dict(value=value, unit=UNIT, cores=threads, kind="oracle", sample=sample),
                e2e=dict(value=value, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="disk-1e6")
    ap.add_argument("--precision", choices=["fp64", "fp32k"], default="fp64")
    ap.add_argument("--validate", action="store_true", help="validate grid descriptions at load")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-matched", action="store_true",
                    help="skip the k-d tree built to the octree's leaf count (quality at equal N_cells)")
    ap.add_argument("--cpu-sample", type=int, default=200_000)
    ap.add_argument("--rays", type=int, default=0,
                    help="torus-1e7 only: rays per step instead of 1e7 (a smaller case of the same kernel for ncu)")
    ap.add_argument("--min-blocks", type=int, choices=[3, 4], default=0,
                    help="register budget of the step's walks: 3 (80 registers) or 4 (64) blocks of 256 per SM")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the torus, 64-grid batch, rope and interaction measurements after the timed step")
    ap.add_argument("--kd-orientations", action="store_true",
                    help="also compare the cyclic and gradient-axis k-d trees (quality and walk speed, untimed)")
    args = ap.parse_args(argv)
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        if args.workload in ("disk-1e6", "disk-1e4"):
            run_reference(args)
        else:
            print(json.dumps(dict(impl="reference", unavailable="the CPU oracle arm covers the disk workloads only")))
    elif args.workload == "torus-1e7":
        run_torus(args)
    elif args.workload == "batch-64":
        run_batch(args)
    elif args.workload == "interact-1e6":
        run_interact(args)
    elif args.workload == "build-1e6":
        run_build(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
