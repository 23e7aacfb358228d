#!/usr/bin/env python3
"""Benchmark of the coupled LB-DPS step on GB300.

Default workload: the 3D riser, D3Q19 256 x 256 x 1024 cells (walls in x
and y, periodic in z), 4,000,000 particles of 54 um at volume fraction 0.03,
FP32 deviation storage (about 10 GB of populations): the largest
single-GPU configuration of the riser of the paper's §3.2 / Table 2,
extended to 3D as §4 suggests.  A "step" is one coupled time step:
deposition + modified-LBE collide-stream, interpolated EMMS drag with the
third-law rescale and integration, cell sort, hard-sphere collision
detection and resolution.  The same line carries the 2D riser section
(D2Q9 256 x 2048, 200,000 particles, mean 2D solid fraction 0.05) under
"riser2d", measured the same way.

Prints one JSON line (rank 0).  Metric: coupled-step MLUPS (cell updates per
second / 1e6), whole job over all ranks.  Multi-GPU runs are independent
replicas of the bed (weak scaling, no data-path collective).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Other modes, one JSON line each: --workload riser2d | bubbling2d (the 2D
riser alone, the small FP64 bubbling bed), --storage f16 | bf16 | f64, --serving
(continuous batching of a Poisson stream of beds against one-by-one FP32),
--precision (per-field error of each storage format against the FP64
oracle), --cfb (solids flux of the circulating-bed riser), --bubble (bubble
diameters of the Table 1 bed with a jet pulse), --dem [--dem-mu M] (the dense
soft-sphere bed, with friction for M > 0), --profile-steps N (build a bed and
run N steps, for ncu).
"""
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "coupled-step MLUPS"
UNIT = "MLUPS"
L2_FLUSH_BYTES = 512 * 1024 * 1024      # > 129 MB L2
KERNELS_PER_STEP = 7                    # collide_stream, drag_step, cell_scan, scatter,
                                        # gather, detect, resolve


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--storage", default="f32", choices=["f32", "f16", "bf16", "f64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--profile-steps", type=int, default=0,
                    help="only build the bed and run this many steps (for ncu captures); "
                         "no timing, no JSON line")
    ap.add_argument("--no-secondary", action="store_true",
                    help="with the 3D riser: skip the 2D riser line beside it")
    ap.add_argument("--workload", default="riser3d",
                    choices=["riser2d", "riser3d", "riser3d-128x128x512", "bubbling2d"])
    ap.add_argument("--serving", action="store_true",
                    help="serving benchmark: Poisson stream of independent beds")
    ap.add_argument("--requests", type=int, default=96)
    ap.add_argument("--rate", type=float, default=50.0)
    ap.add_argument("--max-active", type=int, default=128)
    ap.add_argument("--steps-per-tick", type=int, default=8)
    ap.add_argument("--no-serving", action="store_true",
                    help="leave the short serving summary out of the default bench line")
    ap.add_argument("--precision", action="store_true",
                    help="per-field error of FP32/FP16/BF16 storage against the FP64 oracle")
    ap.add_argument("--precision-steps", type=int, default=1000)
    ap.add_argument("--cfb", action="store_true",
                    help="circulating-bed riser of Table 2 with the solids loop closed: "
                         "solids flux through the outlet over time")
    ap.add_argument("--cfb-steps", type=int, default=60000)
    ap.add_argument("--bubble", action="store_true",
                    help="single-orifice bed of Table 1 with a 0.006 s jet pulse: equivalent "
                         "bubble diameter over time")
    ap.add_argument("--bubble-time", type=float, default=0.05)
    ap.add_argument("--bubble-cs", type=float, default=0.1,
                    help="Smagorinsky constant of the bubbling bed (Table 1's tau is 0.50089)")
    ap.add_argument("--dem", action="store_true",
                    help="dense soft-sphere bed (Table 1 particles, 256 x 1024 cells, lower half "
                         "packed): step time, kernel split and the contact kernel's roofline")
    ap.add_argument("--dem-steps", type=int, default=400)
    ap.add_argument("--dem-mu", type=float, default=0.0,
                    help="friction coefficient of the dense bed (0: normal contacts only; "
                         "> 0 adds friction with gamma_t = 0.05 m_p / dt and particle spin)")
    return ap.parse_args()


def workload(storage, name="riser2d"):
    from paper_1303_2653_gb300 import workloads as W
    st = {"f32": W.STORE_F32, "f16": W.STORE_F16, "bf16": W.STORE_BF16, "f64": W.STORE_F64}[storage]
    if name == "riser3d":
        return W.riser3d(storage=st)
    if name == "bubbling2d":
        # the small single-jet bed (64 x 128, 2,000 particles), FP64 as in
        # its table row unless another storage is asked for
        return W.bubbling2d(storage=st)
    if name == "riser3d-128x128x512":
        # the 3D riser at the same solid fraction on an eighth of the lattice
        # (1.6 GB of populations): the case ncu captures of the 3D kernels use
        return W.scaled_riser3d(nx=128, ny=128, nz=512, storage=st)
    return W.riser2d(storage=st)


def config_dict(w, n_gpus, storage):
    shape = "x".join(str(v) for v in w.n)
    lattice = "D2Q9" if w.dim == 2 else "D3Q19"
    return {"workload": f"{w.name.split('-')[0]} {lattice} {shape}, {w.n_particles} particles, "
                        f"{storage} population storage",
            "cells": w.ncell, "particles": w.n_particles, "lattice": lattice,
            "storage": storage, "l2": "flushed before each timed step (512 MB write, then 256 MB read)",
            "parallelism": f"replicas x{n_gpus}"}


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ roofline

def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def collide_stream_bytes(w, storage):
    """Algorithmic bytes of one collide_stream launch: populations read and
    written once, the cell_start offset, the node outputs (rho, u, F_p->g,
    beta) written once, and each particle velocity read once."""
    q = 9 if w.dim == 2 else 19
    s_f = {"f32": 4, "f16": 2, "bf16": 2, "f64": 8}[storage]
    s_r = 8 if storage == "f64" else 4
    # populations read and written, the cell-list offset read, and rho,
    # u_act[dim], F_p->g[dim], beta and 1 - eps written per cell
    per_cell = 2 * q * s_f + 4 + (3 + 2 * w.dim) * s_r
    per_particle = w.dim * s_r
    return w.ncell * per_cell + w.n_particles * per_particle, per_cell, per_particle


def drag_step_bytes(w, storage):
    """Algorithmic bytes of one drag_step launch: per particle the cell key,
    the FP64 position and the velocity and in-cell offset read, the same
    three written, the new key and its histogram count; per cell the node
    fields of the interpolation and the Eq. 28 rescale (rho, u_act[dim],
    F_p->g[dim], beta, 1 - eps) and the cell-list offset, each read once."""
    s_r = 8 if storage == "f64" else 4
    d = w.dim
    per_particle = 4 + 2 * (d * 8 + 2 * d * s_r) + 4 + 4
    per_cell = (3 + 2 * d) * s_r + 4
    return w.ncell * per_cell + w.n_particles * per_particle, per_cell, per_particle


def kernel_roofline(alg_bytes, ms, peak):
    """Achieved GB/s of a launch moving alg_bytes in ms, and its fraction of
    the peak (None when the kernel was not timed)."""
    if not ms or ms <= 0:
        return None
    achieved = alg_bytes / (ms / 1e3) / 1e9
    return {"achieved": achieved, "frac": achieved / peak, "ms": ms, "algorithmic_bytes": alg_bytes}


def profiled_traffic(workload_name):
    """DRAM bytes per collide_stream launch from the committed ncu summary of
    this workload, if it was taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", f"collide_stream_{workload_name}.md")
    src = os.path.join(ROOT, "paper_1303_2653_gb300", "csrc", "lbm_kernels.cu")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(r"source sha256:\s*([0-9a-f]{16})", text)
    t = re.search(r"dram bytes per launch:\s*([0-9.eE+]+)", text)
    if not m or not t:
        return None
    cur = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    return float(t.group(1)) if cur == m.group(1) else None


# ------------------------------------------------------------------ CPU oracle

def oracle_sample(full, max_cells=1_000_000):
    """The bed the CPU oracle is timed on, and its description: the full bed
    when it has at most max_cells cells, else a slab of it (the full cross
    section, fewer planes along the vertical axis, the same solid fraction);
    the oracle's cost per cell does not depend on the slab's height."""
    from paper_1303_2653_gb300 import workloads as W
    if full.ncell <= max_cells:
        return full.with_(storage=W.STORE_F64), "the full bed"
    plane = full.ncell // full.n[-1]
    nv = max(4, max_cells // plane)
    n_p = int(round(full.n_particles * nv / full.n[-1]))
    if full.dim == 2:
        sample = W.scaled_riser2d(nx=full.n[0], ny=nv, n_particles=n_p, storage=W.STORE_F64)
    else:
        sample = W.scaled_riser3d(nx=full.n[0], ny=full.n[1], nz=nv, n_particles=n_p,
                                  storage=W.STORE_F64)
    shape = "x".join(str(v) for v in sample.n)
    return sample, f"a {shape} slab of the bed ({n_p} particles, same solid fraction)"


def oracle_rate(w, budget_s):
    """Time the FP64 oracle (single thread) on the workload for about
    budget_s seconds; returns (MLUPS, steps, seconds)."""
    from oracle import oracle as O
    bed = O.OracleBed(w)
    t0 = time.perf_counter()
    bed.step(1)
    t1 = time.perf_counter()
    per = t1 - t0
    steps = max(1, int(budget_s / max(per, 1e-6)) - 1)
    t0 = time.perf_counter()
    bed.step(steps)
    dt = time.perf_counter() - t0
    return w.ncell * steps / dt / 1e6, steps, dt


def _oracle_worker(args):
    """One process of the all-cores oracle timing: build the bed, step it for
    about budget_s seconds, return (cell updates, seconds)."""
    w, budget_s = args
    from oracle import oracle as O
    bed = O.OracleBed(w)
    t0 = time.perf_counter()
    bed.step(1)
    per = time.perf_counter() - t0
    steps = max(1, int(budget_s / max(per, 1e-6)) - 1)
    t0 = time.perf_counter()
    bed.step(steps)
    return w.ncell * steps, time.perf_counter() - t0, steps


def oracle_rate_all_cores(w, budget_s, cores):
    """The FP64 oracle on every host core at once: `cores` independent
    one-thread processes (started with spawn), each stepping its own copy of
    the bed; returns (aggregate MLUPS, steps of one process, the slowest
    process's seconds)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        res = pool.map(_oracle_worker, [(w, budget_s)] * cores)
    slowest = max(r[1] for r in res)
    return sum(r[0] for r in res) / slowest / 1e6, min(r[2] for r in res), slowest


def max_over_ranks(x, dist=None, device="cuda"):
    """Max over all ranks of a per-rank figure (a time); barrier after."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def whole_job_mlups(world, cells, steps, seconds):
    """Cell updates of all ranks (each rank steps its own bed) per second / 1e6."""
    return world * cells * steps / seconds / 1e6


def reference_main(args, rank, world):
    """The oracle as the reference arm: K timed steps, each a bounded sample
    (a slab of the riser at the same solid fraction) so the run stays short."""
    from paper_1303_2653_gb300 import workloads as W
    from oracle import oracle as O
    if rank != 0:
        return
    full = workload(args.storage, args.workload)
    total = args.steps + args.warmup
    per_step_budget = 120.0 / max(total, 1)
    # oracle cost is close to 1.2 us per cell (2D) and at most 3 us (3D) at
    # these densities; the sample keeps the full cross-section and takes
    # fewer rows (planes) along the vertical axis, and only once that is at
    # its floor a smaller cross-section too, at the same solid fraction
    if full.dim == 2:
        cells = per_step_budget / 1.2e-6
        ny = int(max(8, min(full.n[1], cells / full.n[0])))
        nx = int(max(16, min(full.n[0], cells / ny)))
        sample = W.scaled_riser2d(nx=nx, ny=ny, n_particles=int(round(
            full.n_particles * nx * ny / full.ncell)), storage=W.STORE_F64)
    else:
        cells = per_step_budget / 3.0e-6
        plane = full.n[0] * full.n[1]
        nz = int(max(4, min(full.n[2], cells / plane)))
        side = min(1.0, math.sqrt(cells / (nz * plane)))
        nx = int(max(16, round(full.n[0] * side)))
        ny = int(max(16, round(full.n[1] * side)))
        sample = W.scaled_riser3d(nx=nx, ny=ny, nz=nz, n_particles=int(round(
            full.n_particles * nx * ny * nz / full.ncell)), storage=W.STORE_F64)
    bed = O.OracleBed(sample)
    bed.step(args.warmup)
    t0 = time.perf_counter()
    bed.step(args.steps)
    dt = time.perf_counter() - t0
    value = sample.ncell * args.steps / dt / 1e6
    shape = "x".join(str(v) for v in sample.n)
    desc = (f"{args.steps} oracle steps of a {shape} slab of the riser "
            f"({sample.n_particles} particles, same solid fraction)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / max(args.steps, 1) * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(full, args.gpus, args.storage),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ main

def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        reference_main(args, rank, world)
        return
    if args.serving:
        if rank == 0:
            serving_main(args)
        return
    if args.precision:
        if rank == 0:
            precision_main(args)
        return
    if args.cfb:
        if rank == 0:
            cfb_main(args)
        return
    if args.bubble:
        if rank == 0:
            bubble_main(args)
        return
    if args.dem:
        if rank == 0:
            dem_main(args)
        return

    import torch
    import __graft_entry__ as ge
    ge.build()
    from paper_1303_2653_gb300 import lbdps as L
    from paper_1303_2653_gb300 import workloads as W

    torch.cuda.set_device(local)
    if args.profile_steps:
        bed = L.Bed(workload(args.storage, args.workload))
        bed.step(args.profile_steps)
        bed.sync()
        bed.close()
        print(f"profile run ok: {args.profile_steps} steps", flush=True)
        return
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    w = workload(args.storage, args.workload)
    peak, peak_kind = measured_peaks()
    res = measure_bed(L, torch, w, args, dist, world, peak, peak_kind, with_e2e=not args.no_e2e)

    # the 2D riser beside the 3D headline: same timing rules, its own roofline
    secondary = None
    if args.workload == "riser3d" and not args.no_secondary:
        w2 = workload(args.storage, "riser2d")
        r2 = measure_bed(L, torch, w2, args, dist, world, peak, peak_kind, with_e2e=False)
        secondary = {"workload": config_dict(w2, world, args.storage)["workload"],
                     "value": r2["value"], "unit": UNIT, "ms_per_step": r2["ms_per_step"],
                     "particle_updates_per_s": r2["particle_updates_per_s"],
                     "roofline": r2["roofline"], "whole_step": r2["whole_step"],
                     "health": r2["health"]}

    # ---- a short serving run (rank 0, N = 1): 32 requests of the serving
    # stream, batched, on per-bed streams, and one by one in plain FP32 ----
    serving = None
    if rank == 0 and world == 1 and not args.no_serving:
        reqs = serving_requests(32, args.rate)
        free, _ = torch.cuda.mem_get_info()
        serving = serving_summary(L, W, reqs, int(0.5 * free), args.max_active,
                                  args.steps_per_tick)

    # ---- CPU oracle on the host cores (rank 0, N = 1) ----
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sample, what = oracle_sample(w)
        rate, n_st, secs = oracle_rate(sample, 15.0)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{n_st} FP64 oracle steps of {what} ({secs:.1f} s, one thread)"}
        cores = os.cpu_count() or 1
        if cores > 1:
            agg, steps_each, secs_all = oracle_rate_all_cores(sample, 10.0, cores)
            cpu["all_cores"] = {
                "value": agg, "unit": UNIT, "cores": cores, "kind": "oracle",
                "sample": f"{cores} independent one-thread oracle processes, each stepping "
                          f"{what} ({steps_each} steps in {secs_all:.1f} s); the aggregate "
                          f"cell updates per second"}

    if rank == 0:
        line = {"metric": METRIC, "value": res["value"], "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": res["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f64" if args.storage == "f64" else "f32",
                "data": "synthetic", "config": config_dict(w, world, args.storage),
                "roofline": res["roofline"], "whole_step": res["whole_step"],
                "cpu_baseline": cpu, "e2e": res["e2e"],
                "gpu_launches": KERNELS_PER_STEP * args.steps * world,
                "clocks": res["clocks"], "health": res["health"],
                "particle_updates_per_s": res["particle_updates_per_s"]}
        if secondary:
            line["riser2d"] = secondary
        if serving:
            line["serving"] = serving
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def whole_step_bytes(w, storage):
    """Algorithmic bytes of one coupled step: populations read and written
    once, per cell the cell-list offset and the node outputs read by the drag,
    per particle its state read and written in the drag and again in the
    sort.  Neighbour, stencil and halo re-reads are cache traffic, not
    counted."""
    q = 9 if w.dim == 2 else 19
    s_f = {"f32": 4, "f16": 2, "bf16": 2, "f64": 8}[storage]
    s_r = 8 if storage == "f64" else 4
    c_cell = 4 + (1 + 2 * w.dim) * s_r
    s_p = w.dim * 8 + w.dim * s_r
    return w.ncell * (2 * q * s_f + c_cell) + w.n_particles * 4 * s_p


E2E_RUNS = 5


def measure_bed(L, torch, w, args, dist, world, peak, peak_kind, with_e2e=True):
    """K timed steps of bed w (L2 flushed before each), the per-kernel-class
    times of profiled steps, and (optionally) the end-to-end run through the
    C ABI from host arrays."""
    bed = L.Bed(w)
    st = bed.stream
    # L2 flush between timed steps: write a buffer larger than L2, then read
    # a second one, so the write-backs of the flush itself happen before the
    # timed step (L2 is left holding clean lines of the read buffer)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    flush_rd = torch.ones(L2_FLUSH_BYTES // 8, dtype=torch.float32, device="cuda")

    def flush_l2():
        flush.zero_()
        flush_rd.sum()

    bed.step(args.warmup)
    bed.sync()

    # ---- timed region: K steps, L2 flushed (untimed) before each ----
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    time.sleep(0.3)
    with torch.cuda.stream(st):
        for k in range(args.steps):
            flush_l2()
            ev[k][0].record(st)
            bed.step(1)
            ev[k][1].record(st)
    torch.cuda.synchronize()
    clock_info = clocks.stop()
    total_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev), dist)
    health = bed.health()
    value = whole_job_mlups(world, w.ncell, args.steps, total_ms / 1e3)

    # ---- dominant-kernel roofline from per-kernel events (L2 flushed) ----
    prof_steps = min(args.steps, 200)
    acc = {}
    with torch.cuda.stream(st):
        for _ in range(prof_steps):
            flush_l2()
            torch.cuda._sleep(2_000_000)
            for k, v in bed.step_profiled(1).items():
                acc[k] = acc.get(k, 0.0) + v
    per_kernel_ms = {k: v / prof_steps for k, v in acc.items()}
    alg_bytes, per_cell, per_particle = collide_stream_bytes(w, args.storage)
    cs_ms = per_kernel_ms["collide_stream"]
    achieved = alg_bytes / (cs_ms / 1e3) / 1e9
    traffic = profiled_traffic(w.name.split("-")[0] + "_" + "x".join(str(v) for v in w.n))
    roofline = {"bound": "hbm", "kernel": "collide_stream", "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_kind,
                "traffic": traffic, "algorithmic_bytes": alg_bytes,
                "bytes_per_cell": per_cell, "bytes_per_particle": per_particle,
                "per_kernel_ms": per_kernel_ms}
    # the drag kernel against the same peak (in 3D the second largest share of
    # the step; in 2D about as long as collide_stream and bound by the
    # latency of dependent loads, not by bytes)
    roofline["drag"] = kernel_roofline(drag_step_bytes(w, args.storage)[0],
                                       per_kernel_ms.get("drag", 0.0), peak)
    ms_step = total_ms / args.steps
    ws_bytes = whole_step_bytes(w, args.storage)
    whole_step = {"algorithmic_bytes": ws_bytes, "ideal_ms": ws_bytes / (peak * 1e9) * 1e3,
                  "achieved": ws_bytes / (ms_step / 1e3) / 1e9,
                  "frac": ws_bytes / (ms_step / 1e3) / 1e9 / peak, "unit": "GB/s"}

    # ---- end to end through the C ABI from host buffers ----
    e2e = None
    if with_e2e:
        # E2E_RUNS complete runs; the median is reported (page faults of the
        # host's memory manager now and then add 10-20 ms to one run's
        # copies), every run's time is listed
        runs = []
        for _ in range(E2E_RUNS):
            torch.cuda.synchronize()
            if dist:
                dist.barrier()
            t0 = time.perf_counter()
            b2 = L.Bed(w)                      # H2D of the particle state from host arrays
            # every step: the step, its FP64 reductions and their copy to
            # pinned host memory, queued without a host wait between steps
            recs = b2.step_monitored(args.steps)
            assert len(recs) == args.steps and recs[-1]["steps"] == args.steps
            P, V = b2.particles()              # D2H of the final particle state
            b2.sync()
            runs.append(max_over_ranks(time.perf_counter() - t0, dist))
            b2.close()
            del P, V, recs
        t_e2e = sorted(runs)[len(runs) // 2]
        # bytes the caller's arrays hold: positions and velocities in FP64
        h2d = w.n_particles * w.dim * 8 * 2
        d2h_step = 13 * 8   # eleven FP64 statistics, the health word and the outlet count
        d2h_final = w.n_particles * w.dim * 8 * 2
        e2e = {"value": whole_job_mlups(world, w.ncell, args.steps, t_e2e), "unit": UNIT,
               "h2d_bytes_per_step": h2d / args.steps,
               "d2h_bytes_per_step": d2h_step + d2h_final / args.steps,
               "runs_ms": [round(r * 1e3, 2) for r in runs],
               "includes": "create from host arrays, K x (step + FP64 statistics copied to "
                           "host, pipelined: lbdps_step_monitored), final particle readback; "
                           f"median of {E2E_RUNS} complete runs"}
    bed.close()
    del flush, flush_rd
    torch.cuda.empty_cache()
    return {"value": value, "ms_per_step": ms_step, "roofline": roofline,
            "whole_step": whole_step, "e2e": e2e, "clocks": clock_info, "health": health,
            "particle_updates_per_s": world * w.n_particles * args.steps / (total_ms / 1e3)}



# ------------------------------------------------------------------ serving

def serving_requests(count, rate, seed=1303004):
    """Seeded stream of bed requests: Poisson arrivals at `rate` per second;
    bubbling or riser with p = 1/2; nx log-uniform in [64, 512] and ny in
    [128, 2048], both multiples of 32; particle count log-uniform in
    [1e3, 5e5], capped at a 2D area fraction of 0.25 in the particle region;
    step count log-uniform in [100, 5000]; FP16 or FP32 storage with p = 1/2;
    every bed runs the Smagorinsky model (Eq. 13-15) with C_s = 0.1, since
    tau is within 2e-3 of 1/2 in both templates."""
    import numpy as np
    from paper_1303_2653_gb300 import workloads as W
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, count))
    reqs = []
    lu = lambda lo, hi: float(np.exp(rng.uniform(np.log(lo), np.log(hi))))
    for i in range(count):
        kind = "bubbling" if rng.random() < 0.5 else "riser"
        nx = max(64, int(round(lu(64, 512) / 32)) * 32)
        ny = max(128, int(round(lu(128, 2048) / 32)) * 32)
        n = int(lu(1e3, 5e5))
        steps = int(lu(100, 5000))
        storage = W.STORE_F16 if rng.random() < 0.5 else W.STORE_F32
        if kind == "riser":
            h = 1.322e-4
            area = math.pi * (0.5 * 54e-6 / h) ** 2
            n = min(n, int(0.25 * nx * ny / area))
            w = W.riser2d(nx=nx, ny=ny, n_particles=n, seed=1303100 + i, storage=storage, h=h,
                          steps=steps, cs_smag=0.1)
        else:
            area = math.pi * (0.5 * 0.5e-3 / 2e-3) ** 2
            n = min(n, int(0.25 * 0.4 * nx * ny / area))
            w = W.bubbling2d(nx=nx, ny=ny, n_particles=n, seed=1303100 + i, storage=storage,
                             steps=steps, cs_smag=0.1)
        reqs.append((float(t[i]), w))
    return reqs


def serve(L, reqs, budget, max_active, steps_per_tick, batching):
    """Run the request stream through the server (arrivals replayed in real
    time); returns per-request latency (submit to completion), the records,
    the makespan and the batch counters."""
    import numpy as np
    server = L.Server(hbm_budget=budget, max_active=max_active, steps_per_tick=steps_per_tick,
                      batching=batching)
    ids, done, lat = {}, {}, {}
    nxt = 0
    t0 = time.perf_counter()
    while len(done) < len(reqs):
        now = time.perf_counter() - t0
        while nxt < len(reqs) and reqs[nxt][0] <= now:
            w = reqs[nxt][1]
            ids[server.submit(w, w.steps)] = nxt
            nxt += 1
        for r in server.poll(wait_s=0.0005):
            i = ids[r["id"]]
            done[i] = r
            lat[i] = (time.perf_counter() - t0) - reqs[i][0]
    makespan = time.perf_counter() - t0 - reqs[0][0]
    info = server.batch_info()
    server.close()
    return np.array([lat[i] for i in range(len(reqs))]), done, makespan, info


def one_by_one(L, W, reqs):
    """The same requests one by one in plain FP32 (FIFO in arrival order):
    latencies, mean voidage of each result, makespan."""
    import numpy as np
    import torch
    t_free, lat, eps = 0.0, [], []
    for arrival, w in reqs:
        b = L.Bed(w, storage=W.STORE_F32)
        torch.cuda.synchronize()
        s0 = time.perf_counter()
        b.step(w.steps)
        b.sync()
        dt = time.perf_counter() - s0
        eps.append(b.stats()["mean_eps_g"])
        b.close()
        begin = max(t_free, arrival)
        t_free = begin + dt
        lat.append(t_free - arrival)
    return np.array(lat), np.array(eps), t_free - reqs[0][0]


def serving_summary(L, W, reqs, budget, max_active, steps_per_tick, compare_streams=True):
    """Served (batched and, optionally, every bed on its own stream) against
    one by one in plain FP32, on the same request stream."""
    import numpy as np
    work = sum(w.ncell * w.steps for _, w in reqs)
    out = {"requests": len(reqs), "cell_updates": work,
           "fp16_requests": sum(1 for _, w in reqs if w.storage == W.STORE_F16)}
    modes = [("served_batched", True)] + ([("served_streams", False)] if compare_streams else [])
    eps_b = ok = None
    for key, batching in modes:
        lat, done, makespan, info = serve(L, reqs, budget, max_active, steps_per_tick, batching)
        failed = [{"request": i, "workload": reqs[i][1].name, "status": done[i]["status"],
                   "health": done[i].get("health")}
                  for i in range(len(reqs)) if done[i]["status"] != 0]
        out[key] = {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                    "aggregate_mlups": work / makespan / 1e6, "makespan_s": makespan,
                    "failed": len(failed), "failed_requests": failed}
        if batching:
            out[key]["batch_ticks"], out[key]["graph_captures"] = info[0], info[1]
            eps_b = np.array([done[i]["mean_eps_g"] for i in range(len(reqs))])
            ok = np.array([done[i]["status"] == 0 for i in range(len(reqs))])
    lat1, eps1, make1 = one_by_one(L, W, reqs)
    out["one_by_one_fp32"] = {"p50_s": float(np.percentile(lat1, 50)),
                              "p99_s": float(np.percentile(lat1, 99)),
                              "aggregate_mlups": work / make1 / 1e6, "makespan_s": make1}
    rel = (np.abs(eps_b - eps1) / eps1)[ok]
    out["served_vs_fp32_alone"] = {"mean_voidage_rel_err_max": float(rel.max()),
                                   "mean_voidage_rel_err_mean": float(rel.mean())}
    return out


def serving_main(args):
    import torch
    import __graft_entry__ as ge
    ge.build()
    from paper_1303_2653_gb300 import lbdps as L
    from paper_1303_2653_gb300 import workloads as W

    torch.cuda.set_device(0)
    reqs = serving_requests(args.requests, args.rate)
    free, total = torch.cuda.mem_get_info()
    budget = int(0.5 * free)
    summ = serving_summary(L, W, reqs, budget, args.max_active, args.steps_per_tick)
    line = {"metric": "served p50/p99 time-to-K-steps and aggregate MLUPS", "unit": "s / MLUPS",
            "rate_per_s": args.rate, "data": "synthetic", "budget_bytes": budget,
            "max_active": args.max_active, "steps_per_tick": args.steps_per_tick}
    line.update(summ)
    line["small_beds"] = small_beds_summary(L, W, budget, args.max_active, args.steps_per_tick)
    print(json.dumps(line), flush=True)


def small_beds_summary(L, W, budget, max_active, steps_per_tick, n=64, steps=500):
    """n small riser beds (64 x 128, about 3,100 particles, FP32 and FP16
    alternating, C_s = 0.1) submitted at once: the case the batched kernels
    are for (each bed's own launches are latency-bound)."""
    reqs = [(0.0, W.scaled_riser2d(nx=64, ny=128, seed=1303300 + i, steps=steps, cs_smag=0.1,
                                   storage=W.STORE_F16 if i % 2 else W.STORE_F32))
            for i in range(n)]
    work = sum(w.ncell * w.steps for _, w in reqs)
    out = {"beds": n, "cells_per_bed": reqs[0][1].ncell, "steps": steps}
    for key, batching in (("batched", True), ("streams", False)):
        lat, done, makespan, info = serve(L, reqs, budget, max_active, steps_per_tick, batching)
        out[key] = {"aggregate_mlups": work / makespan / 1e6, "makespan_s": makespan,
                    "failed": sum(1 for r in done.values() if r["status"] != 0)}
    return out



# ------------------------------------------------------------------ precision table

def precision_main(args):
    """Per-field error of FP32, FP16 and BF16 population storage against the
    FP64 oracle on the riser (scaled to a lattice the oracle steps quickly),
    after 1 step and after args.precision_steps steps, all started from the
    same description.  After many steps the particle trajectories are
    chaotic, so bed-averaged quantities are reported beside the pointwise
    errors."""
    import numpy as np
    import torch
    import __graft_entry__ as ge
    ge.build()
    from oracle import oracle as O
    from paper_1303_2653_gb300 import lbdps as L
    from paper_1303_2653_gb300 import workloads as W

    torch.cuda.set_device(0)
    w = W.scaled_riser2d(nx=64, ny=512, seed=1303002)
    mask = L.FIELD_RHO | L.FIELD_U | L.FIELD_FPG | L.FIELD_VS | L.FIELD_NTOT | L.FIELD_EPS_G
    names = {"f64": W.STORE_F64, "f32": W.STORE_F32, "f16": W.STORE_F16, "bf16": W.STORE_BF16}
    beds = {k: L.Bed(w, storage=v, diagnostics=True) for k, v in names.items()}
    ob = O.OracleBed(w)
    table = {}
    done = 0
    for target in (1, args.precision_steps):
        ob.step(target - done)
        for b in beds.values():
            b.step(target - done)
        done = target
        ref = {"rho": ob.field(O.F_RHO), "u": ob.field(O.F_U), "fpg": ob.field(O.F_FPG),
               "vs": ob.field(O.F_VS), "eps_g": ob.field(O.F_EPS_G)}
        Po, vo = ob.particles()
        so = ob.stats()
        row = {}
        for k, b in beds.items():
            g = b.fields(mask)
            Pg, vg = b.particles()
            st = b.stats()
            e = {f: float(np.abs(g[f] - ref[f]).max() / max(np.abs(ref[f]).max(), 1e-300))
                 for f in ("u", "fpg", "vs")}
            e["rho_abs"] = float(np.abs(g["rho"] - ref["rho"]).max())
            e["eps_g_abs"] = float(np.abs(g["eps_g"] - ref["eps_g"]).max())
            e["P_abs_max"] = float(np.abs(Pg - Po).max())
            e["v"] = float(np.abs(vg - vo).max() / np.abs(vo).max())
            e["mean_eps_g_rel"] = float(abs(st["mean_eps_g"] - so["mean_eps_g"]) / so["mean_eps_g"])
            e["mean_slip_rel"] = float(abs(st["mean_slip"] - so["mean_slip"]) / so["mean_slip"])
            e["mass_rel"] = float(abs(st["mass"] - so["mass"]) / so["mass"])
            row[k] = e
        table[f"after_{target}_steps"] = row
    line = {"metric": "per-field error against the FP64 oracle", "workload":
            f"riser2d D2Q9 {w.n[0]}x{w.n[1]}, {w.n_particles} particles", "table": table,
            "note": "u, fpg, vs, v: max|d|/max|oracle|; rho, eps_g: max|d|; P: max|d| in cells; "
                    "mean_*: relative error of the lattice/particle averages"}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ circulating bed

def cfb_main(args):
    """The riser of Table 2 (60 x 720, 123,921 particles, inlet 1.52 m/s,
    outlet at the top, solids loop closed, C_s = 0.1) run for args.cfb_steps
    steps: the solids flux through the outlet, G_s = (particles out) m_p /
    (outlet area x time), per window of 5,000 steps, with the outlet area the
    bed width times the cell depth h (a 2D cell is h deep)."""
    import numpy as np
    import torch
    import __graft_entry__ as ge
    ge.build()
    from paper_1303_2653_gb300 import lbdps as L
    from paper_1303_2653_gb300 import workloads as W

    torch.cuda.set_device(0)
    w = W.cfb_riser2d(steps=args.cfb_steps)
    bed = L.Bed(w)
    m_p = w.rho_s * math.pi * w.d_p ** 3 / 6.0
    area = w.n[0] * w.h * w.h
    window = 5000
    series, t_dev = [], 0.0
    prev = bed.stats()["solids_out"]
    st = bed.stream
    done = 0
    while done < args.cfb_steps:
        k = min(window, args.cfb_steps - done)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        bed.step(k)
        b.record(st)
        s = bed.stats()
        t_dev += a.elapsed_time(b) / 1e3
        done += k
        n_out = s["solids_out"] - prev
        prev = s["solids_out"]
        series.append({"t_s": done * w.dt, "flux_kg_m2s": n_out * m_p / (area * k * w.dt),
                       "health": s["health"]})
        if s["health"]:
            break
    half = [x["flux_kg_m2s"] for x in series[len(series) // 2:]]
    line = {"metric": "solids flux through the outlet of the circulating-bed riser",
            "unit": "kg/(m^2 s)", "workload": f"{w.name}, C_s = {w.cs_smag}, dt = {w.dt:.3e} s",
            "data": "synthetic", "steps": done, "physical_time_s": done * w.dt,
            "mean_flux_second_half": float(np.mean(half)) if half else None,
            "series": series, "mlups": w.ncell * done / t_dev / 1e6,
            "note": "the paper reports 13.8 kg/(m^2 s) from its own (longer) run, §3.2; context only"}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ bubbling bed

def bubble_main(args):
    """The bed of Table 1 (25 x 100, 15,000 particles, background inlet
    0.0025 m/s) with the jet of 0.8 m/s on the central three cells for
    0.006 s (§3.1), then the background only; every 100 steps the equivalent
    diameter D_e = 2 h sqrt(A / pi) of the largest region with eps_2d > 0.85
    below the bed surface (lbdps_bubbles)."""
    import torch
    import __graft_entry__ as ge
    ge.build()
    from paper_1303_2653_gb300 import lbdps as L
    from paper_1303_2653_gb300 import workloads as W

    torch.cuda.set_device(0)
    # LES on: tau is 0.50089 in Table 1 (reading R20)
    w = W.bubbling_table1(cs_smag=args.bubble_cs)
    bed = L.Bed(w, check_every=100)
    pulse = int(round(0.006 / w.dt))
    total = int(round(args.bubble_time / w.dt))
    every = 100
    series, best = [], (0.0, 0.0)
    st = bed.stream
    t_dev, done = 0.0, 0
    while done < total:
        k = min(every, total - done)
        if done < pulse <= done + k:        # end the pulse exactly at step `pulse`
            k = pulse - done
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        try:
            bed.step(k)
        except L.LbdpsError as err:       # diverged: report how far it got
            series.append({"t_s": done * w.dt, "stopped": str(err)})
            break
        b.record(st)
        bub = bed.bubbles(0.85, L.VOIDAGE_2D)
        t_dev += a.elapsed_time(b) / 1e3
        done += k
        if done == pulse:
            bed.set_inlet(W.background_inlet(w))
        de = 2.0 * w.h * math.sqrt(bub["largest"] / math.pi)
        series.append({"t_s": done * w.dt, "de_m": de, "regions": bub["count"]})
        if de > best[0]:
            best = (de, done * w.dt)
    line = {"metric": "maximum equivalent bubble diameter, single-orifice bed", "unit": "m",
            "value": best[0], "at_s": best[1],
            "workload": f"{w.name}, jet 0.8 m/s for 0.006 s, C_s = {w.cs_smag}",
            "data": "synthetic", "steps": done, "health": bed.health(),
            "mlups": w.ncell * done / t_dev / 1e6,
            "series": series[::10] + series[-1:]}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------- soft spheres

def contact_bytes(w, storage, friction=False):
    """Algorithmic bytes of one soft-sphere contact launch, per particle: its
    cell index, in-cell offsets and velocity read once, the contact force
    written once, and the cell-list entries of its 3 (2D) or 9 (3D)
    neighbour rows (two ints each).  Reads of the neighbours' state are
    re-reads of the same arrays (served by L1/L2) and are not counted, nor
    are the FP64 positions, which only pairs within the exact-test band and
    particles next to a face read."""
    r = 8 if storage == "f64" else 4
    d = w.dim
    rows = 3 if d == 2 else 9
    per_particle = 4 + d * r + d * r + d * r + rows * 2 * 4
    if friction:   # spin read and the new spin written
        per_particle += 2 * (1 if d == 2 else 3) * r
    return per_particle * len(w.pos)


def dem_main(args):
    """Dense soft-sphere bed: Table 1 particles (54 um, 930 kg/m^3, h = 2.7e-4
    m, dt = 1.35e-6 s) packed to an area fraction of 0.35 in the lower half of
    a closed 256 x 1024 box, centres at least 0.9 d_p apart (many start in
    contact), pair contacts 20 steps long, e = 0.7."""
    import numpy as np
    import torch
    import __graft_entry__ as ge
    ge.build()
    from paper_1303_2653_gb300 import lbdps as L
    from paper_1303_2653_gb300 import workloads as W

    torch.cuda.set_device(0)
    storage = args.storage
    st_code = {"f32": W.STORE_F32, "f16": W.STORE_F16, "bf16": W.STORE_BF16,
               "f64": W.STORE_F64}[storage]
    w = W.packed_bed(dim=2, n=(256, 1024), storage=st_code, cs_smag=0.1)
    if args.dem_mu > 0:
        w = W.with_friction(w, mu=args.dem_mu, gamma_frac=0.05)
    bed = L.Bed(w, check_every=0)
    st = bed.stream
    bed.step(max(args.warmup, 3))
    bed.sync()
    clocks = ClockSampler(0)
    clocks.start()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(st)
    bed.step(args.dem_steps)
    b.record(st)
    b.synchronize()
    clk = clocks.stop()
    t = a.elapsed_time(b) / 1e3
    prof_steps = 50
    ms = bed.step_profiled(prof_steps)
    peak, peak_kind = measured_peaks()
    t_contact = ms["collide_particles"] / 1e3 / prof_steps
    nb = contact_bytes(w, storage, friction=args.dem_mu > 0)
    ach = nb / t_contact / 1e9
    s = bed.stats()
    line = {"metric": "dense soft-sphere bed: coupled step throughput", "unit": "MLUPS",
            "value": w.ncell * args.dem_steps / t / 1e6,
            "particle_updates_per_s": len(w.pos) * args.dem_steps / t,
            "ms_per_step": 1e3 * t / args.dem_steps, "steps": args.dem_steps,
            "warmup": max(args.warmup, 3), "dtype": {"f64": "f64"}.get(storage, "f32"),
            "storage": storage, "data": "synthetic",
            "config": {"workload": w.name, "cells": w.ncell, "particles": len(w.pos),
                       "contact_steps": 20, "e": w.e, "cs_smag": w.cs_smag,
                       "friction_mu": w.dem_mu, "gamma_t_kg_s": w.dem_gamma_t},
            "kernel_ms_per_step": {k: v / prof_steps for k, v in ms.items()},
            "roofline_contacts": {"bound": "hbm", "achieved": ach, "peak": peak,
                                  "peak_kind": peak_kind, "unit": "GB/s", "frac": ach / peak,
                                  "bytes_per_launch": nb,
                                  "limiter": "instruction issue: the walk over the candidates "
                                             "of the cells within reach"},
            "health": s["health"], "clocks": clk}
    print(json.dumps(line), flush=True)
    bed.close()


if __name__ == "__main__":
    main()
