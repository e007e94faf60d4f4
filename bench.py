"""Benchmark of the TreeRay/OnTheSpot hot path on GB300.

One step = one pass of the whole hot path over the turbulent-cloud workload
(128^3 cells, 10 point sources, N_PIX = 48, theta_lim = 0.5): source mapping,
per-cell netting and tree build (tr_build_tree), then walk + node->ray
mapping + far-to-near sweep + sum over rays for every cell (tr_walk_sweep).
The headline `value` is target-cell-rays/s of the FP32 + FP64-sweep form
(FP32 node moments and deposits, every segment of the sweep in FP64) with
inputs resident in HBM; the plain FP64 form and the FP32 + double-FP32-sweep
form are timed beside it.  `e2e` is the same metric through tr_solve with
host buffers (host->device copy of the inputs and device->host copy of the
flux inside the timed region).  The other workloads (the Stromgren test, the
AMR cluster, the 256^3 source-count series) are timed once each under
`configs`, and a Poisson stream of requests through the serving loop under
`serving`.  The CPU oracle is timed on a bounded sample of the workload.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
python bench.py --walk-only --workload W --precision P --reps R   (profiling:
    build once, then R launches of the fused walk kernel, nothing else)
python bench.py --sweep-only --workload W --precision P --targets T --reps R
    (profiling: walk and map T sampled cells once into stored ray bins,
    then R launches of the stored-bins sweep)
Under torchrun every rank solves its own copy of the workload (independent
problems, weak scaling); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "target-cell-rays/s at N_PIX=48 (FP32+FP64-sweep vs plain FP64); p50/p99 latency"
UNIT = "cell-rays/s"
WORKLOAD = "turbulent128"
FORM_NAMES = {0: "plain FP64", 1: "FP32 moments and deposits + FP64 sweep",
              2: "FP32 moments and deposits + double-FP32 sweep"}
EXTRA_CONFIGS = ("stromgren32", "amr_cluster", "sourcecount256_s1", "sourcecount256_s100",
                 "sourcecount256_s10000", "diffuse256")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--cpu-sample", type=int, default=300000,
                    help="targets in the CPU-oracle sample (about 10-15 s of oracle work on 16 cores)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--fp64-steps", type=int, default=None)
    ap.add_argument("--serving", type=int, default=40,
                    help="requests in the continuous-batching serving run (0 skips it)")
    ap.add_argument("--serving-sizes", default="32,64,128,256")
    ap.add_argument("--serving-nsides", default="2,4")
    ap.add_argument("--serving-load", type=float, default=0.8,
                    help="Poisson arrival rate as a fraction of the measured single-stream capacity")
    ap.add_argument("--configs", default="all", help="'all', 'none' or a comma list of extra workloads to time")
    ap.add_argument("--walk-only", action="store_true", help="profiling: R launches of the fused walk only")
    ap.add_argument("--precision", type=int, default=1, help="--walk-only: tr_precision of the tree")
    ap.add_argument("--reps", type=int, default=2, help="--walk-only / --sweep-only: launches")
    ap.add_argument("--sweep-only", action="store_true",
                    help="profiling: R launches of the stored-bins sweep over a sample of targets")
    ap.add_argument("--targets", type=int, default=65536, help="--sweep-only: sampled targets")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------- ranks

def reduce_max(x: float, world: int, device=None) -> float:
    """Max of x over all ranks (the slowest rank sets the job's time)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: int, steps: int, max_total_ms: float, world: int) -> float:
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return world * units_per_rank * steps / (max_total_ms * 1e-3)


# ---------------------------------------------------------------- CPU oracle

def _oracle_worker(args):
    name, targets = args
    sys.path.insert(0, ROOT)
    import oracle
    from workloads import workload
    w = workload(name)
    t = oracle.Tree(w)
    p = oracle.params_for(w)
    t0 = time.perf_counter()
    t.solve_pass(p, targets=targets)
    return time.perf_counter() - t0


def cpu_baseline(name, n_targets, pool):
    """Oracle walk + map + sweep on a seeded random sample of targets, split
    over the host cores; the tree build of each worker is not timed."""
    import numpy as np
    from workloads import workload
    w = workload(name)
    rng = np.random.default_rng(2105)
    targets = np.sort(rng.choice(w.N ** 3, size=n_targets, replace=False)).astype(np.int64)
    nproc = pool._processes if pool is not None else 1
    chunks = [(name, c) for c in np.array_split(targets, nproc)]
    t0 = time.perf_counter()
    if pool is None:
        times = [_oracle_worker(chunks[0])]
    else:
        times = pool.map(_oracle_worker, chunks)
    wall = max(times)
    return dict(value=n_targets * w.npix / wall, unit=UNIT, cores=nproc, kind="oracle",
                sample=f"{n_targets} seeded random target cells of {name} ({w.N}^3, N_PIX={w.npix}), "
                       f"FP64 oracle walk+map+sweep, split over {nproc} processes; tree build not timed",
                seconds=wall, wall_total=time.perf_counter() - t0)


# ---------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.samples = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) == 7:
                self.samples.append(parts)

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


# ---------------------------------------------------------------- our arm

def walk_profile(name, kernel_src_sha):
    """Per-launch counters of the walk from a committed ncu summary
    (profiles/<name>.json), if it was taken on the current walk source."""
    try:
        d = json.load(open(os.path.join(ROOT, "profiles", name)))
    except (OSError, ValueError):
        return None
    return d if d.get("kernel_source_sha256") == kernel_src_sha else None


def walk_src_sha():
    return hashlib.sha256(open(os.path.join(ROOT, "paper_2105_09644_gb300", "csrc", "tr_walk.cu"), "rb").read()).hexdigest()


def make_problem(B, name, devn):
    """Device inputs, grid/source structs, output buffers and parameters of a
    named workload (uniform grids and the AMR cluster)."""
    import numpy as np
    import torch
    if name.startswith("amr"):
        from workloads.amr import amr_cluster
        w = amr_cluster(N_base=16) if name == "amr_mid" else amr_cluster()
        n = torch.from_numpy(np.ascontiguousarray(w.n_H.ravel())).to(devn)
        grid = B.make_amr_grid(w.N_base, w.max_level, w.blk_level, w.blk_pos, n, w.dx_fine)
        build = B.tr_build_tree_amr
        shape, ncell = (w.n_leaves,), w.n_leaves
    else:
        from workloads import workload
        w = workload(name)
        n = torch.from_numpy(np.ascontiguousarray(w.n_H)).to(devn)
        nd = torch.from_numpy(np.ascontiguousarray(w.ndot_cell)).to(devn) if w.ndot_cell is not None else None
        grid = B.make_grid(n, w.dx, ndot=nd)
        build = B.tr_build_tree
        shape, ncell = (w.N,) * 3, w.N ** 3
    x = torch.from_numpy(np.ascontiguousarray(w.src_xyz)).to(devn)
    q = torch.from_numpy(np.ascontiguousarray(w.src_Q)).to(devn)
    src = B.make_sources(x, q)
    out = dict(F=torch.empty(shape, dtype=torch.float64, device=devn))
    out["E"] = torch.empty_like(out["F"])
    out["ion"] = torch.empty(shape, dtype=torch.uint8, device=devn)

    def params(prec):
        return B.tr_params_default(theta_lim=w.theta_lim, theta_if=w.theta_if, theta_src=w.theta_src,
                                   nside=w.nside, eta_r=w.eta_r, alpha_B=w.alpha_B, hnu=w.hnu, precision=prec)
    keep = [grid, n, x, q] + ([nd] if not name.startswith("amr") else [])
    return dict(w=w, grid=grid, src=src, build=build, out=out, params=params, ncell=ncell, keep=keep)


def run_walk_only(args):
    """Profiling entry: build the tree once, then `reps` launches of the
    fused walk kernel (CUDA events around each); prints the counters."""
    import torch
    import paper_2105_09644_gb300 as pkg
    pkg.build()
    from paper_2105_09644_gb300 import binding as B
    devn = torch.device("cuda", 0)
    pr = make_problem(B, args.workload, devn)
    tree = pr["build"](pr["grid"], pr["src"], pr["params"](args.precision))
    o = pr["out"]
    ms = []
    for _ in range(args.reps):
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record()
        B.tr_walk_sweep(tree, o["F"], o["E"], o["ion"])
        s1.record()
        torch.cuda.synchronize()
        ms.append(s0.elapsed_time(s1))
    print(json.dumps({"workload": args.workload, "precision": args.precision, "form": FORM_NAMES[args.precision],
                      "counters": B.tr_tree_stats(tree), "tree": tree.info(), "ms_per_launch": ms}), flush=True)


def run_sweep_only(args):
    """Profiling entry for the sweep alone: walk and map a seeded sample of
    `targets` cells once into stored ray bins (tr_walk_map), then `reps`
    launches of the stored-bins sweep (tr_ray_sweep, CUDA events around
    each)."""
    import torch
    import paper_2105_09644_gb300 as pkg
    pkg.build()
    from paper_2105_09644_gb300 import binding as B
    devn = torch.device("cuda", 0)
    pr = make_problem(B, args.workload, devn)
    tree = pr["build"](pr["grid"], pr["src"], pr["params"](args.precision))
    g = torch.Generator().manual_seed(5)
    tg = torch.randint(0, pr["ncell"], (args.targets,), generator=g, dtype=torch.int64).to(devn)
    rays = B.tr_walk_map(tree, targets=tg)
    F = torch.empty(args.targets, dtype=torch.float64, device=devn)
    ms = []
    for _ in range(args.reps):
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record()
        B.tr_ray_sweep(rays, F)
        s1.record()
        torch.cuda.synchronize()
        ms.append(s0.elapsed_time(s1))
    print(json.dumps({"workload": args.workload, "precision": args.precision, "form": FORM_NAMES[args.precision],
                      "targets": args.targets, "tree": tree.info(), "sweep_ms_per_launch": ms}), flush=True)


def l2_copy_peak(devn, mb=32, reps=20):
    """L2 bandwidth ceiling: device copies between two `mb` MB buffers that
    stay resident in the 129 MB L2 (read + write bytes), `reps` of them
    captured in one CUDA graph so that they run back to back with no host
    launch gaps; best of 10 replays.  Each copy still pays a kernel
    boundary, so this is a lower bound on the ceiling (and the fraction
    against it an upper bound)."""
    import torch
    a = torch.ones(mb << 18, dtype=torch.float32, device=devn)
    b = torch.empty_like(a)
    side = torch.cuda.Stream(device=devn)
    side.wait_stream(torch.cuda.current_stream(devn))
    with torch.cuda.stream(side):
        for _ in range(3):
            b.copy_(a)
    torch.cuda.current_stream(devn).wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        for _ in range(reps):
            b.copy_(a)
    g.replay()
    torch.cuda.synchronize()
    best = math.inf
    for _ in range(10):
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record()
        g.replay()
        s1.record()
        torch.cuda.synchronize()
        best = min(best, s0.elapsed_time(s1) / reps)
    return 2 * a.numel() * 4 / (best * 1e-3) / 1e9


def launches_per_build(N, mode):
    """Kernels of one tr_build_tree: emission init, sources, FP64 leaves and
    log2 N parent levels; in the FP32 forms also FP32 leaves, parents and the
    finalize pass."""
    L = int(round(math.log2(N)))
    return 2 + (1 + L) + ((1 + L + 1) if mode != 0 else 0)


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    if args.sweep_only:
        run_sweep_only(args)
        return
    if args.walk_only:
        run_walk_only(args)
        return
    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    devn = torch.device("cuda", local)
    pool = None
    if rank == 0 and world == 1 and not args.no_cpu:
        import multiprocessing as mp
        pool = mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1))

    import paper_2105_09644_gb300 as pkg
    pkg.build()
    from paper_2105_09644_gb300 import binding as B

    pr = make_problem(B, args.workload, devn)
    w = pr["w"]
    N = w.N
    ncell = N ** 3
    units = ncell * w.npix                               # cell-rays per step
    host = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory()
            for k, v in (("n_H", w.n_H), ("xyz", w.src_xyz), ("Q", w.src_Q))}
    d = {k: v.to(devn) for k, v in host.items()}
    o = pr["out"]
    F, E, ion = o["F"], o["E"], o["ion"]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=devn)   # > L2 (129 MB)
    stream = torch.cuda.current_stream()
    grid = B.make_grid(d["n_H"], w.dx)
    src = B.make_sources(d["xyz"], d["Q"])
    params = pr["params"]

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()

    def timed_device(prec, steps, warmup):
        p = params(prec)
        tree = B.Tree()
        for _ in range(warmup):
            B.tr_build_tree(grid, src, p, tree)
            B.tr_walk_sweep(tree, F, E, ion)
        barrier()
        step_ms, walk_ms = [], []
        for _ in range(steps):
            flush.zero_()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            ev[0].record(stream)
            B.tr_build_tree(grid, src, p, tree)
            ev[1].record(stream)
            B.tr_walk_sweep(tree, F, E, ion)
            ev[2].record(stream)
            torch.cuda.synchronize()
            step_ms.append(ev[0].elapsed_time(ev[2]))
            walk_ms.append(ev[1].elapsed_time(ev[2]))
        barrier()
        return dict(step_ms=step_ms, walk_ms=walk_ms, stats=B.tr_tree_stats(tree), info=tree.info())

    def max_over_ranks(x):
        return reduce_max(x, world, devn)

    def form_summary(prec, r, k):
        ms = max_over_ranks(sum(r["step_ms"])) / k
        return {"form": FORM_NAMES[prec], "value": world * units / (ms * 1e-3), "ms_per_step": ms,
                "walk_ms": statistics.mean(r["walk_ms"]), "p50_ms": statistics.median(r["step_ms"]),
                "p99_ms": percentile(r["step_ms"], 99), "steps": k,
                "fp64_redecided": {"mac": r["stats"]["fp64_mac"], "setup": r["stats"]["fp64_setup"],
                                   "of_visited": r["stats"]["visited"]}}

    # headline: FP32 moments and deposits + FP64 sweep, inputs resident
    with ClockSampler(local) as clk:
        r1 = timed_device(1, args.steps, args.warmup)
    total_ms = max_over_ranks(sum(r1["step_ms"]))
    ms_per_step = total_ms / args.steps
    value = job_rate(units, args.steps, total_ms, world)

    # the other two forms beside it
    k_other = args.fp64_steps if args.fp64_steps is not None else max(2, min(args.steps, 3))
    r0 = timed_device(0, k_other, max(1, min(args.warmup, 2)))
    r2 = timed_device(2, max(2, min(args.steps, 5)), max(1, min(args.warmup, 2)))

    # end to end through tr_solve with host buffers
    p1 = params(1)
    F_host = torch.empty((N, N, N), dtype=torch.float64).pin_memory()

    def e2e_step():
        for k in d:
            d[k].copy_(host[k], non_blocking=True)
        B.tr_solve(grid, src, p1, F, E, ion)
        F_host.copy_(F, non_blocking=True)

    for _ in range(args.warmup):
        e2e_step()
    barrier()
    e2e_ms = []
    for _ in range(args.steps):
        flush.zero_()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        e2e_step()
        s1.record(stream)
        torch.cuda.synchronize()
        e2e_ms.append(s0.elapsed_time(s1))
    e2e_total = max_over_ranks(sum(e2e_ms))
    h2d = sum(v.numel() * v.element_size() for v in host.values())
    d2h = F_host.numel() * F_host.element_size()

    if world > 1:
        dist.barrier()
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    # roofline of the dominant kernel (the fused walk + map + sweep)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm_peak = peaks.get("hbm_gbs")
    hbm_src = "measured" if hbm_peak else "fallback"
    hbm_peak = hbm_peak or 6800.0
    sm_max = peaks.get("sm_max_mhz") or 2070.0
    l2_peak = l2_copy_peak(devn)
    st = r1["stats"]
    alg_bytes = st["visited"] * 32 + st["accepted"] * 8 + st["entries"] * 4 + ncell * (8 + 8 + 1)
    walk_s = statistics.mean(r1["walk_ms"]) * 1e-3
    achieved = alg_bytes / walk_s / 1e9
    sha = walk_src_sha()
    prof = walk_profile("walk_turbulent128_fp32_sweep64.json", sha) if args.workload == WORKLOAD else None
    traffic = prof.get("dram_bytes_per_launch") if prof else None
    inst = prof.get("warp_instructions_per_launch") if prof else None
    issue_peak = 152 * 4 * sm_max * 1e6                   # warp instructions per second (4 schedulers per SM)
    hbm = {"achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
           "peak_source": f"{hbm_src} hbm_gbs (MEASURED_PEAKS.json)"}
    l2 = {"achieved": achieved, "peak": l2_peak, "unit": "GB/s", "frac": achieved / l2_peak,
          "peak_source": "measured in this run: 20 device copies between two 32 MB L2-resident buffers in "
                         "one CUDA graph (a lower bound on the L2 ceiling)"}
    issue = None
    if inst:
        ia = inst / walk_s / 1e9
        issue = {"achieved": ia, "peak": issue_peak / 1e9, "unit": "G warp-instructions/s", "frac": ia / (issue_peak / 1e9),
                 "instructions_per_launch": inst, "peak_source": "152 SMs x 4 schedulers x 1 warp-instruction/clock "
                 f"x {sm_max:.0f} MHz (MEASURED_PEAKS.json sm_max_mhz); instructions from ncu smsp__inst_executed.sum"}
    if issue:
        roof = {"bound": "alu", "achieved": issue["achieved"], "peak": issue["peak"], "unit": issue["unit"],
                "frac": issue["frac"]}
    else:
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak}
    roof.update({"traffic": traffic, "binds": "instruction issue (the tree is L2-resident: DRAM carries it once)"
                 if issue else "unmeasured issue rate: HBM fraction shown",
                 "issue": issue, "l2": l2, "hbm": hbm,
                 "kernel": "k_walk<1, fused, 128, default> (walk + map + FP64 sweep, FP32 moments)",
                 "algorithmic_bytes_per_launch": alg_bytes, "walk_ms": statistics.mean(r1["walk_ms"]),
                 "counters": st})
    launches = (launches_per_build(N, 1) + 1) * args.steps
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": workload_name(w, r1["info"]["nr"]),
                   "precision": "FP32 node moments (Kahan-Neumaier over children, centre of mass as an offset from "
                                "the node centre), FP32 ray deposits summed exactly in 64-bit fixed point, every "
                                "segment of the sweep (R_ij, Phi_j, clipping) in FP64; opening decisions FP32 cannot "
                                "settle re-taken in FP64 (accepted lists identical to the FP64 form)",
                   "l2": "flushed (256 MB write) before every timed step",
                   "parallelism": f"independent problem per GPU x{world}"},
        "latency_ms": {"p50": statistics.median(r1["step_ms"]), "p99": percentile(r1["step_ms"], 99),
                       "note": "over the timed steps; see solve_latency_ms and the serving block for distributions"},
        "forms": {"fp32_sweep64": form_summary(1, r1, args.steps), "fp64": form_summary(0, r0, k_other),
                  "fp32_sweepdf": form_summary(2, r2, max(2, min(args.steps, 5)))},
        "plain_fp64": form_summary(0, r0, k_other),
        "e2e": {"value": world * units * args.steps / (e2e_total * 1e-3), "unit": UNIT,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": e2e_total / args.steps, "api": "tr_solve"},
        "roofline": roof,
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }
    if world == 1:
        out["solve_latency_ms"] = solve_latency(B, devn)
    if world == 1 and args.configs != "none":
        names = EXTRA_CONFIGS if args.configs == "all" else tuple(args.configs.split(","))
        out["configs"] = extra_configs(B, names, devn, sha)
    if args.serving > 0 and world == 1:
        out["serving"] = serving_run(args, out["forms"]["fp32_sweep64"]["value"])
    if pool is not None:
        out["cpu_baseline"] = cpu_baseline(args.workload, args.cpu_sample, pool)
        pool.close()
    print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def percentile(xs, p):
    xs = sorted(xs)
    return xs[min(len(xs) - 1, max(0, int(math.ceil(p / 100.0 * len(xs))) - 1))]


def solve_latency(B, devn, name="stromgren32", n=100):
    """Latency distribution of n end-to-end tr_solve calls (host inputs in
    pinned memory, host copy of the flux) on a small problem, one after
    another, FP32 + FP64-sweep form."""
    import numpy as np
    import torch
    from workloads import workload
    w = workload(name, theta_src=0.25)
    host = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory()
            for k, v in (("n_H", w.n_H), ("xyz", w.src_xyz), ("Q", w.src_Q))}
    d = {k: v.to(devn) for k, v in host.items()}
    F = torch.empty((w.N,) * 3, dtype=torch.float64, device=devn)
    F_host = torch.empty_like(F, device="cpu").pin_memory()
    g, s = B.make_grid(d["n_H"], w.dx), B.make_sources(d["xyz"], d["Q"])
    p = B.tr_params_default(theta_src=w.theta_src, precision=1)
    ms = []
    for k in range(n + 5):
        t0 = time.perf_counter()
        for key in d:
            d[key].copy_(host[key], non_blocking=True)
        B.tr_solve(g, s, p, F)
        F_host.copy_(F)
        if k >= 5:
            ms.append(1e3 * (time.perf_counter() - t0))
    return {"workload": f"{name} ({w.N}^3, N_PIX={w.npix})", "calls": n, "p50": percentile(ms, 50),
            "p99": percentile(ms, 99), "max": max(ms), "clock": "host wall clock around each call"}


def extra_configs(B, names, devn, sha):
    """One build and one timed walk (CUDA events) per workload and form:
    the Stromgren test, the AMR cluster and the 256^3 source-count series."""
    import torch
    res = {}
    for name in names:
        pr = make_problem(B, name, devn)
        w, o = pr["w"], pr["out"]
        npix = 12 * w.nside * w.nside
        entry = {}
        forms = (1, 2, 0) if name == "stromgren32" else (1, 2)
        for prec in forms:
            tree = pr["build"](pr["grid"], pr["src"], pr["params"](prec))
            B.tr_walk_sweep(tree, o["F"], o["E"], o["ion"])        # first launch: kernel attributes, clocks
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record()
            B.tr_walk_sweep(tree, o["F"], o["E"], o["ion"])
            s1.record()
            torch.cuda.synchronize()
            ms = s0.elapsed_time(s1)
            stt = B.tr_tree_stats(tree)
            nr = tree.info()["nr"]
            entry[{0: "fp64", 1: "fp32_sweep64", 2: "fp32_sweepdf"}[prec]] = {
                "walk_ms": ms, "cell_rays_per_s": pr["ncell"] * npix / (ms * 1e-3), "visited": stt["visited"],
                "entries": stt["entries"], "fp64_redecided": stt["fp64_mac"] + stt["fp64_setup"]}
            del tree
        entry.update({"cells": pr["ncell"], "npix": npix, "nr": nr, "sources": int(len(w.src_Q))})
        res[name] = entry
        del pr
        torch.cuda.empty_cache()
    s = res.get("sourcecount256_s1"), res.get("sourcecount256_s10000")
    if all(s):
        res["sourcecount_ratio_s10000_over_s1"] = {f: s[1][f]["walk_ms"] / s[0][f]["walk_ms"]
                                                   for f in ("fp32_sweep64", "fp32_sweepdf")}
    return res


def serving_run(args, capacity_rays_per_s):
    """Continuous batching of a Poisson stream of requests (serving loop):
    grids drawn from --serving-sizes, N_PIX from --serving-nsides, 1-1000
    sources; the arrival rate is --serving-load times the capacity the
    headline form measured, in requests per second of mean request work."""
    import numpy as np
    from paper_2105_09644_gb300.serving import Server, poisson_stream, percentile as pct
    sizes = tuple(int(x) for x in args.serving_sizes.split(","))
    nsides = tuple(int(x) for x in args.serving_nsides.split(","))
    # mean work of a request in cell-rays (walk cost grows ~ N_PIX at fixed theta)
    mean_rays = np.mean([n ** 3 for n in sizes]) * np.mean([12 * k * k for k in nsides])
    rate = args.serving_load * capacity_rays_per_s / mean_rays
    reqs = poisson_stream(args.serving, rate, seed=2105, sizes=sizes, nsides=nsides, max_sources=1000, lazy=True)
    srv = Server(budget_bytes=96 << 30, tick_targets=1 << 20, precision=1, keep_results=False)
    t0 = time.perf_counter()
    done = srv.run(reqs)
    wall = time.perf_counter() - t0
    lat = [1e3 * r.latency for r in done]
    rays = sum(r.N ** 3 * 12 * r.nside * r.nside for r in done)
    return {"requests": len(done), "arrival_rate_hz": rate, "load": args.serving_load, "sizes": list(sizes),
            "nsides": list(nsides), "sources": "1-1000 per request, log-uniform count", "theta_lim": 0.5,
            "p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99), "max_ms": max(lat),
            "cell_rays_per_s": rays / wall, "wall_s": wall, "launches": srv.launches,
            "precision": FORM_NAMES[1]}


# ---------------------------------------------------------------- reference arm

def workload_name(w, nr):
    """The workload as both arms name it in their config."""
    return (f"{w.name}: {w.N}^3 log-normal (sigma_ln 1.5, k^-4), box 10 pc, {len(w.src_Q)} point sources, "
            f"N_PIX={w.npix}, N_R={nr}, theta_lim={w.theta_lim}")


def run_reference(args):
    """The oracle, as it stands, on the host cores: each step a bounded sample
    of the workload's targets."""
    rank, world, local = dist_env()
    if rank != 0:
        return
    import multiprocessing as mp
    import oracle
    from workloads import workload
    w = workload(args.workload)
    pool = mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1))
    n = max(256, args.cpu_sample // 4)
    for _ in range(args.warmup):
        cpu_baseline(args.workload, 64, pool)
    vals, times = [], []
    for _ in range(args.steps):
        r = cpu_baseline(args.workload, n, pool)
        vals.append(r["value"])
        times.append(r["seconds"])
    pool.close()
    value = statistics.mean(vals)
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": workload_name(w, oracle.num_points(w.eta_r, w.N * math.sqrt(3.0))),
                      "precision": "plain FP64 CPU oracle",
                      "sample": f"{n} seeded random target cells per step",
                      "parallelism": f"{r['cores']} host processes"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": r["cores"], "kind": "oracle",
                            "sample": r["sample"]},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)
