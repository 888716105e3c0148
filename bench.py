#!/usr/bin/env python
"""Benchmark of the DRGraph layout path on one GB300 (or N, as replicas).

A step is one pass of the whole path on one synthetic graph: canonical graph
from the edge list, k-order distance matrix, similarity and alias tables,
heavy-edge-matching hierarchy, random coarsest layout, then every level's
epochs and refinement.  The metric is edge-sample gradient updates per second
(one update = one positive sample with its M negatives: 1 attractive and M
repulsive forces), counted over all levels, with the step's wall time on the
device.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
                  [--mode hogwild|sync] [--precision fp32|fp16|bf16]
                  [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun every rank lays out its own
replica (graph id = rank); there is no collective on the data path.
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

WORKLOADS = {
    # the workload the metric is quoted on (1M-node layout time)
    "dcsbm1m": dict(graph="dcsbm1m", k=2, M=5, epochs=500, b=1.0, stop_nodes=1000,
                    desc="DC-SBM 1,000,000 nodes, 64 equal blocks, Pareto degree weights exponent 2.5, "
                         "mean degree 8, in:out 20:1, seed 2; multilevel HEM to <1000 nodes, k=2, M=5, "
                         "500 epochs per level, b=1"),
    "ba100k": dict(graph="ba100k", k=3, M=5, epochs=500, b=1.0, stop_nodes=1000,
                   desc="Barabasi-Albert 100,000 nodes, m=3, seed 1; multilevel HEM to <1000 nodes, k=3, M=5, "
                        "500 epochs per level, b=1"),
    "grid32": dict(graph="grid32", k=3, M=5, epochs=500, b=3.0, stop_nodes=1000, multilevel=0,
                   desc="32x32 grid, single level, k=3, M=5, 500 epochs, b=3"),
    "batch256": dict(graph="batch256", k=2, M=5, epochs=300, b=2.0, stop_nodes=1000,
                     desc="256 graphs (grids b=3, random binary trees and Barabasi-Albert m=2 b=2), node counts "
                          "log-uniform in [1k, 50k], seed 3; multilevel, k=2, M=5, 300 epochs, one batched launch "
                          "per sub-step across graphs"),
}


class Job:
    """One step's input and the two ways to run it: device-resident edges and
    positions (`step`), or host buffers with the copies inside (`e2e`)."""

    def __init__(self, drg, ctx, wl, p, np, torch):
        import graphgen as gg
        self.drg, self.ctx, self.p, self.np, self.torch = drg, ctx, p, np, torch
        if wl["graph"] == "batch256":
            items = gg.batch_mix(256, 1000, 50000, 3)
            self.graphs = [g for _, g in items]
            self.b = [3.0 if kind == "grid" else 2.0 for kind, _ in items]
        else:
            self.graphs = [gg.workload(wl["graph"])]
            self.b = None
        self.n = sum(g[0] for g in self.graphs)
        self.m = sum(len(g[1]) for g in self.graphs)
        self.dev = [(g[0], torch.from_numpy(g[1].view(np.int32)).cuda(), torch.from_numpy(g[2].view(np.int32)).cuda())
                    for g in self.graphs]
        self.pos = [torch.zeros(2 * g[0], dtype=torch.float32, device="cuda") for g in self.graphs]
        self.host = None

    def _run(self, edges, pos):
        drg, ctx = self.drg, self.ctx
        if self.b is None:
            n, s, d = edges[0]
            drg.layout_edges(ctx, n, s, d, self.p, pos[0])
        else:
            gs = [drg.graph_from_edges(ctx, n, s, d) for n, s, d in edges]
            dpos = pos if pos[0].is_cuda else [self.torch.zeros(x.shape, device="cuda") for x in pos]
            drg.layout_batch(ctx, gs, self.p, dpos, b=self.b)
            if dpos is not pos:
                for x, y in zip(pos, dpos):
                    x.copy_(y)

    def step(self):
        self._run(self.dev, self.pos)

    def e2e(self):
        np, torch = self.np, self.torch
        if self.host is None:
            self.host = ([(g[0], torch.from_numpy(g[1].view(np.int32)).pin_memory(),
                           torch.from_numpy(g[2].view(np.int32)).pin_memory()) for g in self.graphs],
                         [torch.zeros(2 * g[0], dtype=torch.float32).pin_memory() for g in self.graphs])
        self._run(*self.host)
        return self.host[1]

ALGO_BYTES_NOTE = ("per sample: edge record (16 B packed below 2^24 nodes, else 20 B read of the 32-B record) + "
                   "M negative records (node table 8 B on level 0; the Hogwild kernel's level node table 16 B on "
                   "coarse levels, the sub-step kernel's node table 8 B + ancestor 4 B) + (2+M) position gathers "
                   "(8 B; 4 B for negatives with half copies) + (2+M) 8-B atomic adds; + 2 ancestor reads of 4 B "
                   "for the endpoints on coarse levels")


def algo_bytes_per_sample(kernel, M, precision, coarse, packed=True):
    edge = 16 if packed else 20
    neg_rec = 16 if (coarse and kernel in ("k_hogwild", "k_hogwild_batch")) else 8
    if coarse and kernel not in ("k_hogwild", "k_hogwild_batch"):
        neg_rec += 4  # ancestor of each negative
    neg_pos = 4 if precision else 8
    b = edge + M * neg_rec + 2 * 8 + M * neg_pos + (2 + M) * 8
    if coarse:
        b += 2 * 4
    return b


def max_over_ranks(x, dist, device):
    """The slowest rank's figure: whole-job timings are the maximum over ranks."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, seconds):
    """Units all ranks processed (independent replicas, weak scaling) per second of the slowest rank."""
    return units_per_rank * world / seconds


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_hash():
    """Hash of the level kernels' device code: layout.cu from its namespace up
    to the batch section (the epoch kernels and every helper they use); the
    committed DRAM-traffic record is used only while it matches."""
    src = open(os.path.join(ROOT, "paper_2008_07799_gb300", "csrc", "layout.cu")).read()
    start = src.index("namespace drg {")
    end = src.index("// ------------------------------------------------------------------ batches of graphs")
    return hashlib.sha256(src[start:end].encode()).hexdigest()[:16]


def epoch_kernel(graph, mode, precision):
    """The kernel that runs a level's samples: one persistent launch per level
    for FP32 Hogwild on one graph, sub-step launches otherwise."""
    one_launch = mode == "hogwild" and precision == "fp32"
    if graph == "batch256":
        return "k_hogwild_batch" if one_launch else "k_epoch_batch"
    return "k_hogwild" if one_launch else "k_epoch"


def ncu_traffic_per_sample(kernel, cfg):
    """DRAM bytes per sample of the level kernel from the committed ncu
    summary, or None when the kernel source has changed since that capture or
    the run's configuration is not the captured one."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        if d.get("kernel_hash") != kernel_hash() or d.get("config") != cfg:
            return None
        return float(d["dram_bytes_per_sample"])
    except Exception:
        return None


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.out = os.path.join("/tmp", f"drg_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.out, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.out):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for name, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def make_params(drg, wl, args, gid):
    p = drg.Params.default(k=wl["k"], M=wl["M"], epochs=wl["epochs"], b=wl["b"], stop_nodes=wl["stop_nodes"],
                           mode=1 if args.mode == "hogwild" else 0,
                           precision={"fp32": 0, "fp16": 1, "bf16": 2}[args.precision], seed=args.seed, gid=gid)
    if "multilevel" in wl:
        p.multilevel = wl["multilevel"]
    if args.substeps:
        p.substeps = args.substeps
    p.coarsen = {"hem": 0, "star": 1}[args.coarsen]
    p.level_tables = 1 if args.level_tables else 0
    p.perplexity = args.perplexity
    return p


# ------------------------------------------------------------------ CPU oracle legs
def oracle_sample(wl, budget_s):
    """The oracle's layout loop on a bounded sample of the workload: the same
    generator and parameters at a node count the oracle handles, level-0
    epochs in sequential mode, until about budget_s seconds of CPU time."""
    import graphgen as gg
    import oracle as orc
    if wl["graph"] == "dcsbm1m":
        n, s, d = gg.dc_sbm(20_000, 64, 2.5, 8.0, 20.0, 2)
        sample = "DC-SBM 20,000 nodes (same generator parameters as the 1M workload), k=2"
    elif wl["graph"] == "batch256":
        n, s, d = gg.barabasi_albert(20_000, 2, 3)
        sample = "one Barabasi-Albert 20,000-node m=2 member of the batch family, k=2"
    elif wl["graph"] == "ba100k":
        n, s, d = gg.barabasi_albert(100_000, 3, 1)
        sample = "Barabasi-Albert 100,000 nodes m=3 (the workload graph), k=3"
    else:
        n, s, d = gg.grid(32, 32)
        sample = "32x32 grid (the workload graph), k=3"
    rp, col = orc.canonical_graph(n, s, d)
    gd = orc.korder(rp, col, wl["k"])
    tab, _ = orc.sampling_tables(*gd, wl["k"])
    p = orc.Params(k=wl["k"], M=wl["M"], epochs=10 ** 6, b=wl["b"], mode=1, seed=0)
    Y = orc.init_positions(p, 0, n) * 1e4
    t0 = time.process_time()
    w0 = time.perf_counter()
    epochs = 0
    while time.process_time() - t0 < budget_s:
        orc.layout_level(tab, Y, 0, None, p, 0.1, epochs, epochs + 1)
        epochs += 1
    wall = time.perf_counter() - w0
    samples = epochs * n
    return samples / wall, samples, f"{sample}; {epochs} level-0 epochs ({samples} samples) of the FP64 oracle, sequential mode"


def oracle_parallel_sample(wl, budget_s):
    """The paper's multi-threaded optimisation (Sec. 4.3) on the same bounded
    sample as oracle_sample: the oracle's sequential loop with each epoch's
    samples shared over every host core without locks.  Returns None when the
    toolchain has no OpenMP."""
    import graphgen as gg
    import oracle as orc
    if orc.build_omp() is None:
        return None
    threads = os.cpu_count() or 1
    if wl["graph"] == "dcsbm1m":
        n, s, d = gg.dc_sbm(20_000, 64, 2.5, 8.0, 20.0, 2)
    elif wl["graph"] == "batch256":
        n, s, d = gg.barabasi_albert(20_000, 2, 3)
    elif wl["graph"] == "ba100k":
        n, s, d = gg.barabasi_albert(100_000, 3, 1)
    else:
        n, s, d = gg.grid(32, 32)
    rp, col = orc.canonical_graph(n, s, d)
    gd = orc.korder(rp, col, wl["k"])
    tab, _ = orc.sampling_tables(*gd, wl["k"])
    p = orc.Params(k=wl["k"], M=wl["M"], epochs=10 ** 6, b=wl["b"], mode=1, seed=0)
    Y = orc.init_positions(p, 0, n) * 1e4
    w0 = time.perf_counter()
    epochs = 0
    while time.perf_counter() - w0 < budget_s:
        orc.layout_level_omp(tab, Y, 0, None, p, 0.1, threads, epochs, epochs + 1)
        epochs += 1
    wall = time.perf_counter() - w0
    samples = epochs * n
    return samples / wall, threads, (f"the cpu_baseline sample; {epochs} level-0 epochs ({samples} samples) of the "
                                     f"FP64 oracle's loop on {threads} lock-free OpenMP threads")


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = WORKLOADS[args.workload]
    per_step = max(0.5, min(args.cpu_budget, 60.0 / max(args.steps + args.warmup, 1)))
    for _ in range(args.warmup):
        oracle_sample(wl, per_step / 4)
    vals = []
    t0 = time.perf_counter()
    sample = ""
    total_samples = 0
    for _ in range(args.steps):
        v, ns, sample = oracle_sample(wl, per_step)
        vals.append(v)
        total_samples += ns
    wall = time.perf_counter() - t0
    value = total_samples / wall
    line = {"impl": "reference", "metric": "edge-sample gradient updates/s", "value": value, "unit": "updates/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * wall / max(args.steps, 1), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "desc": wl["desc"]},
            "cpu_baseline": {"value": value, "unit": "updates/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="dcsbm1m", choices=sorted(WORKLOADS))
    ap.add_argument("--mode", default="hogwild", choices=["hogwild", "sync"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp16", "bf16"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--cpu-budget", type=float, default=15.0,
                    help="seconds of oracle work for cpu_baseline; also caps each reference-arm step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-parallel", action="store_true",
                    help="also time the oracle's loop on every host core without locks (the paper's "
                         "multi-threaded mode), on the same bounded sample")
    ap.add_argument("--k", type=int, default=None, help="override the distance-matrix order (profiling cases)")
    ap.add_argument("--single-level", action="store_true", help="lay out G^0 only (profiling cases)")
    ap.add_argument("--once", action="store_true", help="run exactly one step and exit (for ncu captures)")
    ap.add_argument("--coarsen", default="hem", choices=["hem", "star"],
                    help="coarsening rule: heavy-edge matching or the paper's star grouping (Sec. 3.2.3)")
    ap.add_argument("--perplexity", type=float, default=0.0,
                    help="> 0: sigma_i of Eq. 9 per node calibrated to this perplexity")
    ap.add_argument("--level-tables", action="store_true",
                    help="each coarse level samples its own distance matrix and tables (the conventional "
                         "multilevel scheme) instead of G^0's through the ancestor map")
    ap.add_argument("--substeps", type=int, default=None, help="override the in-flight bound n_l / substeps (profiling cases)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    import graphgen as gg
    import paper_2008_07799_gb300 as drg
    from paper_2008_07799_gb300 import build
    build.build()

    wl = dict(WORKLOADS[args.workload])
    if args.k is not None:
        wl["k"] = args.k
        wl["desc"] += f" (k overridden to {args.k})"
    if args.single_level:
        wl["multilevel"] = 0
        wl["desc"] += " (single level)"
    if args.coarsen == "star":
        wl["desc"] = wl["desc"].replace("multilevel HEM", "multilevel star grouping")
    if args.level_tables:
        wl["desc"] += "; each coarse level samples its own distance matrix and tables"
    if args.perplexity > 0:
        wl["desc"] += f"; sigma_i per node at perplexity {args.perplexity:g}"
    stream = torch.cuda.current_stream()
    ctx = drg.Context(local, stream.cuda_stream)
    p = make_params(drg, wl, args, gid=rank)
    job = Job(drg, ctx, wl, p, np, torch)
    n, m = job.n, job.m
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.int32, device="cuda")  # 1 GiB > L2
    step = job.step

    if args.once:
        step()
        torch.cuda.synchronize()
        print(json.dumps({"once": args.workload, "k": wl["k"], "launches": ctx.launches}), flush=True)
        return

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # one profiled pass: per-kernel CUDA events on the library's stream
    ctx.profile_reset()
    ctx.profile(True)
    step()
    torch.cuda.synchronize()
    ep_ms, ep_launches, ep_samples = ctx.profile_read(drg.PROF_EPOCH)
    ap_ms, ap_launches, _ = ctx.profile_read(drg.PROF_APPLY)
    dm_ms, _, nnz = ctx.profile_read(drg.PROF_DMAT)
    hi_ms, _, levels = ctx.profile_read(drg.PROF_HIER)
    sub_ms = {name: ctx.profile_read(w)[0] for name, w in
              (("graph", drg.PROF_GRAPH), ("bfs", drg.PROF_BFS), ("similarity", drg.PROF_SIM),
               ("alias_tables", drg.PROF_ALIAS), ("host_alloc", drg.PROF_ALLOC))}
    ctx.profile(False)

    # timed region
    clocks = Clocks(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    launches0 = ctx.launches
    times = []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    launches = ctx.launches - launches0
    clk = clocks.stop()
    ms = max_over_ranks(sum(times) / len(times), dist, "cuda")
    if dist:
        dist.barrier()
    samples_per_step = ep_samples
    value = whole_job_rate(samples_per_step, world, ms / 1000.0)

    # end to end through the public API from pinned host buffers
    e2e_times = []
    hpos = None
    for _ in range(max(1, min(args.steps, 3))):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hpos = job.e2e()  # host pointers: the copies happen inside the calls
        torch.cuda.synchronize()
        e2e_times.append(time.perf_counter() - t0)
    e2e_s = max_over_ranks(sum(e2e_times) / len(e2e_times), dist, "cuda")
    e2e_value = whole_job_rate(samples_per_step, world, e2e_s)
    assert all(np.isfinite(x.numpy()).all() for x in hpos)

    if rank != 0:
        return
    hbm, peak_kind = peaks()
    n0 = n
    s0 = n0 * wl["epochs"]
    coarse = max(ep_samples - s0, 0)
    prec = {"fp32": 0, "fp16": 1, "bf16": 2}[args.precision]
    kname = epoch_kernel(wl["graph"], args.mode, args.precision)
    packed = n < (1 << 24)
    bytes_total = (s0 * algo_bytes_per_sample(kname, wl["M"], prec, False, packed)
                   + coarse * algo_bytes_per_sample(kname, wl["M"], prec, True, packed))
    achieved = bytes_total / (ep_ms / 1000.0) / 1e9
    tps = None if (args.level_tables or args.perplexity > 0) else ncu_traffic_per_sample(kname, {"workload": args.workload, "k": wl["k"], "coarsen": args.coarsen,
                                         "mode": args.mode, "precision": args.precision,
                                         "multilevel": bool(wl.get("multilevel", 1))})
    avg_launch_samples = ep_samples / max(ep_launches, 1)
    line = {
        "metric": "edge-sample gradient updates/s",
        "value": value,
        "unit": "updates/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32" if prec == 0 else ("f32+f16" if prec == 1 else "f32+bf16"),
        "data": "synthetic",
        "config": {"workload": args.workload, "desc": wl["desc"], "mode": args.mode, "precision": args.precision,
                   "coarsen": args.coarsen, "level_tables": bool(args.level_tables),
                   "perplexity": args.perplexity, "n": n, "edges_in": m, "distance_matrix_entries": nnz, "levels": levels,
                   "samples_per_step": samples_per_step, "layout_time_ms": ms,
                   "l2": "1 GiB buffer written between timed steps (flush)",
                   "parallelism": f"replicas x{world}"},
        "phases_ms": {"distance_matrix_and_tables": dm_ms, "hierarchy": hi_ms, "layout_levels": ep_ms, **sub_ms},
        "phases_note": "CUDA-event timers of one profiled step, in which builds that the timed steps run "
                       "concurrently (hierarchy beside the distance matrix; a batch's graphs) run one after another",
        "gpu_launches": launches,
        "roofline": {"kernel": kname, "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "peak_kind": peak_kind,
                     "traffic": None if tps is None else tps * avg_launch_samples,
                     "algorithmic_bytes_note": ALGO_BYTES_NOTE,
                     "avg_launch_ms": ep_ms / max(ep_launches, 1), "launches": ep_launches},
        "e2e": {"value": e2e_value, "unit": "updates/s", "h2d_bytes_per_step": 2 * m * 4,
                "d2h_bytes_per_step": 2 * n * 4, "seconds_per_step": e2e_s},
        "clocks": clk,
    }
    if not args.no_cpu_baseline:
        v, ns, sample = oracle_sample(wl, args.cpu_budget)
        line["cpu_baseline"] = {"value": v, "unit": "updates/s", "cores": 1, "kind": "oracle", "sample": sample}
    if args.cpu_parallel:
        par = oracle_parallel_sample(wl, args.cpu_budget)
        if par is not None:
            line["cpu_parallel_baseline"] = {"value": par[0], "unit": "updates/s", "cores": par[1],
                                             "kind": "oracle, lock-free OpenMP threads (Sec. 4.3)",
                                             "sample": par[2]}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
