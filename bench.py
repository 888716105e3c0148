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
    # a smaller graph of the 1M workload's generator (profiling captures)
    "dcsbm100k": dict(graph="dcsbm100k", k=2, M=5, epochs=500, b=1.0, stop_nodes=1000,
                      desc="DC-SBM 100,000 nodes with the 1M workload's generator parameters, seed 2; multilevel "
                           "HEM to <1000 nodes, k=2, M=5, 500 epochs per level, b=1"),
    "rmat22": dict(graph="rmat22", k=1, M=5, epochs=300, b=1.0, stop_nodes=1000,
                   desc="R-MAT scale 22 (4,194,304 nodes), edge factor 8, a,b,c,d = .57,.19,.19,.05, duplicates and "
                        "self-loops removed, seed 4; multilevel HEM to <1000 nodes, k=1 (k=2 exceeds 2^32 entries), "
                        "M=5, 300 epochs per level, b=1"),
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
        self.one_by_one = False

    def _run(self, edges, pos):
        drg, ctx = self.drg, self.ctx
        if self.b is None:
            n, s, d = edges[0]
            drg.layout_edges(ctx, n, s, d, self.p, pos[0])
        elif self.one_by_one:
            # the same graphs laid out one after another, each as its own job
            for g, ((n, s, d), x, b) in enumerate(zip(edges, pos, self.b)):
                drg.layout_edges(ctx, n, s, d, self.p.replace(b=b, gid=g), x)
        else:
            gs = [drg.graph_from_edges(ctx, n, s, d) for n, s, d in edges]
            dpos = pos if pos[0].is_cuda else [self.torch.zeros(x.shape, device="cuda") for x in pos]
            drg.layout_batch(ctx, gs, self.p, dpos, b=self.b)
            if dpos is not pos:
                for x, y in zip(pos, dpos):
                    x.copy_(y)

    def step(self):
        self._run(self.dev, self.pos)

    def pin_host(self):
        """Pinned host copies of the edges and positions (made once, outside any timed region)."""
        np, torch = self.np, self.torch
        if self.host is None:
            self.host = ([(g[0], torch.from_numpy(g[1].view(np.int32)).pin_memory(),
                           torch.from_numpy(g[2].view(np.int32)).pin_memory()) for g in self.graphs],
                         [torch.zeros(2 * g[0], dtype=torch.float32).pin_memory() for g in self.graphs])

    def e2e(self):
        self.pin_host()
        self._run(*self.host)
        return self.host[1]

# Per-sample accesses of the level kernels, by kind (the probe that bounds
# each): table records and position gathers of 4 or 8 bytes cost one L2
# request like an 8-byte load; 16-byte records like a 16-byte load; every
# touched node one 8-byte vector atomic add; the edge record is the one
# access that misses L2 (its table is far larger than L2).
def sample_accesses(kernel, M, precision, coarse):
    """(load8, load16, red8, hbm16, l2_bytes) per sample."""
    hog = kernel in ("k_hogwild", "k_hogwild_batch")
    load8 = 2 + M  # position gathers (negatives from the half copy when precision > 0: 4 bytes, one request)
    load16 = 0
    l2_bytes = 2 * 8 + M * (4 if precision else 8)
    if coarse and hog:
        load16 += M        # level node records {thresh, anc(own), anc(alias)}
        l2_bytes += 16 * M
        load8 += 2         # ancestors of the two endpoints
        l2_bytes += 8
    else:
        load8 += M         # node records {thresh, alias}
        l2_bytes += 8 * M
        if coarse:
            load8 += 2 + M  # ancestors of every drawn node
            l2_bytes += 4 * (2 + M)
    red8 = 2 + M
    l2_bytes += 8 * red8
    if precision and hog:
        # the copy of every node rewritten once per epoch (n_l samples): one
        # coalesced 8-byte read and 4-byte write per sample, 12/32 of a sector
        load8 += 12 / 32
        l2_bytes += 12
    return load8, load16, red8, 1, l2_bytes


PROBE_L2_BYTES = 32 << 20     # inside L2 (about a quarter of it), like the level kernels' working set
PROBE_HBM_BYTES = 8 << 30     # far larger than L2, like the edge table


def measure_probes(drg, ctx):
    """Random-access ceilings of this GPU (accesses/s), each the best of three
    launches after a warm-up: L2-resident 8-byte loads, 16-byte loads and
    8-byte atomic adds, each alone, and a layout sample's mix (read-only table
    loads, position loads and atomic adds, one to one to one);
    16-byte loads over a buffer far larger than L2 (plain
    and evict-first); and the streaming copy (GB/s, read + written)."""
    out = {}
    for name, kind, size, count in (("l2_load8", drg.PROBE_LOAD8, PROBE_L2_BYTES, 400_000_000),
                                    ("l2_load16", drg.PROBE_LOAD16, PROBE_L2_BYTES, 400_000_000),
                                    ("l2_red8", drg.PROBE_RED8, PROBE_L2_BYTES, 400_000_000),
                                    ("l2_mix", drg.PROBE_MIX_LOAD8_RED8, PROBE_L2_BYTES, 400_000_000),
                                    ("hbm_load16", drg.PROBE_LOAD16, PROBE_HBM_BYTES, 40_000_000),
                                    ("hbm_load16_evict_first", drg.PROBE_LOAD16_EVICT_FIRST, PROBE_HBM_BYTES,
                                     40_000_000),
                                    ("copy", drg.PROBE_COPY, PROBE_HBM_BYTES, 1)):
        best = 0.0
        for rep in range(4):
            ms, done = drg.probe_memory(ctx, kind, size, count)
            if rep:
                rate = (done * 32 / ms / 1e6) if kind == drg.PROBE_COPY else (done / (ms / 1e3))
                best = max(best, rate)
        out[name] = best
    out["unit"] = "accesses/s (copy: GB/s read + written)"
    out["buffers"] = {"l2": PROBE_L2_BYTES, "hbm": PROBE_HBM_BYTES}
    return out


def roofline_l2_hbm(kernel, M, precision, level_samples, kernel_ms, probes, hbm_copy_peak):
    """Both ceilings of a level-kernel run.  level_samples: [(samples, coarse)].
    L2: the time the run's L2 accesses take at the probes' rates, against the
    kernel's time -- at the rate of the probe that interleaves loads and
    atomic adds as a layout sample does (the headline: mixing them costs
    throughput, so the kinds' separate rates overstate the ceiling), and at
    the kinds' separate rates; HBM: the edge records, one random 16-byte read
    per sample, against the random-read probe and against the copy peak."""
    t_sep = 0.0
    t_mix = 0.0
    l2_bytes = 0.0
    samples = 0
    for cnt, coarse in level_samples:
        l8, l16, r8, _, b = sample_accesses(kernel, M, precision, coarse)
        t_sep += cnt * (l8 / probes["l2_load8"] + l16 / probes["l2_load16"] + r8 / probes["l2_red8"])
        t_mix += cnt * (l8 + l16 + r8) / probes["l2_mix"]
        l2_bytes += cnt * b
        samples += cnt
    sec = kernel_ms / 1e3
    l2 = {"achieved": l2_bytes / sec / 1e9, "peak": l2_bytes / t_mix / 1e9, "unit": "GB/s", "frac": t_mix / sec,
          "algorithmic_bytes_per_sample": l2_bytes / max(samples, 1),
          "peak_kind": "measured: random-access probe (drg_probe_memory, PROBE_MIX_LOAD8_RED8) of this run, 8-byte "
                       "read-only table loads, position loads and position atomic adds interleaved one to one to one "
                       "over a 32 MiB buffer, at the kernel's count of "
                       "L2 accesses per sample",
          "separate": {"peak": l2_bytes / t_sep / 1e9, "frac": t_sep / sec,
                       "peak_kind": "measured: the probes of each access kind alone (8-byte loads, 16-byte loads, "
                                    "8-byte atomic adds), weighted by the kernel's per-sample mix"}}
    hbm_ach = samples * 16 / sec / 1e9
    hbm = {"achieved": hbm_ach, "unit": "GB/s", "bytes_per_sample": 16,
           "peak_random16": probes["hbm_load16"] * 16 / 1e9, "frac_random16": samples / probes["hbm_load16"] / sec,
           "peak_copy": hbm_copy_peak, "frac_copy": hbm_ach / hbm_copy_peak}
    return l2, hbm


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
    in Hogwild mode, sub-step launches in synchronous mode."""
    one_launch = mode == "hogwild"
    if graph == "batch256":
        return "k_hogwild_batch" if one_launch else "k_epoch_batch"
    return "k_hogwild" if one_launch else "k_epoch"


def ncu_traffic_per_sample(kernel, cfg, root=ROOT):
    """DRAM bytes per sample of the level kernel from the committed ncu
    summary, or None when the kernel source has changed since that capture or
    the run's configuration is not the captured one."""
    path = os.path.join(root, "profiles", f"{kernel}_traffic.json")
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
    p.row_cap = args.row_cap
    return p


# ------------------------------------------------------------------ CPU oracle legs
def cpu_sample_graph(wl):
    """The bounded sample of a workload that the oracle times: the same
    generator family and parameters at a node count the oracle handles."""
    import graphgen as gg
    g = wl["graph"]
    if g in ("dcsbm1m", "dcsbm100k"):
        return gg.dc_sbm(20_000, 64, 2.5, 8.0, 20.0, 2), "DC-SBM 20,000 nodes (the 1M workload's generator parameters)"
    if g == "batch256":
        return gg.barabasi_albert(20_000, 2, 3), "one Barabasi-Albert 20,000-node m=2 member of the batch family"
    if g == "ba100k":
        return gg.barabasi_albert(20_000, 3, 1), "Barabasi-Albert 20,000 nodes m=3 (the workload's generator)"
    if g == "rmat22":
        return gg.rmat(14, 8, 0.57, 0.19, 0.19, 4), "R-MAT scale 14 (the workload's generator parameters)"
    return gg.grid(32, 32), "32x32 grid (the workload graph)"


def _oracle_params(wl, epochs, mode):
    import oracle as orc
    return orc.Params(k=wl["k"], M=wl["M"], epochs=epochs, b=wl["b"], mode=mode, seed=0, stop_nodes=wl["stop_nodes"],
                      multilevel=bool(wl.get("multilevel", 1)))


def oracle_whole_path(wl, budget_s):
    """The oracle's whole path (canonical graph, distance matrix, tables,
    hierarchy, every level's epochs in sequential mode, refinement) on the
    workload's bounded sample, single-threaded, with the workload's epochs
    per level scaled down when a calibration run says the full count would
    exceed budget_s.  Returns (updates/s, samples, description)."""
    import oracle as orc
    (n, s, d), desc = cpu_sample_graph(wl)
    E = wl["epochs"]
    cal = []
    for e in (2, 12):  # the fixed part (tables, hierarchy) and the cost per epoch
        t0 = time.perf_counter()
        _, st = orc.run(n, s, d, _oracle_params(wl, e, 1), return_state=True)
        cal.append(time.perf_counter() - t0)
    sizes = [lv.n for lv in st["levels"]]
    per_epoch = max((cal[1] - cal[0]) / 10.0, 1e-6)
    fixed = max(cal[0] - 2 * per_epoch, 0.0)
    if fixed + per_epoch * E > budget_s:
        E = max(10, int((budget_s - fixed) / per_epoch))
    p = _oracle_params(wl, E, 1)
    t0 = time.perf_counter()
    orc.run(n, s, d, p, return_state=False)
    wall = time.perf_counter() - t0
    samples = sum(sizes) * E
    # the run's steps before the level runs, timed one by one in a second
    # pass (the phase boundaries of the GPU line's phases_ms); the level runs
    # and refinement are the rest of the whole run's time
    phases = {}
    t = time.perf_counter()
    rp, col = orc.canonical_graph(n, s, d)
    phases["graph"] = time.perf_counter() - t
    t = time.perf_counter()
    gd = orc.korder(rp, col, wl["k"])
    phases["distance_matrix"] = time.perf_counter() - t
    t = time.perf_counter()
    orc.sampling_tables(*gd, wl["k"], p.sigma)
    phases["similarity_and_alias_tables"] = time.perf_counter() - t
    t = time.perf_counter()
    orc.hierarchy(rp, col, p)
    phases["hierarchy"] = time.perf_counter() - t
    phases["layout_levels_and_refinement"] = max(wall - sum(phases.values()), 0.0)
    phases = {k: round(v * 1e3, 1) for k, v in phases.items()}
    return samples / wall, samples, (f"{desc}, k={wl['k']}, M={wl['M']}, b={wl['b']:g}; the FP64 oracle's whole path "
                                     f"(tables, hierarchy of {len(sizes)} levels, {E} epochs per level in "
                                     f"sequential mode, refinement) on one core: {samples} samples in {wall:.1f} s"), \
        phases


def oracle_sample(wl, budget_s):
    """The oracle's layout loop on the workload's bounded sample: level-0
    epochs in sequential mode, until about budget_s seconds of CPU time."""
    import oracle as orc
    (n, s, d), desc = cpu_sample_graph(wl)
    rp, col = orc.canonical_graph(n, s, d)
    gd = orc.korder(rp, col, wl["k"])
    tab, _ = orc.sampling_tables(*gd, wl["k"])
    p = _oracle_params(wl, 10 ** 6, 1)
    Y = orc.init_positions(p, 0, n) * 1e4
    t0 = time.process_time()
    w0 = time.perf_counter()
    epochs = 0
    while time.process_time() - t0 < budget_s:
        orc.layout_level(tab, Y, 0, None, p, 0.1, epochs, epochs + 1)
        epochs += 1
    wall = time.perf_counter() - w0
    samples = epochs * n
    return samples / wall, samples, (f"{desc}, k={wl['k']}; {epochs} level-0 epochs ({samples} samples) of the FP64 "
                                     f"oracle, sequential mode, one core")


def oracle_parallel_sample(wl, budget_s, reps=5):
    """The paper's multi-threaded optimisation (Sec. 4.3) on the workload's
    bounded sample: the oracle's sequential loop with each epoch's samples
    shared over every host core without locks; the median of `reps` timed
    runs of budget_s / reps seconds each.  Returns None when the toolchain
    has no OpenMP."""
    import oracle as orc
    if orc.build_omp() is None:
        return None
    threads = os.cpu_count() or 1
    (n, s, d), desc = cpu_sample_graph(wl)
    rp, col = orc.canonical_graph(n, s, d)
    gd = orc.korder(rp, col, wl["k"])
    tab, _ = orc.sampling_tables(*gd, wl["k"])
    p = _oracle_params(wl, 10 ** 6, 1)
    Y = orc.init_positions(p, 0, n) * 1e4
    rates = []
    epochs = 0
    for _ in range(reps):
        w0 = time.perf_counter()
        e0 = epochs
        while time.perf_counter() - w0 < budget_s / reps:
            orc.layout_level_omp(tab, Y, 0, None, p, 0.1, threads, epochs, epochs + 1)
            epochs += 1
        rates.append((epochs - e0) * n / (time.perf_counter() - w0))
    return statistics.median(rates), threads, (f"{desc}, k={wl['k']}; level-0 epochs of the FP64 oracle's loop on "
                                               f"{threads} lock-free OpenMP threads (all host cores), median of "
                                               f"{reps} runs of {budget_s / reps:.1f} s")


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = WORKLOADS[args.workload]
    # each step: the oracle's whole path on the workload's bounded sample,
    # sized so that warm-up and timed steps take about two minutes in all
    per_step = max(2.0, min(args.cpu_budget, 120.0 / max(args.steps + args.warmup, 1)))
    for _ in range(args.warmup):
        oracle_sample(wl, 0.5)
    t0 = time.perf_counter()
    sample = ""
    total_samples = 0
    for _ in range(args.steps):
        v, ns, sample, _ = oracle_whole_path(wl, per_step)
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
    ap.add_argument("--no-autotune", action="store_true", help="keep the level kernels' default launch shape")
    ap.add_argument("--one-by-one", action="store_true",
                    help="batch256: lay the graphs out one after another (the single-graph form) instead of as one job")
    ap.add_argument("--row-cap", type=int, default=0,
                    help="> 0: every row of the distance matrix keeps its row-cap nearest nodes (pattern K u K^T)")
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
    if args.row_cap > 0:
        wl["desc"] += f"; rows capped to their {args.row_cap} nearest nodes (pattern K u K^T)"
    stream = torch.cuda.current_stream()
    ctx = drg.Context(local, stream.cuda_stream)
    ctx.autotune(not args.no_autotune)
    p = make_params(drg, wl, args, gid=rank)
    probes = None if args.once else measure_probes(drg, ctx)
    job = Job(drg, ctx, wl, p, np, torch)
    job.one_by_one = bool(args.one_by_one)
    if args.one_by_one:
        wl["desc"] += "; the graphs laid out one after another, each as its own job"
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

    # end to end through the public API from pinned host buffers: the buffers
    # are pinned and the host path warmed up once before the timed calls
    job.pin_host()
    job.e2e()
    torch.cuda.synchronize()
    e2e_times = []
    hpos = None
    for _ in range(max(1, args.steps)):
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
    if peak_kind == "fallback" and probes.get("copy"):
        hbm, peak_kind = probes["copy"], "measured by this run's streaming-copy probe (drg_probe_memory)"
    n0 = n
    s0 = n0 * wl["epochs"]
    coarse = max(ep_samples - s0, 0)
    prec = {"fp32": 0, "fp16": 1, "bf16": 2}[args.precision]
    kname = epoch_kernel("single" if args.one_by_one else wl["graph"], args.mode, args.precision)
    tps = None if (args.level_tables or args.perplexity > 0 or args.row_cap > 0) else ncu_traffic_per_sample(kname, {"workload": args.workload, "k": wl["k"], "coarsen": args.coarsen,
                                         "mode": args.mode, "precision": args.precision,
                                         "multilevel": bool(wl.get("multilevel", 1))})
    avg_launch_samples = ep_samples / max(ep_launches, 1)
    l2, hbm_roof = roofline_l2_hbm(kname, wl["M"], prec, [(s0, False), (coarse, True)], ep_ms, probes, hbm)
    if l2["frac"] >= hbm_roof["frac_random16"]:
        top = {"bound": "l2", "achieved": l2["achieved"], "peak": l2["peak"], "frac": l2["frac"],
               "peak_kind": l2["peak_kind"]}
    else:
        top = {"bound": "hbm", "achieved": hbm_roof["achieved"], "peak": hbm_roof["peak_random16"],
               "frac": hbm_roof["frac_random16"],
               "peak_kind": "measured: random 16-byte-read probe over 8 GiB (drg_probe_memory)"}
    roofline = {"kernel": kname, **top, "unit": "GB/s",
                "traffic": None if tps is None else tps * avg_launch_samples,
                "traffic_note": "DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum of an ncu capture "
                                "of this configuration and kernel source)",
                "l2": l2, "hbm": {**hbm_roof, "peak_copy_kind": peak_kind}, "probes": probes,
                "avg_launch_ms": ep_ms / max(ep_launches, 1), "launches": ep_launches}
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
                   "perplexity": args.perplexity, "row_cap": args.row_cap, "one_by_one": bool(args.one_by_one), "n": n, "edges_in": m, "distance_matrix_entries": nnz, "levels": levels,
                   "samples_per_step": samples_per_step, "layout_time_ms": ms,
                   "l2": "1 GiB buffer written between timed steps (flush)",
                   "parallelism": f"replicas x{world}"},
        "phases_ms": {"distance_matrix_and_tables": dm_ms, "hierarchy": hi_ms, "layout_levels": ep_ms, **sub_ms},
        "phases_note": "CUDA-event timers of one profiled step, in which builds that the timed steps run "
                       "concurrently (hierarchy beside the distance matrix; a batch's graphs) run one after another",
        "gpu_launches": launches,
        "autotune": drg.autotune_table(),
        "roofline": roofline,
        "e2e": {"value": e2e_value, "unit": "updates/s", "h2d_bytes_per_step": 2 * m * 4,
                "d2h_bytes_per_step": 2 * n * 4, "seconds_per_step": e2e_s},
        "clocks": clk,
    }
    if not args.no_cpu_baseline:
        v, ns, sample, ph = oracle_whole_path(wl, args.cpu_budget)
        line["cpu_baseline"] = {"value": v, "unit": "updates/s", "cores": 1, "kind": "oracle", "sample": sample,
                                "nproc": os.cpu_count(), "phases_ms": ph,
                                "phases_note": "the steps before the level runs timed one by one in a second pass; "
                                               "layout_levels_and_refinement is the rest of the whole run"}
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
