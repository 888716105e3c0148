"""Seeded synthetic graph generators: the inputs of the DRGraph layout path.

This module produces raw undirected edge lists ``(n, src, dst)`` (numpy uint32
arrays; duplicates and self-loops allowed) and nothing else.  It holds none of
the layout method's arithmetic: canonicalising a graph, building its distance
matrix, sampling and optimising are done independently by the CUDA library and
by the CPU oracle.  Both consume the same generated edge lists.

The paper evaluates on SuiteSparse / tsNET graphs (Sec. 4, Table 1) that are not
available here.  These generators stand in for them with the structural
families those datasets cover: grids (grid17, mesh3e1), trees (price_1000,
visbrazil), preferential-attachment and degree-corrected block graphs (the
collaboration / social networks), and R-MAT (web and social graphs).

All randomness is numpy's PCG64 seeded explicitly, so a (generator, seed)
pair gives the same edge list on every machine.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "path", "cycle", "grid", "random_binary_tree", "barabasi_albert",
    "dc_sbm", "rmat", "erdos_renyi", "batch_mix", "workload",
]


def _pack(n, src, dst):
    return int(n), np.ascontiguousarray(src, dtype=np.uint32), np.ascontiguousarray(dst, dtype=np.uint32)


def path(n: int):
    """Path 0-1-2-...-(n-1)."""
    v = np.arange(max(n - 1, 0), dtype=np.uint32)
    return _pack(n, v, v + 1)


def cycle(n: int):
    """Cycle on n >= 3 nodes."""
    v = np.arange(n, dtype=np.uint32)
    return _pack(n, v, (v + 1) % n)


def grid(rows: int, cols: int):
    """rows x cols 4-neighbour grid; node id = r * cols + c."""
    ids = np.arange(rows * cols, dtype=np.uint32).reshape(rows, cols)
    right = (ids[:, :-1].ravel(), ids[:, 1:].ravel())
    down = (ids[:-1, :].ravel(), ids[1:, :].ravel())
    return _pack(rows * cols, np.r_[right[0], down[0]], np.r_[right[1], down[1]])


def random_binary_tree(n: int, seed: int):
    """Random binary tree: node v >= 1 attaches to a uniformly chosen free child slot."""
    rng = np.random.default_rng(seed)
    src = np.empty(max(n - 1, 0), np.uint32)
    dst = np.empty(max(n - 1, 0), np.uint32)
    slots = [0, 0]  # each entry is a parent with one free child position
    for v in range(1, n):
        k = int(rng.integers(len(slots)))
        p = slots[k]
        slots[k] = slots[-1]
        slots.pop()
        src[v - 1] = p
        dst[v - 1] = v
        slots.append(v)
        slots.append(v)
    return _pack(n, src, dst)


def barabasi_albert(n: int, m: int, seed: int):
    """Preferential attachment (Barabasi-Albert).

    Nodes 0..m-1 start without edges; node m links to all of them; every later
    node v links to m distinct earlier nodes drawn with probability
    proportional to their current degree (the classic repeated-endpoint list).
    """
    rng = np.random.default_rng(seed)
    if n <= m:
        return _pack(n, np.zeros(0, np.uint32), np.zeros(0, np.uint32))
    total = (n - m) * m
    src = np.empty(total, np.uint32)
    dst = np.empty(total, np.uint32)
    ends = np.empty(2 * total, np.int64)  # every edge endpoint seen so far
    ne = 0
    targets = list(range(m))
    for v in range(m, n):
        for t in targets:
            src[ne] = v
            dst[ne] = t
            ends[2 * ne] = v
            ends[2 * ne + 1] = t
            ne += 1
        chosen = set()
        lim = 2 * ne
        while len(chosen) < m:
            draws = ends[rng.integers(0, lim, size=2 * m)]
            for d in draws.tolist():
                chosen.add(d)
                if len(chosen) == m:
                    break
        targets = sorted(chosen)
    return _pack(n, src[:ne], dst[:ne])


def dc_sbm(n: int, blocks: int, exponent: float, mean_degree: float, ratio: float, seed: int):
    """Degree-corrected stochastic block model.

    Node v belongs to block v * blocks // n (equal blocks).  Degree weights
    theta_v follow a Pareto law with density exponent ``exponent``.  The edge
    probability of a pair is proportional to theta_u * theta_v times ``ratio``
    for pairs inside one block and times 1 across blocks.  About
    n * mean_degree / 2 edge slots are drawn; duplicates and self-loops are
    left for the consumer to drop.
    """
    rng = np.random.default_rng(seed)
    theta = 1.0 + rng.pareto(exponent - 1.0, size=n)
    blk = (np.arange(n, dtype=np.int64) * blocks) // n
    m = int(round(n * mean_degree / 2))
    tb = np.bincount(blk, weights=theta, minlength=blocks)
    intra_mass = ratio * float((tb ** 2).sum())
    inter_mass = float(tb.sum() ** 2 - (tb ** 2).sum())
    p_in = intra_mass / (intra_mass + inter_mass)
    cs = np.cumsum(theta)
    cs /= cs[-1]
    starts = np.searchsorted(blk, np.arange(blocks + 1))
    lo_cs = np.r_[0.0, cs]
    intra = rng.random(m) < p_in
    n_in = int(intra.sum())
    # intra-block pairs: block ~ tb^2, both ends ~ theta inside the block
    bsel = np.searchsorted(np.cumsum(tb ** 2) / float((tb ** 2).sum()), rng.random(n_in), side="right")
    bsel = np.minimum(bsel, blocks - 1)
    lo = lo_cs[starts[bsel]]
    hi = lo_cs[starts[bsel + 1]]
    u_in = np.searchsorted(cs, lo + rng.random(n_in) * (hi - lo), side="right")
    v_in = np.searchsorted(cs, lo + rng.random(n_in) * (hi - lo), side="right")
    # inter-block pairs: both ends ~ theta over all nodes, resampled while in one block
    n_out = m - n_in
    u_out = np.searchsorted(cs, rng.random(n_out), side="right")
    v_out = np.searchsorted(cs, rng.random(n_out), side="right")
    same = blk[np.minimum(u_out, n - 1)] == blk[np.minimum(v_out, n - 1)]
    while same.any():
        k = int(same.sum())
        v_out[same] = np.searchsorted(cs, rng.random(k), side="right")
        same = blk[np.minimum(u_out, n - 1)] == blk[np.minimum(v_out, n - 1)]
    u = np.minimum(np.r_[u_in, u_out], n - 1)
    v = np.minimum(np.r_[v_in, v_out], n - 1)
    return _pack(n, u, v)


def rmat(scale: int, edge_factor: int, a: float, b: float, c: float, seed: int):
    """R-MAT (recursive matrix) graph with 2**scale nodes and edge_factor * 2**scale edge slots."""
    rng = np.random.default_rng(seed)
    n = 1 << scale
    m = n * edge_factor
    u = np.zeros(m, np.uint32)
    v = np.zeros(m, np.uint32)
    chunk = 1 << 22
    for s in range(0, m, chunk):
        e = min(m, s + chunk)
        uu = np.zeros(e - s, np.uint32)
        vv = np.zeros(e - s, np.uint32)
        for bit in range(scale):
            x = rng.random(e - s)
            row = x >= a + b                       # quadrants c, d
            colb = ((x >= a) & (x < a + b)) | (x >= a + b + c)   # quadrants b, d
            uu |= row.astype(np.uint32) << np.uint32(bit)
            vv |= colb.astype(np.uint32) << np.uint32(bit)
        u[s:e] = uu
        v[s:e] = vv
    return _pack(n, u, v)


def erdos_renyi(n: int, m: int, seed: int):
    """m uniformly random node pairs (duplicates / self-loops possible)."""
    rng = np.random.default_rng(seed)
    return _pack(n, rng.integers(0, n, size=m), rng.integers(0, n, size=m))


def batch_mix(count: int, n_min: int, n_max: int, seed: int):
    """A batch of uneven graphs: grids, random binary trees and BA (m=2) graphs.

    Node counts are log-uniform in [n_min, n_max]; the family is drawn
    uniformly.  Returns a list of (kind, (n, src, dst)).
    """
    rng = np.random.default_rng(seed)
    out = []
    for g in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        kind = ("grid", "tree", "ba")[int(rng.integers(3))]
        sub = int(rng.integers(1 << 31))
        if kind == "grid":
            r = max(2, int(round(math.sqrt(n))))
            cdim = max(2, int(round(n / r)))
            out.append((kind, grid(r, cdim)))
        elif kind == "tree":
            out.append((kind, random_binary_tree(n, sub)))
        else:
            out.append((kind, barabasi_albert(n, 2, sub)))
    return out


def workload(name: str):
    """The named synthetic workloads the layout path is measured and tested on."""
    if name == "grid32":
        return grid(32, 32)
    if name == "ba100k":
        return barabasi_albert(100_000, 3, 1)
    if name == "dcsbm1m":
        return dc_sbm(1_000_000, 64, 2.5, 8.0, 20.0, 2)
    if name == "dcsbm100k":
        return dc_sbm(100_000, 64, 2.5, 8.0, 20.0, 2)
    if name == "rmat22":
        return rmat(22, 8, 0.57, 0.19, 0.19, 4)
    raise KeyError(name)
