"""Parity at the workloads' own sizes, in the same launch configuration as
the benchmark, on outputs the oracle can compute one by one (sampled rows of
the distance matrix, their similarity weights, hierarchies) and on properties
that hold at any size (the alias tables represent the weights they were built
from; isolated nodes never move).

Workloads: Barabasi-Albert 100,000 nodes m=3 (k=3, multilevel), the
degree-corrected block model with 1,000,000 nodes (k=2, the benchmark graph)
and R-MAT scale 22 (k=1, mixed precision, Hogwild).
"""
import numpy as np
import pytest

import graphgen as gg

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def env():
    import paper_2008_07799_gb300 as drg
    from paper_2008_07799_gb300 import build
    build.build()
    ctx = drg.Context(0, torch.cuda.current_stream().cuda_stream)
    return drg, ctx


def _check_graph(drg, ctx, orc, g):
    G = drg.graph_from_edges(ctx, *g)
    rp, col, _ = G.download()
    orp, ocol = orc.canonical_graph(*g)
    assert np.array_equal(rp, orp) and np.array_equal(col, ocol)
    return G, orp, ocol


def _check_rows(drg, D, orc, orp, ocol, k, rows, entries_only=()):
    """Sampled rows: entries, distances, FP32 weights, row sums -- exact.
    Rows in `entries_only` are checked for their entries and distances only."""
    nodes = D.download_nodes()
    rb = orc.RowBFS(orp, ocol, k)
    g = orc.gaussians(k)
    got_rows = {}
    need = set(int(i) for i in rows)
    for i in list(rows) + list(entries_only):
        c, d = rb.row(int(i))
        e0, e1 = int(nodes["rp"][i]), int(nodes["rp"][i + 1])
        assert e1 - e0 == len(c), i
        got = D.download_range(e0, e1)
        assert np.array_equal(got["col"], c) and np.array_equal(got["dist"], d), i
        if i in entries_only:
            continue
        got_rows[int(i)] = (c, d, got)
        need.update(int(x) for x in c)
    need = np.array(sorted(need), np.uint32)
    counts = orc.class_counts(orp, ocol, k, need)
    Z = {int(v): orc.normaliser(counts[x], g) for x, v in enumerate(need)}
    for i, (c, d, got) in got_rows.items():
        assert np.float32(Z[i]) == nodes["Z"][i]
        q = np.array([orc.entry_weight(g[dd - 1], Z[i], Z[int(j)]) for j, dd in zip(c, d)], np.uint32)
        assert np.array_equal(got["q"], q), i
        assert int(nodes["r"][i]) == int(q.astype(np.uint64).sum()), i
    return nodes


def _check_alias_represents(thresh, alias, weights):
    """The table draws item i with probability weights_i / W: per item, the
    table's mass (in units of 2^-32 / N) is within the rounding of each
    bucket that holds part of it, and every alias lands on an item whose
    scaled weight reaches the capacity (a heavy item) or on itself."""
    N = len(weights)
    w = weights.astype(np.float64)
    W = w.sum()
    t = thresh.astype(np.float64)
    mass = np.bincount(np.arange(N), weights=t, minlength=N) + np.bincount(alias.astype(np.int64),
                                                                            weights=2.0 ** 32 - t, minlength=N)
    holders = 1 + np.bincount(alias.astype(np.int64), minlength=N)
    expect = w * N * 2.0 ** 32 / W
    assert np.all(np.abs(mass - expect) <= holders + 1e-6 * expect)
    self_alias = alias == np.arange(N)
    heavy = weights.astype(np.float64) * N >= W * (1 - 1e-12)
    assert np.all(self_alias | heavy[alias.astype(np.int64)])


def test_ba100k_k3(env, orc):
    drg, ctx = env
    g = gg.workload("ba100k")
    G, orp, ocol = _check_graph(drg, ctx, orc, g)
    D = drg.build_distance_matrix(ctx, G, 3)
    n = g[0]
    rows = np.random.default_rng(1).choice(n, 60, replace=False)
    rows = np.r_[rows, [0, 1, 2, n - 1]]  # the oldest BA nodes are the hubs
    nodes = _check_rows(drg, D, orc, orp, ocol, 3, rows)
    # full row pointer from the oracle's class counts of every node
    counts = orc.class_counts(orp, ocol, 3, np.arange(n, dtype=np.uint32))
    rp = np.zeros(n + 1, np.uint64)
    np.cumsum(counts.sum(axis=1), out=rp[1:])
    assert np.array_equal(nodes["rp"], rp)
    full = D.download()
    _check_alias_represents(full["e_thresh"], full["e_alias"], full["q"])
    r32 = (full["r"] >> np.uint64(full["shift"])).astype(np.uint64)
    assert int(full["r"].max()) >> full["shift"] < 2 ** 32 and (full["shift"] == 0 or int(full["r"].max()) >> (full["shift"] - 1) >= 2 ** 32)
    _check_alias_represents(full["v_thresh"], full["v_alias"], r32)
    # the whole hierarchy, exactly
    p = drg.Params.default(k=3, stop_nodes=1000, seed=0)
    H = drg.build_hierarchy(ctx, G, p)
    levels = orc.hierarchy(orp, ocol, orc.Params(stop_nodes=1000, seed=0))
    assert H.sizes() == [lv.n for lv in levels]
    for l in range(1, len(levels)):
        assert np.array_equal(H.parent(l - 1), levels[l - 1].parent)
        crp, ccol, cw = H.graph(l).download()
        assert np.array_equal(crp, levels[l].rp) and np.array_equal(ccol, levels[l].col)
        assert np.array_equal(cw, levels[l].w)


def test_dcsbm1m_k2(env, orc):
    drg, ctx = env
    g = gg.workload("dcsbm1m")
    G, orp, ocol = _check_graph(drg, ctx, orc, g)
    D = drg.build_distance_matrix(ctx, G, 2)
    n = g[0]
    deg = np.diff(orp).astype(np.int64)
    rng = np.random.default_rng(2)
    rows = rng.choice(np.nonzero(deg > 0)[0], 24, replace=False)
    nodes = _check_rows(drg, D, orc, orp, ocol, 2, rows, entries_only=(int(np.argmax(deg)),))
    assert nodes["nnz"] == int(nodes["rp"][-1]) and nodes["nnz"] < 2 ** 32
    # first coarsening level, exactly
    p = drg.Params.default(k=2, stop_nodes=1000, seed=0)
    parent = torch.zeros(n, dtype=torch.int32, device="cuda")
    C1 = drg.coarsen(ctx, G, 0, p, parent)
    cid, nc = orc.cluster_ids(orc.hem_match(orp, ocol, None, orc.Params(seed=0), 0))
    assert np.array_equal(parent.cpu().numpy().astype(np.uint32), cid)
    crp, ccol, cw = orc.contract(orp, ocol, None, cid, nc)
    rp1, col1, w1 = C1.download()
    assert np.array_equal(rp1, crp) and np.array_equal(col1, ccol) and np.array_equal(w1, cw)


def test_rmat22_k1_mixed_hogwild(env, orc):
    drg, ctx = env
    g = gg.workload("rmat22")
    G, orp, ocol = _check_graph(drg, ctx, orc, g)
    n = g[0]
    deg = np.diff(orp).astype(np.int64)
    D = drg.build_distance_matrix(ctx, G, 1)
    rows = np.r_[np.random.default_rng(4).choice(np.nonzero(deg > 0)[0], 40, replace=False), [int(np.argmax(deg))]]
    _check_rows(drg, D, orc, orp, ocol, 1, rows)
    # the whole path: multilevel, k=1, M=5, 300 epochs per level, FP16 gathers, Hogwild
    p = drg.Params.default(k=1, M=5, epochs=300, b=1.0, mode=1, precision=1, stop_nodes=1000, seed=4)
    pos = torch.zeros(2 * n, device="cuda")
    drg.layout(ctx, G, p, pos)
    torch.cuda.synchronize()
    Y = pos.cpu().numpy().reshape(-1, 2)
    assert np.all(np.isfinite(Y))
    iso = deg == 0
    # isolated nodes are never drawn, so they keep their coarsest-level start
    assert np.all(np.abs(Y[iso]) <= 1e-4)
    assert np.ptp(Y[~iso], axis=0).max() > 10.0


def test_dcsbm1m_hogwild_matches_sync_quality(env, orc):
    """Whole runs on the benchmark graph: the one-launch Hogwild levels keep the
    local quality of the synchronous method (NP on 2000 sampled nodes within
    10 %).  Epochs must stay in step: without the epoch barrier NP fell to .024
    against .039."""
    drg, ctx = env
    g = gg.workload("dcsbm1m")
    n = g[0]
    rp, col = orc.canonical_graph(*g)
    deg = np.diff(rp)
    nodes = np.random.default_rng(0).choice(np.nonzero(deg > 0)[0], 2000, replace=False).astype(np.uint32)
    G = drg.graph_from_edges(ctx, *g)
    nps = {}
    for mode in (0, 1):
        p = drg.Params.default(k=2, M=5, epochs=500, b=1.0, mode=mode, stop_nodes=1000, seed=0)
        pos = torch.zeros(2 * n, device="cuda")
        drg.layout(ctx, G, p, pos)
        Y = pos.cpu().numpy().astype(np.float64).reshape(-1, 2)
        nps[mode] = orc.neighbourhood_preservation(rp, col, Y, 2, nodes)
    assert nps[1] >= 0.9 * nps[0], nps


def test_dcsbm1m_star_hierarchy_and_quality(env, orc):
    """The paper's star grouping on the benchmark graph: the whole hierarchy
    exactly as the oracle's walk gives it, and a whole Hogwild run on it.
    Groups of a node with all its ungrouped neighbours shrink the graph faster
    than pairs (4 levels, 1.96M samples per epoch over all levels against 5
    levels and 2.64M) and refinement starts each neighbourhood at one point:
    NP on 2000 sampled nodes measured .0293 against .0395 with heavy-edge
    matching.  The bar keeps that ratio (0.74) with margin and stays far above
    a random layout (NP ~ 1e-4)."""
    drg, ctx = env
    g = gg.workload("dcsbm1m")
    n = g[0]
    rp, col = orc.canonical_graph(*g)
    G = drg.graph_from_edges(ctx, *g)
    H = drg.build_hierarchy(ctx, G, drg.Params.default(k=2, stop_nodes=1000, seed=0, coarsen=1))
    levels = orc.hierarchy(rp, col, orc.Params(stop_nodes=1000, seed=0, coarsen=1))
    assert H.sizes() == [lv.n for lv in levels]
    for l in range(1, len(levels)):
        assert np.array_equal(H.parent(l - 1), levels[l - 1].parent)
        crp, ccol, cw = H.graph(l).download()
        assert np.array_equal(crp, levels[l].rp) and np.array_equal(ccol, levels[l].col)
        assert np.array_equal(cw, levels[l].w)
    deg = np.diff(rp)
    nodes = np.random.default_rng(0).choice(np.nonzero(deg > 0)[0], 2000, replace=False).astype(np.uint32)
    nps = {}
    for rule in (0, 1):
        p = drg.Params.default(k=2, M=5, epochs=500, b=1.0, mode=1, stop_nodes=1000, seed=0, coarsen=rule)
        pos = torch.zeros(2 * n, device="cuda")
        drg.layout(ctx, G, p, pos)
        Y = pos.cpu().numpy().astype(np.float64).reshape(-1, 2)
        nps[rule] = orc.neighbourhood_preservation(rp, col, Y, 2, nodes)
    assert nps[1] >= 0.65 * nps[0] and nps[1] > 0.02, nps


def test_dcsbm1m_perplexity_calibration(env, orc):
    """sigma_i calibrated per node on the 3.4e9-entry k=2 matrix of the bench
    graph: beta_i of sampled rows (the hubs among them) bit for bit against
    the oracle's calibration of the same class counts."""
    drg, ctx = env
    g = gg.workload("dcsbm1m")
    n = g[0]
    rp, col = orc.canonical_graph(*g)
    G = drg.graph_from_edges(ctx, *g)
    D = drg.build_distance_matrix(ctx, G, 2, perplexity=30.0)
    beta = D.calibration()
    deg = np.diff(rp).astype(np.int64)
    rows = np.r_[np.random.default_rng(5).choice(np.nonzero(deg > 0)[0], 40, replace=False),
                 np.argsort(deg)[-4:]].astype(np.uint32)
    counts = orc.class_counts(rp, col, 2, rows)
    for x, i in enumerate(rows):
        want = orc.calibrate_row(counts[x], 30.0)
        assert beta[i].view(np.uint64) == np.float64(want).view(np.uint64), (int(i), beta[i], want)
    assert np.all(beta[deg == 0] == 0.0)
