"""Paths the benchmark graphs never take, forced on the host: the k-order
rows, plain or capped, when the staging area is too small (all rows, or part
of them, are traversed again at their final offsets), and resuming a level run from its
positions and epoch counter."""
import os

import numpy as np
import pytest

import graphgen as gg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def drg():
    import paper_2008_07799_gb300 as m
    from paper_2008_07799_gb300 import build
    build.build()
    return m


@pytest.mark.parametrize("limit", ["0", "4000"])
@pytest.mark.parametrize("name,k,cap", [("ba", 2, 0), ("ba", 3, 0), ("grid", 2, 0), ("ba", 3, 40), ("grid", 3, 7)])
def test_distance_matrix_without_enough_staging(drg, orc, limit, name, k, cap):
    g = gg.barabasi_albert(3000, 3, 21) if name == "ba" else gg.grid(40, 37)
    old = os.environ.get("DRG_BFS_STAGE_LIMIT")
    os.environ["DRG_BFS_STAGE_LIMIT"] = limit
    try:
        ctx = drg.Context(0, torch.cuda.current_stream().cuda_stream)
    finally:
        if old is None:
            del os.environ["DRG_BFS_STAGE_LIMIT"]
        else:
            os.environ["DRG_BFS_STAGE_LIMIT"] = old
    G = drg.graph_from_edges(ctx, *g)
    D = drg.build_distance_matrix(ctx, G, k, row_cap=cap)
    got = D.download()
    orp, ocol = orc.canonical_graph(*g)
    if cap:
        rp, col, dist, own, back = orc.korder_capped(orp, ocol, k, cap)
        sim = orc.similarity_capped(rp, col, dist, own, back, k, 1.0)
    else:
        rp, col, dist = orc.korder(orp, ocol, k)
        sim = orc.similarity(rp, col, dist, k, 1.0)
    assert np.array_equal(got["rp"], rp) and np.array_equal(got["col"], col) and np.array_equal(got["dist"], dist)
    assert np.array_equal(got["q"], sim["q"])


def test_resume_is_exact_with_one_sample_in_flight(drg):
    # positions + epoch counter are the whole state of a level run: with one
    # sample in flight the run is deterministic, so stopping after epoch 10
    # and resuming gives the same bits as running through
    ctx = drg.Context(0, torch.cuda.current_stream().cuda_stream)
    g = gg.barabasi_albert(1500, 2, 4)
    n = g[0]
    G = drg.graph_from_edges(ctx, *g)
    D = drg.build_distance_matrix(ctx, G, 2)
    p = drg.Params.default(k=2, M=5, epochs=20, b=2.0, mode=1, substeps=n, stop_nodes=200, seed=9)
    H = drg.build_hierarchy(ctx, G, p)
    for level in (0, 1):
        nl = H.sizes()[level]
        p.substeps = nl
        y0 = torch.from_numpy((np.random.default_rng(level).normal(size=2 * nl) * 5).astype(np.float32)).cuda()
        a, b = y0.clone(), y0.clone()
        drg.layout_level(ctx, D, H, level, a, p, 0.1, 0, 20)
        drg.layout_level(ctx, D, H, level, b, p, 0.1, 0, 10)
        drg.layout_level(ctx, D, H, level, b, p, 0.1, 10, 20)
        torch.cuda.synchronize()
        assert torch.equal(a, b)
        assert float((a - y0).abs().max()) > 1e-3
