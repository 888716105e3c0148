"""The allocation-free level run, for callers that cannot allocate device
memory while they run, against the ordinary level run.

drg_layout_level_noalloc keeps its gradient buffer and epoch state in a
static device array instead of allocating them per call.  It must give the
same layout as drg_layout_level (within the per-epoch tolerance of the parity
tests, 1e-5 of the layout extent: the two differ only in the order of FP32
atomic adds) on consecutive calls that share that array, and refuse what the
array cannot hold.  This file is collected last and runs alone as well.
"""
import ctypes as C

import numpy as np
import pytest

import graphgen as gg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def env():
    import paper_2008_07799_gb300 as drg
    from paper_2008_07799_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    ctx = drg.Context(0, torch.cuda.current_stream().cuda_stream)
    return drg, ctx


def _noalloc(drg, ctx, D, H, level, pos, p, gamma, t0, t1):
    return drg.lib().drg_layout_level_noalloc(ctx.h, D.h, None if H is None else H.h, level, pos.data_ptr(),
                                              C.byref(p), gamma, t0, t1)


def test_two_calls_in_a_row_match_layout_level(env):
    drg, ctx = env
    g = gg.barabasi_albert(3000, 3, 5)
    G = drg.graph_from_edges(ctx, *g)
    D = drg.build_distance_matrix(ctx, G, 2)
    p = drg.Params.default(k=2, M=5, epochs=100, b=1.0, mode=0, stop_nodes=300, seed=9)
    H = drg.build_hierarchy(ctx, G, p)
    sizes = H.sizes()
    assert len(sizes) >= 2
    for level in (0, 1):  # level 1 goes through the ancestor map
        n = sizes[level]
        Y0 = (np.random.default_rng(level).normal(size=(n, 2)) * 8).astype(np.float32)
        cur = torch.from_numpy(Y0.reshape(-1)).cuda()
        for t in (40, 41):  # consecutive calls share the static scratch
            before = cur.clone()
            ref = cur.clone()
            drg.layout_level(ctx, D, H, level, ref, p, 0.1, t, t + 1)
            st = _noalloc(drg, ctx, D, H, level, cur, p, 0.1, t, t + 1)
            assert st == 0, drg.lib().drg_last_error(ctx.h)
            torch.cuda.synchronize()
            got = cur.cpu().numpy().astype(np.float64).reshape(n, 2)
            want = ref.cpu().numpy().astype(np.float64).reshape(n, 2)
            ext = float(np.max(np.ptp(want, axis=0)))
            assert np.max(np.abs(got - want)) <= 1e-5 * ext, (level, t)
            assert torch.max(torch.abs(cur - before)).item() > 1e-3  # the epoch moved the layout


def test_coarse_level_with_its_own_tables(env):
    # a coarse level's own distance matrix (no ancestor map), as drg_layout_level takes it
    drg, ctx = env
    g = gg.barabasi_albert(3000, 3, 6)
    G = drg.graph_from_edges(ctx, *g)
    p = drg.Params.default(k=2, M=5, epochs=100, b=1.0, mode=0, stop_nodes=300, seed=4)
    H = drg.build_hierarchy(ctx, G, p)
    D1 = drg.build_distance_matrix(ctx, H.graph(1), 2)
    n = H.sizes()[1]
    cur = torch.from_numpy((np.random.default_rng(7).normal(size=(n, 2)) * 8).astype(np.float32).reshape(-1)).cuda()
    for t in (10, 11):
        ref = cur.clone()
        drg.layout_level(ctx, D1, H, 1, ref, p, 0.1, t, t + 1)
        st = _noalloc(drg, ctx, D1, H, 1, cur, p, 0.1, t, t + 1)
        assert st == 0, drg.lib().drg_last_error(ctx.h)
        torch.cuda.synchronize()
        got = cur.cpu().numpy().astype(np.float64).reshape(n, 2)
        want = ref.cpu().numpy().astype(np.float64).reshape(n, 2)
        ext = float(np.max(np.ptp(want, axis=0)))
        assert np.max(np.abs(got - want)) <= 1e-5 * ext, t


def test_limits_are_refused(env):
    drg, ctx = env
    g = gg.grid(8, 8)
    G = drg.graph_from_edges(ctx, *g)
    D = drg.build_distance_matrix(ctx, G, 1)
    pos = torch.zeros(2 * 64, device="cuda")
    p = drg.Params.default(k=1, epochs=10, mode=1)
    assert _noalloc(drg, ctx, D, None, 0, pos, p, 0.1, 0, 1) == 5       # Hogwild: unsupported
    p = drg.Params.default(k=1, epochs=10, mode=0, precision=1)
    assert _noalloc(drg, ctx, D, None, 0, pos, p, 0.1, 0, 1) == 5       # half-precision copies: unsupported
    n = (1 << 20) + 1                                                     # one node beyond the static scratch
    big = drg.graph_from_edges(ctx, *gg.path(n))
    Db = drg.build_distance_matrix(ctx, big, 1)
    posb = torch.zeros(2 * n, device="cuda")
    p = drg.Params.default(k=1, epochs=10, mode=0)
    assert _noalloc(drg, ctx, Db, None, 0, posb, p, 0.1, 0, 1) == 5
    assert b"1048576" in drg.lib().drg_last_error(ctx.h)
