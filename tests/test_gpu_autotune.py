"""The launch-shape autotuner of the Hogwild level kernels: a long run tunes
its shape once per key, later runs reuse it, the chosen shape is one of the
candidates, and runs with a tuned shape lay out as well as with the default
(the shape changes only thread timing).  Switching the tuner off keeps the
default shape and tunes nothing."""
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
    return drg, drg.Context(0, torch.cuda.current_stream().cuda_stream)


def _np(orc, g, Y):
    rp, col = orc.canonical_graph(*g)
    return orc.neighbourhood_preservation(rp, col, Y, 2)


def test_tuned_shapes_and_quality(env, orc):
    # NP varies by ~15 % from seed to seed on this graph, so tuned and
    # default runs are compared as means over 16 seeds each, within three
    # standard errors of their difference
    drg, ctx = env
    g = gg.barabasi_albert(8000, 3, 21)
    n = g[0]
    p = drg.Params.default(k=2, M=5, epochs=120, b=1.0, mode=1, stop_nodes=1000, seed=2)
    quality = {}
    for on in (False, True):
        drg.autotune_clear()
        ctx.autotune(on)
        nps = []
        for seed in range(16):
            pos = torch.zeros(2 * n, device="cuda")
            drg.layout_edges(ctx, n, g[1], g[2], p.replace(seed=seed), pos)
            Y = pos.cpu().numpy().astype(np.float64).reshape(n, 2)
            assert np.all(np.isfinite(Y))
            nps.append(_np(orc, g, Y))
        quality[on] = np.array(nps)
        table = drg.autotune_table()
        if not on:
            assert table == []
        else:
            assert table, "no shape tuned"
            for e in table:
                assert e["kernel"] == "k_hogwild" and e["block"] in (64, 128, 256) and e["divisor"] in (1, 2, 4)
                assert e["M"] == 5 and e["ms_per_epoch"] > 0
            # one entry per size bucket of the levels (each level once, reused by later seeds)
            assert len({(e["ancestors"], e["bucket"]) for e in table}) == len(table)
    ctx.autotune(True)
    se = np.hypot(*(np.std(q, ddof=1) / np.sqrt(len(q)) for q in quality.values()))
    assert abs(quality[True].mean() - quality[False].mean()) <= 3 * se, (quality, se)


def test_batch_block_size_is_tuned(env):
    drg, ctx = env
    drg.autotune_clear()
    ctx.autotune(True)
    items = gg.batch_mix(12, 1000, 6000, 5)
    graphs = [drg.graph_from_edges(ctx, *gph) for _, gph in items]
    pos = [torch.zeros(2 * gph[0], device="cuda") for _, gph in items]
    p = drg.Params.default(k=2, M=5, epochs=60, b=2.0, mode=1, stop_nodes=300, seed=1)
    drg.layout_batch(ctx, graphs, p, pos)
    for x in pos:
        assert torch.isfinite(x).all()
    table = [e for e in drg.autotune_table() if e["kernel"] == "k_hogwild_batch"]
    assert table and all(e["block"] in (64, 128, 256) and e["divisor"] == 1 for e in table)
