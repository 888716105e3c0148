"""The epoch gates of a Hogwild level run (a warp waits for the others'
completion counters before it runs ahead): a wait completes when every
expected arrival comes, and when one cannot (a gate that expects more
arrivals than run) every wait ends after its limit with DRG_ETIMEOUT and the
context stays usable."""
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
    return drg, drg.Context(0, torch.cuda.current_stream().cuda_stream)


def test_barrier_completes(env):
    drg, ctx = env
    for blocks in (1, 2, 7):
        assert drg.check_epoch_barrier(ctx, blocks, blocks, rounds=50, timeout_ms=2000) == 0


def test_barrier_times_out_and_context_survives(env):
    drg, ctx = env
    assert drg.check_epoch_barrier(ctx, 2, 3, rounds=3, timeout_ms=50) == 4   # DRG_ETIMEOUT
    assert drg.check_epoch_barrier(ctx, 3, 3, rounds=3, timeout_ms=2000) == 0
    # the library still works on this context afterwards
    g = gg.barabasi_albert(2000, 2, 3)
    p = drg.Params.default(k=2, M=5, epochs=20, b=2.0, mode=1, stop_nodes=200, seed=1)
    pos = torch.zeros(2 * 2000, device="cuda")
    drg.layout_edges(ctx, g[0], g[1], g[2], p, pos)
    assert torch.isfinite(pos).all() and float(pos.abs().max()) > 0.1


def test_barrier_argument_errors(env):
    drg, ctx = env
    assert drg.check_epoch_barrier(ctx, 0, 1) == 1
    assert drg.check_epoch_barrier(ctx, 1, 1, timeout_ms=0) == 1
