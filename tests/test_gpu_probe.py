"""The memory probes that give the level kernels' roofline its measured
ceilings: every kind runs, counts what it did, and the ceilings order as the
memory hierarchy says they must (random reads that stay in L2 beat random
reads of HBM, also when loads and atomic adds are mixed; a streaming copy
moves far more bytes than random 16-byte reads).  Arguments outside the documented ranges are refused before any
device work."""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def env():
    import paper_2008_07799_gb300 as drg
    from paper_2008_07799_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    return drg, drg.Context(0, torch.cuda.current_stream().cuda_stream)


def test_probe_kinds_and_ordering(env):
    drg, ctx = env
    rate = {}
    for name, kind, size, count in (("l2_load8", drg.PROBE_LOAD8, 32 << 20, 50_000_000),
                                    ("l2_load16", drg.PROBE_LOAD16, 32 << 20, 50_000_000),
                                    ("l2_red8", drg.PROBE_RED8, 32 << 20, 50_000_000),
                                    ("l2_mix", drg.PROBE_MIX_LOAD8_RED8, 32 << 20, 48_000_000),
                                    ("hbm_load16", drg.PROBE_LOAD16, 2 << 30, 10_000_000),
                                    ("hbm_ef", drg.PROBE_LOAD16_EVICT_FIRST, 2 << 30, 10_000_000)):
        drg.probe_memory(ctx, kind, size, count)  # warm-up
        ms, done = drg.probe_memory(ctx, kind, size, count)
        assert done >= count and ms > 0
        rate[name] = done / ms * 1e3
    ms, vecs = drg.probe_memory(ctx, drg.PROBE_COPY, 2 << 30, 1)
    assert vecs == (2 << 30) // 32
    copy_gbs = vecs * 32 / ms / 1e6
    assert rate["l2_load8"] > 2 * rate["hbm_load16"], rate
    assert rate["l2_mix"] > 2 * rate["hbm_load16"], rate
    assert copy_gbs > rate["hbm_load16"] * 16 / 1e9, (copy_gbs, rate)
    assert copy_gbs > 1000, copy_gbs


def test_probe_refuses_bad_arguments(env):
    drg, ctx = env
    L = drg.lib()
    import ctypes as C
    ms, done = C.c_double(), C.c_uint64()
    assert L.drg_probe_memory(ctx.h, 9, 32 << 20, 1000, 1, C.byref(ms), C.byref(done)) == 1       # kind
    assert L.drg_probe_memory(ctx.h, 0, 1 << 10, 1000, 1, C.byref(ms), C.byref(done)) == 1        # buffer < 1 MiB
    assert L.drg_probe_memory(ctx.h, 0, 32 << 20, 0, 1, C.byref(ms), C.byref(done)) == 1          # no accesses
    assert L.drg_probe_memory(ctx.h, 0, 32 << 20, 1000, 9, C.byref(ms), C.byref(done)) == 1       # blocks per SM
    assert L.drg_probe_memory(ctx.h, 0, 1 << 50, 1000, 1, C.byref(ms), C.byref(done)) == 1       # > 64 GiB
