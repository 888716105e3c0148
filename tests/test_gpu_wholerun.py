"""Whole multilevel runs on the GPU against the oracle's (Sec. 3.2, Fig. 1
pipeline; quality measures of Sec. 4.1).

Single runs diverge chaotically from the oracle's trajectory (any rounding
difference grows), so parity of whole runs is a statement about the
distribution of the result: the neighbourhood preservation (Eq. 15) and
normalised stress (Eq. 16) over the same 96 seeds must agree within 1 % of
the oracle's, compared as 10 %-trimmed means (a rare run that ends with part of
the graph folded away -- stress .61 against .21 for one oracle seed in 48 --
would otherwise move a mean by more than the bar).  The oracle's per-seed
values are in tests/golden/wholerun_quality.json (written by
make_wholerun_quality.py from oracle/ alone); both sides are measured on the
same node and source samples.  The test also checks that twice the bootstrap
standard error of the difference is below 1 % of the mean, so the bar
resolves a 1 % gap.

Configurations: DC-SBM and Barabasi-Albert graphs of 20,000 nodes, heavy-edge
hierarchy to < 1000 nodes, k = 2, M = 5, 500 epochs per level, b = 1; the
GPU's synchronous FP32 mode against the oracle's synchronous mode, and the
bench's Hogwild mode (one launch per level, at most n_l / 16 samples in
flight, epoch gates) against the oracle's sequential loop; and the
synchronous mode with FP16 copies for the negatives' gathers (rewritten after
every sub-step run, so they differ from the masters by rounding only).  In
Hogwild mode the one-launch kernel rewrites the copies once per epoch; that
staleness leaves some DC-SBM runs with a distorted global structure (stress
+6.8 % with FP16, +9.9 % with BF16 copies, NP within 0.6 %), so Hogwild runs
with copies are not held to this bar.
"""
import json
import os

import numpy as np
import pytest

from conftest import golden

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

_GOLD = {}


def _gold():
    if not _GOLD:
        _GOLD.update(json.load(open(golden("wholerun_quality.json"))))
    return _GOLD


@pytest.fixture(scope="module")
def env():
    import paper_2008_07799_gb300 as drg
    from paper_2008_07799_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    return drg, drg.Context(0, torch.cuda.current_stream().cuda_stream)


def _graph(name):
    import graphgen as gg
    g = _gold()["graphs"][name]
    return getattr(gg, g["gen"])(*g["args"])


def _samples(n):
    G = _gold()
    rng = np.random.default_rng(G["sample_seed"])
    nodes = np.sort(rng.choice(n, G["nodes"], replace=False)).astype(np.uint32)
    sources = np.sort(rng.choice(n, G["sources"], replace=False)).astype(np.uint32)
    return nodes, sources


TRIM = 0.1


def _tmean(x):
    from scipy.stats import trim_mean
    return float(trim_mean(x, TRIM))


def _boot_se(x, reps=2000):
    rng = np.random.default_rng(0)
    return float(np.std([_tmean(x[rng.integers(0, len(x), len(x))]) for _ in range(reps)]))


@pytest.mark.parametrize("name", ["dcsbm20k", "ba20k"])
@pytest.mark.parametrize("mode,oracle_mode,precision", [(0, "sync", 0), (1, "sequential", 0), (0, "sync", 1)])
def test_whole_run_quality_matches_oracle(env, orc, name, mode, oracle_mode, precision):
    drg, ctx = env
    n, s, d = _graph(name)
    rp, col = orc.canonical_graph(n, s, d)
    nodes, sources = _samples(n)
    ref = np.array(_gold()["runs"][name][oracle_mode])  # [seed] -> (NP, stress)
    prm = _gold()["params"]
    src = torch.from_numpy(s.view(np.int32)).cuda()
    dst = torch.from_numpy(d.view(np.int32)).cuda()
    got = []
    for seed in range(len(ref)):
        p = drg.Params.default(k=prm["k"], M=prm["M"], epochs=prm["epochs"], b=prm["b"], stop_nodes=prm["stop_nodes"],
                               mode=mode, precision=precision, seed=seed)
        pos = torch.zeros(2 * n, device="cuda")
        drg.layout_edges(ctx, n, src, dst, p, pos)
        Y = pos.cpu().numpy().astype(np.float64).reshape(n, 2)
        got.append((orc.neighbourhood_preservation(rp, col, Y, 2, nodes=nodes),
                    orc.stress(rp, col, Y, sources=sources)))
    got = np.array(got)
    for c, what in ((0, "NP"), (1, "stress")):
        m_ref, m_got = _tmean(ref[:, c]), _tmean(got[:, c])
        res = 2 * np.hypot(_boot_se(ref[:, c]), _boot_se(got[:, c]))
        print(f"{name} {oracle_mode} precision {precision} {what}: GPU {m_got:.5f} oracle {m_ref:.5f} "
              f"({(m_got / m_ref - 1) * 100:+.2f} %, 2 SE {res / m_ref * 100:.2f} %)")
        assert res < 0.01 * m_ref, f"{what}: seeds do not resolve 1 % ({res:.3g} vs mean {m_ref:.4g})"
        assert abs(m_got - m_ref) <= 0.01 * m_ref, (what, m_got, m_ref, res)
