"""drg_layout_step_explicit: one synchronous step over caller-given samples
(Eqs. 11-12 with the samples fixed instead of drawn).

- The samples of one oracle epoch, passed explicitly, move the layout as the
  oracle's synchronous epoch in a single run does (within the per-epoch bar,
  1e-5 of the extent).
- The equilibrium of Eq. 12: a source with its positive target at distance
  d* = (M gamma)^(1/2b) and all M negatives at the target's place (another
  node there) feels no net force, while the target and the negatives move.
- Finite differences of the sampled objective (Eq. 11) of random samples
  match the step's update for every node and role.
- Ids >= n and invalid parameters are refused.
"""
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


def _u32(x):
    return torch.from_numpy(np.ascontiguousarray(x, np.uint32).view(np.int32)).cuda()


def test_oracle_epoch_as_explicit_samples(env, orc):
    drg, ctx = env
    n, s, d = gg.barabasi_albert(1500, 3, 9)
    rp, col = orc.canonical_graph(n, s, d)
    gd = orc.korder(rp, col, 2)
    tab, _ = orc.sampling_tables(*gd, 2)
    M, t, gamma, b = 5, 7, 0.1, 1.0
    p = orc.Params(k=2, M=M, epochs=100, b=b, mode=0, substeps=1, seed=3)
    Y0 = (np.random.default_rng(1).normal(size=(n, 2)) * 10).astype(np.float32).astype(np.float64)
    ref = orc.layout_level(tab, Y0.copy(), 0, None, p, gamma, t, t + 1)
    draws = [orc.sample_draws(tab, p.seed, p.gid, 0, t, x, M) for x in range(n)]
    src = _u32([x[0] for x in draws])
    dst = _u32([x[1] for x in draws])
    neg = _u32(np.concatenate([x[2] for x in draws]))
    pos = torch.from_numpy(Y0.astype(np.float32).reshape(-1)).cuda()
    lr = p.lr0 * (1 - t / p.epochs)
    drg.layout_step_explicit(ctx, pos, src, dst, neg, M, gamma, b, lr, p.clip)
    got = pos.cpu().numpy().astype(np.float64).reshape(n, 2)
    ext = float(np.max(np.ptp(ref, axis=0)))
    assert np.max(np.abs(ref - Y0)) > 1e-3
    assert np.max(np.abs(got - ref)) <= 1e-5 * ext


@pytest.mark.parametrize("b,M,gamma", [(1.0, 5, 0.1), (2.0, 3, 0.3), (3.0, 5, 0.1)])
def test_equilibrium_distance(env, b, M, gamma):
    drg, ctx = env
    dstar = (M * gamma) ** (1.0 / (2 * b))
    Y = np.array([[0.0, 0.0], [dstar, 0.0], [dstar, 0.0]], np.float32)  # source, target, a node at the target
    pos = torch.from_numpy(Y.reshape(-1)).cuda()
    drg.layout_step_explicit(ctx, pos, _u32([0]), _u32([1]), _u32([2] * M), M, gamma, b, 1.0, 1e30)
    out = pos.cpu().numpy().reshape(3, 2).astype(np.float64)
    attr = 2 * b * dstar ** (2 * b - 1) / (1 + dstar ** (2 * b))  # size of the attraction at d*
    assert np.max(np.abs(out[0])) <= 1e-5 * attr               # no net force on the source
    assert abs((out[1, 0] - dstar) + attr) <= 1e-5 * attr      # the target moves back by the attraction
    assert abs((out[2, 0] - dstar) - attr) <= 1e-5 * attr      # the negatives, summed, push it away as much


def test_update_is_gradient_of_sampled_objective(env, orc):
    drg, ctx = env
    rng = np.random.default_rng(5)
    n, S, M, gamma, b = 12, 20, 3, 0.3, 1.5
    Y0 = rng.normal(size=(n, 2)) * 1.3
    a = rng.integers(0, n, S)
    c = (a + rng.integers(1, n, S)) % n
    negs = rng.integers(0, n, (S, M))
    pos = torch.from_numpy(Y0.astype(np.float32).reshape(-1)).cuda()
    drg.layout_step_explicit(ctx, pos, _u32(a), _u32(c), _u32(negs.reshape(-1)), M, gamma, b, 1.0, 1e30)
    G = pos.cpu().numpy().astype(np.float64).reshape(n, 2) - Y0.astype(np.float32).astype(np.float64)
    Yf = Y0.astype(np.float32).astype(np.float64)

    def objective(Y):
        tot = 0.0
        for x in range(S):
            keep = [m for m in negs[x] if m != a[x] and m != c[x]]
            tot += orc.sample_objective(Y[a[x]], Y[c[x]], Y[keep].reshape(-1, 2), gamma, b)
        return tot

    h = 1e-6
    num = np.zeros_like(Yf)
    for v in range(n):
        for x in range(2):
            e = np.zeros_like(Yf)
            e[v, x] = h
            num[v, x] = (objective(Yf + e) - objective(Yf - e)) / (2 * h)
    assert np.allclose(G, num, rtol=2e-4, atol=2e-4 * np.max(np.abs(num)))


def test_refusals(env):
    drg, ctx = env
    L = drg.lib()
    pos = torch.zeros(2 * 4, device="cuda")
    ok = _u32([0, 1])
    bad = _u32([0, 4])
    negs = _u32([2, 3])
    assert L.drg_layout_step_explicit(ctx.h, 4, pos.data_ptr(), 2, bad.data_ptr(), ok.data_ptr(), negs.data_ptr(),
                                      1, 0.1, 1.0, 1.0, 5.0) == 1
    assert L.drg_layout_step_explicit(ctx.h, 4, pos.data_ptr(), 2, ok.data_ptr(), ok.data_ptr(), negs.data_ptr(),
                                      65, 0.1, 1.0, 1.0, 5.0) == 1
    assert L.drg_layout_step_explicit(ctx.h, 4, pos.data_ptr(), 2, ok.data_ptr(), ok.data_ptr(), negs.data_ptr(),
                                      1, 0.1, 0.0, 1.0, 5.0) == 1
    assert L.drg_layout_step_explicit(ctx.h, 4, pos.data_ptr(), 0, None, None, None, 1, 0.1, 1.0, 1.0, 5.0) == 0
