"""Pins of the CPU oracle against things other than itself (CPU only).

Philox against the published known-answer vectors; the k-order distance
matrix against closed forms and scipy's all-pairs shortest paths; the
similarity against its normalisation identities; the alias tables against
exact mass conservation, brute-force enumeration and a chi-square test.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.csgraph as csg
from scipy import stats

import graphgen as gg
from conftest import golden


# ---------------------------------------------------------------- Philox
def test_philox_known_answers(orc):
    rows = [l.split() for l in open(golden("philox_kat.txt")) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = orc.philox(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_philox_counter_sensitivity(orc):
    base = orc.philox([1, 2, 3, 4], [5, 6])
    for lane in range(4):
        c = [1, 2, 3, 4]
        c[lane] ^= 1
        assert not np.array_equal(orc.philox(c, [5, 6]), base)
    assert not np.array_equal(orc.philox([1, 2, 3, 4], [5, 7]), base)


# ---------------------------------------------------------------- distance matrix
def _dense_from_gd(gd, n):
    rp, col, dist = gd
    D = np.zeros((n, n), np.int64)
    rows = np.repeat(np.arange(n), np.diff(rp).astype(np.int64))
    D[rows, col.astype(np.int64)] = dist
    return D


def _expected_dense(spd, k):
    n = spd.shape[0]
    E = np.where((spd <= k) & (spd > 0), spd, 0)
    E[np.arange(n), np.arange(n)] = 0
    return E.astype(np.int64)


@pytest.mark.parametrize("k", [1, 2, 3, 5])
def test_korder_path_cycle_grid_closed_forms(orc, k):
    n = 23
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    cases = [
        (gg.path(n), np.abs(ii - jj)),
        (gg.cycle(n), np.minimum(np.abs(ii - jj), n - np.abs(ii - jj))),
    ]
    R, Cc = 5, 7
    r, c = np.divmod(np.arange(R * Cc), Cc)
    cases.append((gg.grid(R, Cc), np.abs(r[:, None] - r[None, :]) + np.abs(c[:, None] - c[None, :])))
    for (nn, s, d), spd in cases:
        rp, col = orc.canonical_graph(nn, s, d)
        gd = orc.korder(rp, col, k)
        assert np.array_equal(_dense_from_gd(gd, nn), _expected_dense(spd, k))
        # rows sorted strictly ascending
        for i in range(nn):
            row = gd[1][gd[0][i]:gd[0][i + 1]]
            assert np.all(np.diff(row.astype(np.int64)) > 0)


def _grid_count(R, Cc, k):
    """Number of ordered pairs of distinct grid points at Manhattan distance <= k."""
    r, c = np.divmod(np.arange(R * Cc), Cc)
    tot = 0
    for i in range(R * Cc):
        d = np.abs(r - r[i]) + np.abs(c - c[i])
        tot += int(((d > 0) & (d <= k)).sum())
    return tot


def test_korder_grid32_counts(orc):
    n, s, d = gg.grid(32, 32)
    rp, col = orc.canonical_graph(n, s, d)
    assert len(col) == 2 * 1984
    for k, expect in [(1, 3968), (2, 11652), (3, 22804)]:
        gd = orc.korder(rp, col, k)
        assert len(gd[1]) == expect == _grid_count(32, 32, k)
        interior = 5 * 32 + 5
        assert gd[0][interior + 1] - gd[0][interior] == 2 * k * (k + 1)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_korder_vs_scipy_shortest_path(orc, seed):
    n, s, d = gg.erdos_renyi(60, 90, seed)
    rp, col = orc.canonical_graph(n, s, d)
    A = sp.csr_matrix((np.ones(len(col)), col.astype(np.int64), rp.astype(np.int64)), shape=(n, n))
    spd = csg.shortest_path(A, unweighted=True, directed=False)
    spd[np.isinf(spd)] = 10 ** 6
    for k in (1, 2, 3, 4):
        gd = orc.korder(rp, col, k)
        D = _dense_from_gd(gd, n)
        assert np.array_equal(D, _expected_dense(spd.astype(np.int64), k))
        assert np.array_equal(D, D.T)  # GD is symmetric


def test_canonical_graph_drops_loops_and_duplicates(orc):
    rp, col = orc.canonical_graph(4, np.array([0, 1, 1, 2, 3, 3]), np.array([1, 0, 1, 3, 2, 2]))
    assert rp.tolist() == [0, 1, 2, 3, 4]
    assert col.tolist() == [1, 0, 3, 2]


# ---------------------------------------------------------------- similarity
def _sim_for(orc, g, k, sigma=1.0):
    n, s, d = g
    rp, col = orc.canonical_graph(n, s, d)
    gd = orc.korder(rp, col, k)
    return n, rp, col, gd, orc.similarity(*gd, k, sigma)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_similarity_normalisation(orc, k):
    n, rp, col, gd, sim = _sim_for(orc, gg.barabasi_albert(300, 2, 7), k, sigma=1.3)
    s32 = float(np.float32(1.3))   # sigma is an FP32 parameter
    g64 = np.exp(-np.arange(1, k + 1) ** 2 / (2 * s32 ** 2))
    assert np.allclose(sim["g"], g64.astype(np.float32), rtol=0, atol=0)
    rows = np.repeat(np.arange(n), np.diff(gd[0]).astype(np.int64))
    dist = gd[2].astype(np.int64)
    # conditional similarities of every row sum to one (Eq. 9)
    Zrow = np.zeros(n)
    np.add.at(Zrow, rows, g64[dist - 1])
    cond = g64[dist - 1] / Zrow[rows]
    sums = np.zeros(n)
    np.add.at(sums, rows, cond)
    assert np.allclose(sums, 1.0)
    assert np.allclose(sim["Z"], Zrow.astype(np.float32), rtol=1e-6)
    # symmetric joint similarity summing to one (Eq. 4)
    ns = sim["ns"]
    key = rows * n + gd[1].astype(np.int64)
    tkey = gd[1].astype(np.int64) * n + rows
    order = np.argsort(key)
    pos = np.searchsorted(key[order], tkey)
    assert np.allclose(ns, ns[order][pos], rtol=1e-14)
    assert math.isclose(ns.sum(), 1.0, rel_tol=1e-12)
    # quantised weights: floor of an FP32 rounding of (p_j|i + p_i|j) * 2^30
    exact = (cond + g64[dist - 1] / Zrow[gd[1].astype(np.int64)]) * 2.0 ** 30
    q = sim["q"].astype(np.float64)
    assert np.all(q <= exact * (1 + 4e-7) + 1e-9)
    assert np.all(q >= exact * (1 - 4e-7) - 1.0)
    assert np.array_equal(sim["r"], np.bincount(rows, weights=sim["q"], minlength=n).astype(np.uint64))


def test_similarity_k1_is_inverse_degree(orc):
    n, rp, col, gd, sim = _sim_for(orc, gg.random_binary_tree(200, 3), 1)
    deg = np.diff(rp).astype(np.float64)
    rows = np.repeat(np.arange(n), np.diff(rp).astype(np.int64))
    j = col.astype(np.int64)
    assert np.allclose(sim["ns"], (1 / deg[rows] + 1 / deg[j]) / (2 * n), rtol=1e-14)



# ------------------------------------------- perplexity-calibrated sigma_i
def test_own_exp_against_the_c_library(orc):
    xs = np.r_[np.linspace(-700.0, 30.0, 40001), [-1e-300, -0.5, 0.5, -np.log(2), 1e-9, -1e-9]]
    got = np.array([orc.exp(x) for x in xs])
    ref = np.exp(xs)
    assert np.max(np.abs(got - ref) / ref) <= 4.5e-16
    assert orc.exp(0.0) == 1.0 and orc.exp(-700.5) == 0.0


def _perplexity_np(counts, beta):
    # exp of the entropy of the row distribution, evaluated with numpy
    d = np.arange(1, len(counts) + 1, dtype=np.float64)
    w = np.repeat(np.exp(-beta * (d * d - 1)), np.asarray(counts, np.int64))
    p = w / w.sum()
    p = p[p > 0]
    return math.exp(-(p * np.log(p)).sum())


@pytest.mark.parametrize("counts,P", [([8, 300], 30.0), ([3, 40, 900], 30.0), ([1, 2, 4, 8, 16], 5.0),
                                      ([25, 10], 30.0), ([5, 5], 9.99), ([40], 7.0), ([2, 4000], 2.5),
                                      ([50, 100], 30.0), ([3, 4], 30.0)])
def test_calibrated_row_perplexity(orc, counts, P):
    beta = orc.calibrate_row(counts, P)
    N, c1 = sum(counts), counts[0]
    if P >= N:                                    # not reachable: uniform row
        assert beta < 1e-12
    elif P <= c1 and len(counts) > 1:             # all weight on the nearest class
        assert beta > 511
    elif len(counts) > 1:
        assert math.isclose(_perplexity_np(counts, beta), P, rel_tol=1e-9)
        # the root of the closed-form entropy, found by scipy
        from scipy.optimize import brentq
        root = brentq(lambda b: math.log(_perplexity_np(counts, b)) - math.log(P), 0.0, 512.0, xtol=1e-14)
        assert math.isclose(beta, root, rel_tol=1e-9, abs_tol=1e-12)
    assert math.isclose(orc.row_perplexity(counts, beta), _perplexity_np(counts, beta), rel_tol=1e-12)


@pytest.mark.parametrize("k,P", [(2, 30.0), (3, 12.0), (1, 5.0)])
def test_similarity_perplexity_rows(orc, k, P):
    n, s, d = gg.barabasi_albert(400, 2, 9)
    rp, col = orc.canonical_graph(n, s, d)
    gd = orc.korder(rp, col, k)
    sim = orc.similarity_perplexity(*gd, k, P)
    rows = np.repeat(np.arange(n), np.diff(gd[0]).astype(np.int64))
    dist = gd[2].astype(np.int64)
    beta = sim["beta"]
    # NS_{j|i} with the calibrated sigma_i sums to one and has perplexity P
    # (or the row's limit) in every row
    w = np.exp(-beta[rows] * (dist * dist - 1))
    Zrow = np.zeros(n)
    np.add.at(Zrow, rows, w)
    cond = w / Zrow[rows]
    H = np.zeros(n)
    np.add.at(H, rows, -cond * np.log(np.where(cond > 0, cond, 1.0)))
    size = np.diff(gd[0]).astype(np.int64)
    c1 = np.bincount(rows[dist == 1], minlength=n)
    mid = (size > P) & (c1 < P)
    assert np.allclose(np.exp(H[mid]), P, rtol=1e-8)
    assert np.allclose(np.exp(H[size <= P]), size[size <= P], rtol=1e-8)
    # FP32 normaliser and quantised weights from the per-node Gaussians
    g32 = np.exp(-beta[rows] * (dist * dist - 1)).astype(np.float32)
    assert np.allclose(sim["Z"][rows], Zrow[rows], rtol=1e-6)
    ns = sim["ns"]
    key = rows * n + gd[1].astype(np.int64)
    tkey = gd[1].astype(np.int64) * n + rows
    order = np.argsort(key)
    assert np.allclose(ns, ns[order][np.searchsorted(key[order], tkey)], rtol=1e-14)
    assert math.isclose(ns.sum(), 1.0, rel_tol=1e-12)
    exact = ns * 2 * n * 2.0 ** 30
    q = sim["q"].astype(np.float64)
    assert np.all(q <= exact * (1 + 4e-7) + 1e-9) and np.all(q >= exact * (1 - 4e-7) - 1.0)
    assert np.array_equal(sim["r"], np.bincount(rows, weights=sim["q"], minlength=n).astype(np.uint64))
    if k == 1:   # one class: the calibration cannot matter, NS_{j|i} = 1/deg
        deg = np.diff(rp).astype(np.float64)
        assert np.allclose(ns, (1 / deg[rows] + 1 / deg[col.astype(np.int64)]) / (2 * n), rtol=1e-14)


# ------------------------------------------------- per-row neighbour cap
@pytest.mark.parametrize("k", [2, 3])
def test_capped_matrix_without_binding_cap_is_the_matrix(orc, k):
    n, s, d = gg.barabasi_albert(300, 2, 7)
    rp, col = orc.canonical_graph(n, s, d)
    gd = orc.korder(rp, col, k)
    sim = orc.similarity(*gd, k, 1.0)
    u = orc.korder_capped(rp, col, k, 10 ** 6)
    assert all(np.array_equal(a, b) for a, b in zip(u[:3], gd)) and u[3].all() and u[4].all()
    sc = orc.similarity_capped(*u, k, 1.0)
    assert np.array_equal(sc["Z"].view(np.uint32), sim["Z"].view(np.uint32))
    assert np.array_equal(sc["q"], sim["q"]) and np.array_equal(sc["r"], sim["r"])


def test_tie_order_is_a_scrambling_bijection(orc):
    # distinct on 2^22 consecutive ids and inside [0, 2^28); unrelated to the
    # id's size (rank correlation near 0; no fixed point at the smallest ids)
    v = np.arange(1 << 22, dtype=np.int64)
    t = orc.tie_order(v)
    assert len(np.unique(t)) == len(v) and t.min() >= 0 and t.max() < (1 << 28)
    assert abs(np.corrcoef(v, t)[0, 1]) < 0.01
    assert np.argmin(t[:64]) != 0
    top = (1 << 28) - (1 << 20) + np.arange(1 << 20, dtype=np.int64)
    assert len(np.unique(np.r_[t[:1 << 20], orc.tie_order(top)])) == 2 << 20


def test_capped_star_by_hand(orc):
    # K_{1,5}, k = 2, cap 2.  The tie order ranks the leaves 5, 4, 2, 1, 3:
    # the hub keeps leaves 5 and 4; every leaf keeps the hub and the first
    # other leaf in that order (5, or 4 for leaf 5)
    assert np.argsort(orc.tie_order(np.arange(1, 6))).tolist() == [4, 3, 1, 0, 2]
    rp, col = orc.canonical_graph(6, np.zeros(5, np.int64), np.arange(1, 6))
    u_rp, u_col, u_dist, own, back = orc.korder_capped(rp, col, 2, 2)
    rows = {i: u_col[int(u_rp[i]):int(u_rp[i + 1])].tolist() for i in range(6)}
    assert rows == {0: [1, 2, 3, 4, 5], 1: [0, 5], 2: [0, 5], 3: [0, 5], 4: [0, 5], 5: [0, 1, 2, 3, 4]}
    flags = {i: list(zip(own[int(u_rp[i]):int(u_rp[i + 1])].tolist(), back[int(u_rp[i]):int(u_rp[i + 1])].tolist()))
             for i in range(6)}
    assert flags[0] == [(False, True), (False, True), (False, True), (True, True), (True, True)]
    assert flags[5] == [(True, True), (False, True), (False, True), (False, True), (True, True)]
    assert flags[4] == [(True, True), (True, True)]
    assert flags[3] == [(True, False), (True, False)]
    sc = orc.similarity_capped(u_rp, u_col, u_dist, own, back, 2, 1.0)
    g1, g2 = np.float32(np.exp(-0.5)), np.float32(np.exp(-2.0))
    assert sc["Z"][0] == np.float32(np.float32(2) * g1) and sc["Z"][3] == np.float32(g1 + g2)
    # (0, 3): only the leaf's side keeps the pair
    e03 = int(u_rp[0]) + 2
    assert sc["q"][e03] == np.uint32(np.float32(np.float32(g1 / sc["Z"][3]) * np.float32(2.0 ** 30)))


@pytest.mark.parametrize("seed,k,cap", [(0, 2, 5), (1, 3, 12), (2, 2, 1)])
def test_capped_sets_against_all_pairs_shortest_paths(orc, seed, k, cap):
    n, s, d = gg.erdos_renyi(120, 200, seed)
    rp, col = orc.canonical_graph(n, s, d)
    A = sp.csr_matrix((np.ones(len(col)), col.astype(np.int64), rp.astype(np.int64)), shape=(n, n))
    D = csg.shortest_path(A, unweighted=True)
    kept = set()
    for i in range(n):
        cand = [(D[i, j], j) for j in range(n) if j != i and D[i, j] <= k]
        kept |= {(i, j) for _, _, j in sorted((dd, int(orc.tie_order(j)), j) for dd, j in cand)[:cap]}
    want = kept | {(j, i) for i, j in kept}
    u_rp, u_col, u_dist, own, back = orc.korder_capped(rp, col, k, cap)
    rows = np.repeat(np.arange(n), np.diff(u_rp).astype(np.int64))
    got = list(zip(rows.tolist(), u_col.tolist()))
    assert set(got) == want and len(got) == len(want)
    assert [p in kept for p in got] == own.tolist()
    assert [(j, i) in kept for i, j in got] == back.tolist()
    assert np.array_equal(u_dist, D[rows, u_col.astype(np.int64)].astype(np.uint8))
    sc = orc.similarity_capped(u_rp, u_col, u_dist, own, back, k, 1.0)
    key = rows * n + u_col.astype(np.int64)
    tkey = u_col.astype(np.int64) * n + rows
    order = np.argsort(key)
    assert np.array_equal(sc["q"], sc["q"][order][np.searchsorted(key[order], tkey)])   # symmetric
    assert math.isclose(sc["ns"].sum(), 1.0 - np.mean(np.diff(rp) == 0), rel_tol=1e-12)

def test_node_weight_shift(orc):
    r = np.array([0, 5, 2 ** 40 + 7, 2 ** 33], np.uint64)
    r32, s = orc.node_weights_u32(r)
    assert s == 9
    assert r32.tolist() == [0, 0, (2 ** 40 + 7) >> 9, 2 ** 24]
    r32, s = orc.node_weights_u32(np.array([3, 4], np.uint64))
    assert s == 0 and r32.tolist() == [3, 4]


# ---------------------------------------------------------------- alias tables
def _mass_per_item(q, th, al, own):
    N = len(q)
    W = int(np.sum(q.astype(object)))
    got = [0] * N
    for b in range(N):
        o = int(own[b])
        got[b] += o
        if int(al[b]) != b:
            got[int(al[b])] += W - o
        else:
            assert o == W
    return got, W


def _draw_prob(th, al):
    N = len(th)
    P = np.zeros(N)
    for b in range(N):
        keep = int(th[b]) / 2.0 ** 32
        P[b] += keep / N
        P[int(al[b])] += (1 - keep) / N
    return P


CASES = [
    np.array([1], np.uint32),
    np.array([3, 3, 3, 3], np.uint32),
    np.array([0, 0, 9, 0], np.uint32),
    np.array([1, 2, 3, 4, 5, 6, 7, 8], np.uint32),
    np.array([2 ** 31, 1, 1, 1, 2 ** 30, 0, 7], np.uint32),
]


@pytest.mark.parametrize("case", range(len(CASES)) )
def test_alias_exact_mass_and_probability(orc, case):
    q = CASES[case]
    th, al, own = orc.alias_build(q)
    got, W = _mass_per_item(q, th, al, own)
    N = len(q)
    assert got == [int(x) * N for x in q]
    P = _draw_prob(th, al)
    assert np.allclose(P, q.astype(np.float64) / W, atol=2.0 ** -31, rtol=0)


def test_alias_random_weights_and_sweep_closed_form(orc):
    rng = np.random.default_rng(11)
    for trial in range(20):
        N = int(rng.integers(1, 400))
        q = rng.integers(0, 2 ** int(rng.integers(1, 32)), size=N).astype(np.uint32)
        if q.sum() == 0:
            q[0] = 1
        th, al, own = orc.alias_build(q)
        got, W = _mass_per_item(q, th, al, own)
        assert got == [int(x) * N for x in q]
        # the sweep equals its merge-rank closed form (Huebschle-Schneider &
        # Sanders): light x goes to the first heavy whose cumulative excess
        # exceeds the lights' cumulative deficit before x.
        a = [int(x) * N for x in q]
        L = [i for i in range(N) if a[i] < W]
        H = [i for i in range(N) if a[i] >= W]
        Dl = [0]
        for i in L:
            Dl.append(Dl[-1] + W - a[i])
        S = []
        acc = 0
        for h in H:
            acc += a[h] - W
            S.append(acc)
        for x, i in enumerate(L):
            y = sum(1 for v in S if v <= Dl[x])
            assert int(al[i]) == H[y] and int(own[i]) == a[i]
        for y, h in enumerate(H):
            xs = sum(1 for v in Dl if v < S[y])
            mass = S[y] + W - Dl[xs]
            assert int(own[h]) == mass
            exp_alias = h if mass == W else H[y + 1]
            assert int(al[h]) == exp_alias
        for b in range(N):
            t = (int(own[b]) << 32) // W
            assert int(th[b]) == min(t, 2 ** 32 - 1)


def test_alias_zero_total_is_error(orc):
    assert orc.alias_build(np.zeros(5, np.uint32)) is None
    assert orc.alias_build(np.zeros(0, np.uint32)) is None


def test_alias_draw_chi_square(orc):
    q = np.array([5, 1, 0, 20, 3, 3, 11, 2, 9, 1], np.uint32)
    th, al, own = orc.alias_build(q)
    rng = np.random.default_rng(5)
    R = rng.integers(0, 2 ** 63, size=60000, dtype=np.uint64) * np.uint64(2) + rng.integers(0, 2, size=60000, dtype=np.uint64)
    U = rng.integers(0, 2 ** 32, size=60000, dtype=np.uint64)
    counts = np.zeros(len(q))
    for r, u in zip(R.tolist(), U.tolist()):
        counts[orc.alias_draw(th, al, r, u)] += 1
    expect = q / q.sum() * len(R)
    assert counts[2] == 0
    m = expect > 0
    chi2 = ((counts[m] - expect[m]) ** 2 / expect[m]).sum()
    assert chi2 < stats.chi2.ppf(0.999, m.sum() - 1)


# ---------------------------------------------------------------- spot-check helpers
@pytest.mark.parametrize("k", [1, 2, 3])
def test_row_helpers_match_full_matrix(orc, k):
    n, s, d = gg.barabasi_albert(700, 3, 4)
    rp, col = orc.canonical_graph(n, s, d)
    gd = orc.korder(rp, col, k)
    sim = orc.similarity(*gd, k, 1.0)
    rows = orc.RowBFS(rp, col, k)
    src = np.array([0, 5, 77, 699, 350], np.uint32)
    counts = orc.class_counts(rp, col, k, src)
    g = orc.gaussians(k)
    assert np.array_equal(g, sim["g"])
    for x, i in enumerate(src.tolist()):
        c, dd = rows.row(i)
        assert np.array_equal(c, gd[1][gd[0][i]:gd[0][i + 1]]) and np.array_equal(dd, gd[2][gd[0][i]:gd[0][i + 1]])
        assert counts[x].tolist() == [int((dd == t).sum()) for t in range(1, k + 1)]
        assert np.float32(orc.normaliser(counts[x], g)) == sim["Z"][i]
    e = int(gd[0][5])
    j = int(gd[1][e])
    zj = orc.normaliser(orc.class_counts(rp, col, k, [j])[0], g)
    assert orc.entry_weight(g[gd[2][e] - 1], sim["Z"][5], zj) == sim["q"][e]
