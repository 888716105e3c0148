// Graphs on the device: the canonical CSR of Sec. 3.1 and the multilevel
// hierarchy of Sec. 3.2.3 (coarsening by heavy-edge matching or by the
// paper's star grouping, contraction and ancestor maps).
#include "prims.cuh"

namespace drg {

// ------------------------------------------------------------------ canonical CSR
// Key of a directed entry: row in the high bits, column in the low `cb` bits.
// Self-loops get the all-ones key, which sorts after every real entry.
__global__ void k_edge_keys(const uint32_t* __restrict__ src, const uint32_t* __restrict__ dst, uint64_t m,
                            uint32_t n, int cb, uint64_t* __restrict__ keys, uint32_t* __restrict__ bad) {
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < m; e += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t s = src[e], d = dst[e];
        if (s >= n || d >= n) {
            *bad = 1u;
            keys[2 * e] = keys[2 * e + 1] = ~0ull;
            continue;
        }
        if (s == d) {
            keys[2 * e] = keys[2 * e + 1] = ~0ull;
        } else {
            keys[2 * e] = ((uint64_t)s << cb) | d;
            keys[2 * e + 1] = ((uint64_t)d << cb) | s;
        }
    }
}

struct HeadFlag {
    const uint64_t* keys;
    __device__ __forceinline__ uint32_t operator()(size_t i) const {
        const uint64_t k = keys[i];
        return (k != ~0ull && (i == 0 || keys[i - 1] != k)) ? 1u : 0u;
    }
};

// Writes col (and summed weights) of every unique key, and the row pointer.
__global__ void k_csr_fill(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ vals,
                           const uint32_t* __restrict__ pos, size_t count, uint32_t n, int cb, uint64_t nnz,
                           uint64_t* __restrict__ rp, uint32_t* __restrict__ col, uint32_t* __restrict__ w) {
    const uint64_t cmask = (cb >= 64) ? ~0ull : ((1ull << cb) - 1);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
        const uint64_t k = keys[i];
        if (k == ~0ull) continue;
        const bool head = (i == 0 || keys[i - 1] != k);
        const uint32_t p = pos[i] + (head ? 0u : 0xFFFFFFFFu);  // index of this key's unique slot
        if (w) atomicAdd(&w[p], vals ? vals[i] : 1u);
        const int64_t r = (int64_t)(k >> cb);
        // the last valid key closes every remaining row
        if (i + 1 == count || keys[i + 1] == ~0ull)
            for (int64_t x = r + 1; x <= (int64_t)n; ++x) rp[x] = nnz;
        if (!head) continue;
        col[p] = (uint32_t)(k & cmask);
        const int64_t rprev = (i == 0) ? -1 : (int64_t)(keys[i - 1] >> cb);
        for (int64_t x = rprev + 1; x <= r; ++x) rp[x] = p;
    }
}

// keys: sorted directed-entry keys (row << cb | col), `count` of them, the
// invalid all-ones key last; vals: per-key weights or nullptr.  Duplicates
// are merged, summing weights when `weighted`.
static void csr_from_sorted(drg_ctx* ctx, uint32_t n, const uint64_t* keys, const uint32_t* vals, size_t count,
                            int cb, bool weighted, drg_graph* out) {
    DBuf<uint32_t> pos(ctx, count + 1);
    DBuf<uint64_t> tot(ctx, 1);
    // positions of unique keys (exclusive); the total is the entry count
    {
        DBuf<uint32_t> tot32(ctx, 1);
        scan<uint32_t>(ctx, HeadFlag{keys}, count, pos.p, false, tot32.p);
        out->nnz = read1(ctx, tot32.p);
    }
    out->n = n;
    out->rp = static_cast<uint64_t*>(dalloc(ctx, sizeof(uint64_t) * ((size_t)n + 1)));
    out->col = static_cast<uint32_t*>(dalloc(ctx, sizeof(uint32_t) * (out->nnz ? out->nnz : 1)));
    out->w = nullptr;
    if (weighted) {
        out->w = static_cast<uint32_t*>(dalloc(ctx, sizeof(uint32_t) * (out->nnz ? out->nnz : 1)));
        DRG_CUDA(cudaMemsetAsync(out->w, 0, sizeof(uint32_t) * (out->nnz ? out->nnz : 1), ctx->stream));
    }
    if (out->nnz == 0) {
        DRG_CUDA(cudaMemsetAsync(out->rp, 0, sizeof(uint64_t) * ((size_t)n + 1), ctx->stream));
        return;
    }
    DRG_LAUNCH(ctx, k_csr_fill, grid_for(count, 256, 65536), 256, 0, keys, vals, pos.p, count, n, cb, out->nnz,
               out->rp, out->col, out->w);
}

drg_graph* graph_from_edges(drg_ctx* ctx, uint32_t n, uint64_t m, const uint32_t* src, const uint32_t* dst,
                            bool on_device) {
    DRG_CHECK(n > 0 && n < 0xFFFFFFFFu, DRG_EINVAL, "n must be in [1, 2^32 - 2]");
    DRG_CHECK(m == 0 || (src && dst), DRG_EINVAL, "null edge arrays");
    DRG_CHECK(2 * m < (1ull << 32), DRG_EUNSUPPORTED, "at most 2^31 - 1 edges");
    const int cb = bitlen(n - 1) ? bitlen(n - 1) : 1;
    const int rb = cb;
    drg_graph* g = new drg_graph();
    g->ctx = ctx;
    try {
        ProfSpan span(ctx, DRG_PROF_GRAPH, m);
        DBuf<uint32_t> ds, dd;
        const uint32_t* s = src;
        const uint32_t* d = dst;
        if (!on_device && m) {
            ds = DBuf<uint32_t>(ctx, m);
            dd = DBuf<uint32_t>(ctx, m);
            h2d(ctx, ds.p, src, m);
            h2d(ctx, dd.p, dst, m);
            s = ds.p;
            d = dd.p;
        }
        const size_t count = 2 * m;
        DBuf<uint64_t> keys(ctx, count), alt(ctx, count);
        DBuf<uint32_t> bad(ctx, 1);
        DRG_CUDA(cudaMemsetAsync(bad.p, 0, 4, ctx->stream));
        DRG_LAUNCH(ctx, k_edge_keys, grid_for(m, 256, 65536), 256, 0, s, d, m, n, cb, keys.p, bad.p);
        DRG_CHECK(read1(ctx, bad.p) == 0, DRG_EINVAL, "edge endpoint >= n");
        uint64_t* kp = keys.p;
        uint64_t* ap = alt.p;
        uint32_t* vnull = nullptr;
        uint32_t* vnull2 = nullptr;
        radix_sort(ctx, kp, ap, vnull, vnull2, count, 0, rb + cb);
        csr_from_sorted(ctx, n, kp, nullptr, count, cb, false, g);
        sync(ctx);
    } catch (...) {
        graph_free(g);
        throw;
    }
    return g;
}

void graph_free(drg_graph* g) {
    if (!g) return;
    if (g->rp) dfree(g->ctx, g->rp);
    if (g->col) dfree(g->ctx, g->col);
    if (g->w) dfree(g->ctx, g->w);
    delete g;
}

// ------------------------------------------------------------------ heavy-edge matching
// One warp per node: every unmatched node proposes to its unmatched
// neighbour of largest (weight, Philox hash of (min id, max id, round),
// smaller id).
__global__ void k_hem_propose(const uint64_t* __restrict__ rp, const uint32_t* __restrict__ col,
                              const uint32_t* __restrict__ w, const uint32_t* __restrict__ match,
                              uint32_t* __restrict__ prop, uint32_t n, uint2 key, uint32_t tag, uint32_t round) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warp0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t vv = warp0; vv < n; vv += nwarps) {
        const uint32_t v = (uint32_t)vv;
        if (match[v] != kNone) {
            if (lane == 0) prop[v] = kNone;
            continue;
        }
        uint32_t bu = kNone, bw = 0, bh = 0;
        for (uint64_t e = rp[v] + lane; e < rp[v + 1]; e += 32) {
            const uint32_t u = col[e];
            if (u == v || match[u] != kNone) continue;
            const uint32_t lo = u < v ? u : v, hi = u < v ? v : u;
            const uint32_t h = philox(make_uint4(lo, hi, tag, round), key).x;
            const uint32_t we = w ? w[e] : 1u;
            bool better;
            if (bu == kNone) better = true;
            else if (we != bw) better = we > bw;
            else if (h != bh) better = h > bh;
            else better = u < bu;
            if (better) { bu = u; bw = we; bh = h; }
        }
#pragma unroll
        for (int off = 16; off; off >>= 1) {
            const uint32_t ou = __shfl_xor_sync(0xFFFFFFFFu, bu, off);
            const uint32_t ow = __shfl_xor_sync(0xFFFFFFFFu, bw, off);
            const uint32_t oh = __shfl_xor_sync(0xFFFFFFFFu, bh, off);
            bool better;
            if (ou == kNone) better = false;
            else if (bu == kNone) better = true;
            else if (ow != bw) better = ow > bw;
            else if (oh != bh) better = oh > bh;
            else better = ou < bu;
            if (better) { bu = ou; bw = ow; bh = oh; }
        }
        if (lane == 0) prop[v] = bu;
    }
}

__global__ void k_hem_accept(uint32_t* __restrict__ match, const uint32_t* __restrict__ prop, uint32_t n) {
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t u = prop[v];
        if (u != kNone && prop[u] == (uint32_t)v) match[v] = u;
    }
}

__global__ void k_hem_finish(uint32_t* __restrict__ match, uint32_t n) {
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x)
        if (match[v] == kNone) match[v] = (uint32_t)v;
}

struct RepFlag {
    const uint32_t* match;
    __device__ __forceinline__ uint32_t operator()(size_t v) const { return match[v] >= (uint32_t)v ? 1u : 0u; }
};

__global__ void k_cluster_ids(const uint32_t* __restrict__ match, const uint32_t* __restrict__ rank,
                              uint32_t* __restrict__ cid, uint32_t n) {
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t m = match[v];
        cid[v] = rank[m < (uint32_t)v ? m : (uint32_t)v];
    }
}

// Source row of every CSR entry (one warp per row).
__global__ void k_expand_rows(const uint64_t* __restrict__ rp, uint32_t n, uint32_t* __restrict__ src) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warp0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t v = warp0; v < n; v += nwarps)
        for (uint64_t e = rp[v] + lane; e < rp[v + 1]; e += 32) src[e] = (uint32_t)v;
}

__global__ void k_contract_keys(const uint32_t* __restrict__ esrc, const uint32_t* __restrict__ col,
                                const uint32_t* __restrict__ w, const uint32_t* __restrict__ cid, uint64_t nnz,
                                int cb, uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < nnz; e += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t a = cid[esrc[e]], b = cid[col[e]];
        keys[e] = (a == b) ? ~0ull : (((uint64_t)a << cb) | b);
        vals[e] = w ? w[e] : 1u;
    }
}

uint32_t hem_cluster(drg_ctx* ctx, const drg_graph* g, uint32_t level, const drg_params& p, uint32_t* cid) {
    const uint32_t n = g->n;
    DBuf<uint32_t> match(ctx, n), prop(ctx, n), rank(ctx, n);
    DRG_CUDA(cudaMemsetAsync(match.p, 0xFF, sizeof(uint32_t) * n, ctx->stream));
    const uint2 key = seed_key(p.seed);
    const uint32_t tag = stream_tag(kPurposeMatch, p.gid, level);
    const uint32_t gw = grid_for((size_t)n * 32, 256, (uint32_t)ctx->num_sms * 16);
    const uint32_t gt = grid_for(n, 256, (uint32_t)ctx->num_sms * 32);
    for (uint32_t r = 0; r < p.match_rounds; ++r) {
        DRG_LAUNCH(ctx, k_hem_propose, gw, 256, 0, g->rp, g->col, g->w, match.p, prop.p, n, key, tag, r);
        DRG_LAUNCH(ctx, k_hem_accept, gt, 256, 0, match.p, prop.p, n);
    }
    DRG_LAUNCH(ctx, k_hem_finish, gt, 256, 0, match.p, n);
    DBuf<uint32_t> nc(ctx, 1);
    scan<uint32_t>(ctx, RepFlag{match.p}, n, rank.p, false, nc.p);
    DRG_LAUNCH(ctx, k_cluster_ids, gt, 256, 0, match.p, rank.p, cid, n);
    return read1(ctx, nc.p);
}

// ------------------------------------------------------------------ star grouping
// Sec. 3.2.3 as the paper states it: walk a random order of the nodes; a node
// not yet grouped when reached becomes a centre and takes its ungrouped
// neighbours.  The centres are the first maximal independent set of the
// order (v is a centre iff none of its earlier neighbours is), and every other
// node joins its earliest centre neighbour.  Rounds decide each open node
// whose earlier neighbours are all decided; a decided state never changes,
// so a stale read only delays a decision, and the earliest open node always
// decides, so at most n rounds run (a handful on random orders).
constexpr uint8_t kStarOpen = 0, kStarCentre = 1, kStarCovered = 2;

__device__ __forceinline__ uint64_t star_key(const uint32_t* prio, uint32_t v) {
    return ((uint64_t)prio[v] << 32) | v;
}

__global__ void k_star_prio(uint32_t* __restrict__ prio, uint32_t n, uint2 key, uint32_t tag) {
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x)
        prio[v] = philox(make_uint4((uint32_t)v, 0u, tag, 0u), key).x;
}

// One warp per open node; `open` counts the nodes still open after the round.
__global__ void k_star_round(const uint64_t* __restrict__ rp, const uint32_t* __restrict__ col,
                             const uint32_t* __restrict__ prio, uint8_t* state, uint32_t n,
                             uint32_t* __restrict__ open) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warp0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const volatile uint8_t* vstate = state;
    for (uint64_t vv = warp0; vv < n; vv += nwarps) {
        const uint32_t v = (uint32_t)vv;
        if (state[v] != kStarOpen) continue;
        const uint64_t kv = star_key(prio, v);
        bool centre = false, pending = false;
        for (uint64_t e = rp[v] + lane; e < rp[v + 1]; e += 32) {
            const uint32_t u = col[e];
            if (star_key(prio, u) >= kv) continue;
            const uint8_t s = vstate[u];
            centre |= s == kStarCentre;
            pending |= s == kStarOpen;
        }
        const bool any_centre = __any_sync(0xFFFFFFFFu, centre);
        const bool any_pending = __any_sync(0xFFFFFFFFu, pending);
        if (lane == 0) {
            if (any_centre) state[v] = kStarCovered;
            else if (!any_pending) state[v] = kStarCentre;
            else atomicAdd(open, 1u);
        }
    }
}

// centre[v]: v for a centre, else the neighbour centre earliest in the order.
// A covered node always has a centre neighbour; `bad` records one without
// (v keeps itself, so every later index stays in range).
__global__ void k_star_assign(const uint64_t* __restrict__ rp, const uint32_t* __restrict__ col,
                              const uint32_t* __restrict__ prio, const uint8_t* __restrict__ state,
                              uint32_t* __restrict__ centre, uint32_t n, uint32_t* __restrict__ bad) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warp0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t vv = warp0; vv < n; vv += nwarps) {
        const uint32_t v = (uint32_t)vv;
        if (state[v] == kStarCentre) {
            if (lane == 0) centre[v] = v;
            continue;
        }
        uint64_t best = ~0ull;
        for (uint64_t e = rp[v] + lane; e < rp[v + 1]; e += 32) {
            const uint32_t u = col[e];
            if (state[u] != kStarCentre) continue;
            const uint64_t ku = star_key(prio, u);
            best = ku < best ? ku : best;
        }
#pragma unroll
        for (int off = 16; off; off >>= 1) {
            const uint64_t o = __shfl_xor_sync(0xFFFFFFFFu, best, off);
            best = o < best ? o : best;
        }
        if (lane == 0) {
            if (best == ~0ull || state[v] != kStarCovered) {
                *bad = 1u;
                centre[v] = v;
            } else {
                centre[v] = (uint32_t)best;
            }
        }
    }
}

struct CentreFlag {
    const uint8_t* state;
    __device__ __forceinline__ uint32_t operator()(size_t v) const { return state[v] == kStarCentre ? 1u : 0u; }
};

__global__ void k_star_ids(const uint32_t* __restrict__ centre, const uint32_t* __restrict__ rank,
                           uint32_t* __restrict__ cid, uint32_t n) {
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x)
        cid[v] = rank[centre[v]];
}

uint32_t star_cluster(drg_ctx* ctx, const drg_graph* g, uint32_t level, const drg_params& p, uint32_t* cid) {
    const uint32_t n = g->n;
    DBuf<uint32_t> prio(ctx, n), centre(ctx, n), rank(ctx, n), open(ctx, 1), nc(ctx, 1), bad(ctx, 1);
    DBuf<uint8_t> state(ctx, n);
    DRG_CUDA(cudaMemsetAsync(state.p, kStarOpen, n, ctx->stream));
    const uint2 key = seed_key(p.seed);
    const uint32_t gw = grid_for((size_t)n * 32, 256, (uint32_t)ctx->num_sms * 16);
    const uint32_t gt = grid_for(n, 256, (uint32_t)ctx->num_sms * 32);
    DRG_LAUNCH(ctx, k_star_prio, gt, 256, 0, prio.p, n, key, stream_tag(kPurposeStar, p.gid, level));
    for (uint64_t round = 0;; ++round) {
        DRG_CHECK(round <= n, DRG_ECUDA, "star grouping made no progress");
        DRG_CUDA(cudaMemsetAsync(open.p, 0, sizeof(uint32_t), ctx->stream));
        DRG_LAUNCH(ctx, k_star_round, gw, 256, 0, g->rp, g->col, prio.p, state.p, n, open.p);
        if (n == 0 || read1(ctx, open.p) == 0) break;
    }
    DRG_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(uint32_t), ctx->stream));
    DRG_LAUNCH(ctx, k_star_assign, gw, 256, 0, g->rp, g->col, prio.p, state.p, centre.p, n, bad.p);
    DRG_CHECK(read1(ctx, bad.p) == 0, DRG_ECUDA, "star grouping left a node without a centre");
    scan<uint32_t>(ctx, CentreFlag{state.p}, n, rank.p, false, nc.p);
    DRG_LAUNCH(ctx, k_star_ids, gt, 256, 0, centre.p, rank.p, cid, n);
    return read1(ctx, nc.p);
}

drg_graph* contract(drg_ctx* ctx, const drg_graph* g, const uint32_t* cid, uint32_t nc) {
    drg_graph* c = new drg_graph();
    c->ctx = ctx;
    try {
        const uint64_t nnz = g->nnz;
        DBuf<uint32_t> esrc(ctx, nnz);
        DRG_LAUNCH(ctx, k_expand_rows, grid_for((size_t)g->n * 32, 256, (uint32_t)ctx->num_sms * 16), 256, 0, g->rp,
                   g->n, esrc.p);
        const int cb = bitlen(nc > 1 ? nc - 1 : 1);
        DBuf<uint64_t> keys(ctx, nnz), kalt(ctx, nnz);
        DBuf<uint32_t> vals(ctx, nnz), valt(ctx, nnz);
        DRG_LAUNCH(ctx, k_contract_keys, grid_for(nnz, 256, 65536), 256, 0, esrc.p, g->col, g->w, cid, nnz, cb,
                   keys.p, vals.p);
        uint64_t* kp = keys.p;
        uint64_t* ap = kalt.p;
        uint32_t* vp = vals.p;
        uint32_t* vq = valt.p;
        radix_sort(ctx, kp, ap, vp, vq, nnz, 0, 2 * cb);
        csr_from_sorted(ctx, nc, kp, vp, nnz, cb, true, c);
    } catch (...) {
        graph_free(c);
        throw;
    }
    return c;
}

// Sec. 3.2.3 coarsening step (heavy-edge matching or the paper's star
// grouping, as p.coarsen selects).  With rho > 0 a candidate keeping more than rho
// of the nodes is rejected (nullptr returned, parent left written).
static drg_graph* coarsen_impl(drg_ctx* ctx, const drg_graph* fine, uint32_t level, const drg_params& p,
                               uint32_t* parent, double rho) {
    const uint32_t nc = p.coarsen == DRG_COARSEN_STAR ? star_cluster(ctx, fine, level, p, parent)
                                                      : hem_cluster(ctx, fine, level, p, parent);
    if (rho > 0.0 && (double)nc > rho * (double)fine->n) return nullptr;
    return contract(ctx, fine, parent, nc);
}

drg_graph* coarsen(drg_ctx* ctx, const drg_graph* fine, uint32_t level, const drg_params& p, uint32_t* parent) {
    drg_graph* c = coarsen_impl(ctx, fine, level, p, parent, 0.0);
    sync(ctx);
    return c;
}

__global__ void k_compose(const uint32_t* __restrict__ parent, const uint32_t* __restrict__ anc_prev,
                          uint32_t* __restrict__ anc, uint32_t n0) {
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n0; v += (uint64_t)gridDim.x * blockDim.x)
        anc[v] = parent[anc_prev ? anc_prev[v] : (uint32_t)v];
}

drg_hier* build_hierarchy(drg_ctx* ctx, const drg_graph* g0, const drg_params& p) {
    drg_hier* h = new drg_hier();
    h->ctx = ctx;
    try {
        ProfSpan span(ctx, DRG_PROF_HIER, 0);
        h->g.push_back(g0);
        h->anc.push_back(nullptr);
        while (p.multilevel && h->g.size() < p.max_levels && h->g.back()->n >= p.stop_nodes) {
            const drg_graph* cur = h->g.back();
            const uint32_t lvl = (uint32_t)h->g.size() - 1;
            DBuf<uint32_t> parent(ctx, cur->n);
            drg_graph* c = coarsen_impl(ctx, cur, lvl, p, parent.p, (double)p.rho);
            if (!c) break;
            h->owned.push_back(c);
            h->g.push_back(c);
            DBuf<uint32_t> anc(ctx, g0->n);
            DRG_LAUNCH(ctx, k_compose, grid_for(g0->n, 256, (uint32_t)ctx->num_sms * 32), 256, 0, parent.p,
                       h->anc.back(), anc.p, g0->n);
            h->parent.push_back(parent.release());
            h->anc.push_back(anc.release());
        }
        span.units = h->g.size();
        sync(ctx);
    } catch (...) {
        hier_free(h);
        throw;
    }
    return h;
}

void hier_free(drg_hier* h) {
    if (!h) return;
    for (auto* g : h->owned) graph_free(g);
    for (auto* p : h->parent) dfree(h->ctx, p);
    for (auto* a : h->anc)
        if (a) dfree(h->ctx, a);
    delete h;
}

}  // namespace drg
