// Sparse k-order distance matrix (Sec. 3.2.1, Eq. 8), node similarity
// (Eqs. 4, 9) and the alias tables the layout epochs draw from (Sec. 3.2.2).
#include "prims.cuh"

#include <cmath>

namespace drg {

__global__ void k_expand_rows(const uint64_t* __restrict__ rp, uint32_t n, uint32_t* __restrict__ src);

// ------------------------------------------------------------------ frontier BFS
// One block per source at a time (rows handed out by an atomic counter).  The
// block keeps a visited bitmap over all nodes (shared memory when it fits,
// else a private global slice), a summary bitmap with one bit per non-empty
// bitmap word, and the list of nodes it discovered, level after level.
// Frontier expansion is load balanced over the block: frontier nodes are
// taken BFS_THREADS at a time, their degrees prefix-summed, and every thread
// walks an equal share of the concatenated adjacency lists.  The row is then
// written sorted by node id straight from the bitmaps (the summary yields the
// touched words in increasing order; a prefix sum of their popcounts gives
// each word's output offset) -- no global sort.  Hop distances: for k = 2 a
// node is at distance 1 exactly when it is in the source's adjacency, whose
// nodes are located in the emitted row by binary search; for k > 2 the
// block records each discovered node's level.
// Staged mode writes each row into a staging area at an offset reserved with
// an atomic cursor (one traversal gives the counts and the rows); direct mode
// writes at the final row offsets and is the fallback when the staging area
// overflows.
constexpr int BFS_THREADS = 512;

struct BfsArgs {
    const uint64_t* rp;
    const uint32_t* col;
    uint32_t n, k;
    uint32_t words;           // bitmap words per block
    uint32_t swords;          // summary words per block
    uint32_t* gbitmaps;       // nullptr: bitmap in shared memory
    uint32_t* lists;          // [gridDim.x * n] discovered nodes
    uint32_t* wlists;         // [gridDim.x * words] touched words
    uint8_t* dlev;            // [gridDim.x * n] hop distance of discovered nodes (k > 2)
    uint32_t* next_row;       // work counter
    uint64_t* counts;         // row sizes (written in both modes)
    int staged;               // 1: write at a reserved staging offset
    unsigned long long* cursor;  // staged: next free staging entry
    uint64_t cap;             // staged: staging capacity
    uint64_t* row_off;        // staged: staging offset of each row
    uint32_t* overflow;       // staged: set when a row did not fit
    const uint64_t* gd_rp;    // direct: row offsets
    uint32_t* out_col;        // staging or final column array
    uint8_t* out_dist;        // staging or final distance array
};

__device__ __forceinline__ void bfs_append(uint32_t v, bool isnew, uint32_t* list, uint32_t* s_len) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t ballot = __ballot_sync(0xFFFFFFFFu, isnew);
    if (!ballot) return;
    uint32_t base = 0;
    if (lane == (uint32_t)(__ffs(ballot) - 1)) base = atomicAdd(s_len, (uint32_t)__popc(ballot));
    base = __shfl_sync(0xFFFFFFFFu, base, __ffs(ballot) - 1);
    if (isnew) list[base + __popc(ballot & lanemask_lt())] = v;
}

// Marks v visited; true for the one thread that marked it first.  The first
// bit set in a word also marks the word in the summary.
__device__ __forceinline__ bool visit(uint32_t* bm, uint32_t* summ, uint32_t v) {
    const uint32_t w = v >> 5, bit = 1u << (v & 31);
    if (*(volatile uint32_t*)&bm[w] & bit) return false;
    const uint32_t old = atomicOr(&bm[w], bit);
    if (old & bit) return false;
    if (old == 0) atomicOr(&summ[w >> 5], 1u << (w & 31));
    return true;
}

template <bool K2>
__global__ void __launch_bounds__(BFS_THREADS) k_bfs(BfsArgs a) {
    extern __shared__ uint32_t dsm[];
    __shared__ uint64_t s_off[BFS_THREADS];
    __shared__ uint64_t s_start[BFS_THREADS];
    __shared__ uint64_t s_wt[BFS_THREADS / 32];
    __shared__ uint32_t s_row, s_len;
    __shared__ uint64_t s_base;
    __shared__ int s_skip;
    uint32_t* bm = a.gbitmaps ? a.gbitmaps + (size_t)blockIdx.x * a.words : dsm;
    uint32_t* summ = a.gbitmaps ? dsm : dsm + a.words;
    uint32_t* list = a.lists + (size_t)blockIdx.x * a.n;
    uint32_t* wl = a.wlists + (size_t)blockIdx.x * a.words;
    uint8_t* dl = K2 ? nullptr : a.dlev + (size_t)blockIdx.x * a.n;
    for (uint32_t w = threadIdx.x; w < a.words; w += BFS_THREADS) bm[w] = 0;
    for (uint32_t w = threadIdx.x; w < a.swords; w += BFS_THREADS) summ[w] = 0;
    __syncthreads();
    for (;;) {
        if (threadIdx.x == 0) {
            s_row = atomicAdd(a.next_row, 1u);
            s_len = 0;
        }
        __syncthreads();
        const uint32_t row = s_row;
        if (row >= a.n) break;
        if (threadIdx.x == 0) visit(bm, summ, row);
        __syncthreads();
        const uint64_t ab = a.rp[row], ae = a.rp[row + 1];
        // level 1: the source's own adjacency
        for (uint64_t x0 = ab; x0 < ae; x0 += BFS_THREADS) {
            const uint64_t x = x0 + threadIdx.x;
            uint32_t v = 0;
            bool isnew = false;
            if (x < ae) {
                v = a.col[x];
                isnew = visit(bm, summ, v);
                if (!K2 && isnew) dl[v] = 1;
            }
            bfs_append(v, isnew, list, &s_len);
        }
        __syncthreads();
        uint32_t lo = 0, hi = s_len;
        __syncthreads();
        for (uint32_t d = 2; d <= a.k && lo < hi; ++d) {
            for (uint32_t c = lo; c < hi; c += BFS_THREADS) {
                const uint32_t idx = c + threadIdx.x;
                uint64_t deg = 0, start = 0;
                if (idx < hi) {
                    const uint32_t u = list[idx];
                    start = a.rp[u];
                    deg = a.rp[u + 1] - start;
                }
                uint64_t tot;
                const uint64_t ex = block_exclusive_scan<uint64_t, BFS_THREADS>(deg, s_wt, tot);
                s_off[threadIdx.x] = ex;
                s_start[threadIdx.x] = start;
                __syncthreads();
                const uint32_t cnt = (hi - c) < (uint32_t)BFS_THREADS ? (hi - c) : (uint32_t)BFS_THREADS;
                for (uint64_t x0 = 0; x0 < tot; x0 += BFS_THREADS) {
                    const uint64_t x = x0 + threadIdx.x;
                    uint32_t v = 0;
                    bool isnew = false;
                    if (x < tot) {
                        // owner: last frontier slot whose offset is <= x
                        uint32_t lo2 = 0, hi2 = cnt;
                        while (hi2 - lo2 > 1) {
                            const uint32_t mid = (lo2 + hi2) >> 1;
                            if (s_off[mid] <= x) lo2 = mid; else hi2 = mid;
                        }
                        v = a.col[s_start[lo2] + (x - s_off[lo2])];
                        isnew = visit(bm, summ, v);
                        if (!K2 && isnew) dl[v] = (uint8_t)d;
                    }
                    bfs_append(v, isnew, list, &s_len);
                }
                __syncthreads();
            }
            lo = hi;
            hi = s_len;
            __syncthreads();
        }
        const uint32_t total = s_len;
        if (threadIdx.x == 0) {
            bm[row >> 5] &= ~(1u << (row & 31));  // the source is not its own neighbour
            a.counts[row] = total;
            uint64_t base = 0;
            int skip = 0;
            if (a.staged) {
                base = atomicAdd(a.cursor, (unsigned long long)total);
                if (base + total > a.cap) {
                    skip = 1;
                    atomicExch(a.overflow, 1u);
                }
                a.row_off[row] = base;
            } else {
                base = a.gd_rp[row];
            }
            s_base = base;
            s_skip = skip;
        }
        __syncthreads();
        // touched words in increasing order (summary words split in equal ranges)
        const uint32_t per = (a.swords + BFS_THREADS - 1) / BFS_THREADS;
        const uint32_t s0 = threadIdx.x * per;
        const uint32_t s1 = s0 + per < a.swords ? s0 + per : a.swords;
        uint64_t mine = 0;
        for (uint32_t s = s0; s < s1; ++s) mine += __popc(summ[s]);
        uint64_t nw;
        uint64_t pos = block_exclusive_scan<uint64_t, BFS_THREADS>(mine, s_wt, nw);
        for (uint32_t s = s0; s < s1; ++s) {
            uint32_t m = summ[s];
            summ[s] = 0;
            while (m) {
                const uint32_t b = __ffs(m) - 1;
                m &= m - 1;
                wl[pos++] = 32 * s + b;
            }
        }
        __syncthreads();
        const bool emit = !s_skip;
        // every touched word's bits, in order
        uint64_t out = s_base;
        for (uint64_t c = 0; c < nw; c += BFS_THREADS) {
            const uint64_t idx = c + threadIdx.x;
            uint32_t wi = 0, w = 0;
            if (idx < nw) {
                wi = wl[idx];
                w = bm[wi];
                bm[wi] = 0;
            }
            uint64_t tot;
            uint64_t o = out + block_exclusive_scan<uint64_t, BFS_THREADS>((uint64_t)__popc(w), s_wt, tot);
            if (emit) {
                while (w) {
                    const uint32_t b = __ffs(w) - 1;
                    w &= w - 1;
                    const uint32_t v = 32 * wi + b;
                    a.out_col[o] = v;
                    a.out_dist[o] = K2 ? (uint8_t)2 : dl[v];
                    ++o;
                }
            }
            out += tot;
        }
        if (K2 && emit) {
            __syncthreads();
            // distance 1: the source's adjacency, located in the emitted (sorted)
            // row by binary search
            const uint32_t* rowc = a.out_col + s_base;
            for (uint64_t x = ab + threadIdx.x; x < ae; x += BFS_THREADS) {
                const uint32_t v = a.col[x];
                uint32_t lo3 = 0, hi3 = total;
                while (lo3 < hi3) {
                    const uint32_t mid = (lo3 + hi3) >> 1;
                    if (rowc[mid] < v) lo3 = mid + 1; else hi3 = mid;
                }
                a.out_dist[s_base + lo3] = 1;
            }
        }
        __syncthreads();
    }
}

// Moves staged rows to their final place (one warp per row).
__global__ void k_unstage(const uint64_t* __restrict__ row_off, const uint64_t* __restrict__ rp, uint32_t n,
                          const uint32_t* __restrict__ scol, const uint8_t* __restrict__ sdist,
                          uint32_t* __restrict__ col, uint8_t* __restrict__ dist) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warp0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t r = warp0; r < n; r += nwarps) {
        const uint64_t src = row_off[r], dst = rp[r], cnt = rp[r + 1] - rp[r];
        for (uint64_t e = lane; e < cnt; e += 32) {
            col[dst + e] = scol[src + e];
            dist[dst + e] = sdist[src + e];
        }
    }
}

__global__ void k_fill_u8(uint8_t* p, uint64_t n, uint8_t v) {
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < n; e += (uint64_t)gridDim.x * blockDim.x)
        p[e] = v;
}

struct DegSq {
    const uint64_t* rp;
    __device__ __forceinline__ uint64_t operator()(size_t v) const {
        const uint64_t d = rp[v + 1] - rp[v];
        return d * d;
    }
};

static void build_korder(drg_ctx* ctx, const drg_graph* g, uint32_t k, drg_dmat* d) {
    const uint32_t n = g->n;
    d->rp = static_cast<uint64_t*>(dalloc(ctx, sizeof(uint64_t) * ((size_t)n + 1)));
    if (k == 1) {
        // NNG(v_i, 1) is the adjacency itself, already sorted by column
        d->nnz = g->nnz;
        d->col = static_cast<uint32_t*>(dalloc(ctx, sizeof(uint32_t) * (d->nnz ? d->nnz : 1)));
        d->dist = static_cast<uint8_t*>(dalloc(ctx, d->nnz ? d->nnz : 1));
        d2d(ctx, d->rp, g->rp, (size_t)n + 1);
        d2d(ctx, d->col, g->col, d->nnz);
        DRG_LAUNCH(ctx, k_fill_u8, grid_for(d->nnz, 256, 65536), 256, 0, d->dist, d->nnz, (uint8_t)1);
        return;
    }
    const bool k2 = k == 2;
    auto kern = k2 ? k_bfs<true> : k_bfs<false>;
    const uint32_t words = (n + 31) / 32;
    const uint32_t swords = (words + 31) / 32;
    const size_t bm_bytes = (size_t)words * 4, sm_bytes = (size_t)swords * 4;
    const bool smem_bm = bm_bytes + sm_bytes + 16384 <= (size_t)ctx->max_smem_optin;
    DRG_CHECK(sm_bytes + 16384 <= (size_t)ctx->max_smem_optin, DRG_EUNSUPPORTED, "graph too large for the BFS");
    const size_t dyn = (smem_bm ? bm_bytes : 0) + sm_bytes;
    DRG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
    int per_sm = 0;
    DRG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BFS_THREADS, dyn));
    if (per_sm < 1) per_sm = 1;
    uint32_t blocks = (uint32_t)ctx->num_sms * (uint32_t)per_sm;
    if (blocks > n) blocks = n;
    // per-block discovered lists, touched words, word offsets / hop distances
    // (and bitmaps when they live in global memory)
    DBuf<uint32_t> lists(ctx, (size_t)blocks * n);
    DBuf<uint32_t> wlists(ctx, (size_t)blocks * words);
    DBuf<uint8_t> dlev(ctx, k2 ? 1 : (size_t)blocks * n);
    DBuf<uint32_t> gbm(ctx, smem_bm ? 1 : (size_t)blocks * words);
    DBuf<uint32_t> counter(ctx, 1), overflow(ctx, 1);
    DBuf<uint64_t> counts(ctx, (size_t)n), row_off(ctx, (size_t)n);
    DBuf<unsigned long long> cursor(ctx, 1);
    // staging capacity: for k = 2 a row has at most deg(i) + sum over its
    // neighbours of (deg(u) - 1) entries, so the total is at most sum deg^2;
    // for k > 2 whatever a quarter of the free memory holds
    uint64_t cap;
    {
        DBuf<uint64_t> s2(ctx, 1);
        DBuf<uint64_t> tmp(ctx, n);
        scan<uint64_t>(ctx, DegSq{g->rp}, n, tmp.p, false, s2.p);
        cap = read1(ctx, s2.p);
    }
    if (!k2) cap *= 4;  // a guess: rows that overflow it are traversed again
    if (cap > 0xFFFFFFFFull) cap = 0xFFFFFFFFull;
    DBuf<uint32_t> scol;
    DBuf<uint8_t> sdist;
    try {
        scol = DBuf<uint32_t>(ctx, cap ? cap : 1);
        sdist = DBuf<uint8_t>(ctx, cap ? cap : 1);
    } catch (const Error& e) {
        if (e.status != DRG_ENOMEM) throw;
        scol.reset();
        sdist.reset();
        cap = 0;  // no room to stage: every row overflows and is traversed twice
        scol = DBuf<uint32_t>(ctx, 1);
        sdist = DBuf<uint8_t>(ctx, 1);
    }
    BfsArgs a{};
    a.rp = g->rp; a.col = g->col; a.n = n; a.k = k; a.words = words; a.swords = swords;
    a.gbitmaps = smem_bm ? nullptr : gbm.p;
    a.lists = lists.p; a.wlists = wlists.p; a.dlev = dlev.p;
    a.next_row = counter.p; a.counts = counts.p;
    a.staged = 1; a.cursor = cursor.p; a.cap = cap; a.row_off = row_off.p; a.overflow = overflow.p;
    a.out_col = scol.p; a.out_dist = sdist.p;
    DRG_CUDA(cudaMemsetAsync(counter.p, 0, 4, ctx->stream));
    DRG_CUDA(cudaMemsetAsync(overflow.p, 0, 4, ctx->stream));
    DRG_CUDA(cudaMemsetAsync(cursor.p, 0, 8, ctx->stream));
    {
        ProfSpan sb(ctx, DRG_PROF_BFS, 0);
        DRG_LAUNCH(ctx, kern, blocks, BFS_THREADS, dyn, a);
    }
    DBuf<uint64_t> tot(ctx, 1);
    scan<uint64_t>(ctx, LoadArr<uint64_t>{counts.p}, n, d->rp, false, tot.p);
    d2d(ctx, d->rp + n, tot.p, 1);
    d->nnz = read1(ctx, tot.p);
    DRG_CHECK(d->nnz < (1ull << 32), DRG_EUNSUPPORTED, "distance matrix has 2^32 entries or more");
    const bool overflowed = read1(ctx, overflow.p) != 0;
    d->col = static_cast<uint32_t*>(dalloc(ctx, sizeof(uint32_t) * (d->nnz ? d->nnz : 1)));
    d->dist = static_cast<uint8_t*>(dalloc(ctx, d->nnz ? d->nnz : 1));
    if (!overflowed) {
        DRG_LAUNCH(ctx, k_unstage, grid_for((size_t)n * 32, 256, (uint32_t)ctx->num_sms * 16), 256, 0, row_off.p,
                   d->rp, n, scol.p, sdist.p, d->col, d->dist);
        return;
    }
    // the staging area was too small: traverse again, writing at the final offsets
    scol.reset();
    sdist.reset();
    a.staged = 0;
    a.gd_rp = d->rp;
    a.out_col = d->col;
    a.out_dist = d->dist;
    DRG_CUDA(cudaMemsetAsync(counter.p, 0, 4, ctx->stream));
    ProfSpan sb(ctx, DRG_PROF_BFS, 0);
    DRG_LAUNCH(ctx, kern, blocks, BFS_THREADS, dyn, a);
}

// ------------------------------------------------------------------ similarity
struct Gauss {
    float g[16];
};

// Z_i = sum over d = 1..k of count_i(d) * g(d), in that order, FP32
// correctly rounded with no fused multiply-add (one warp per row).
__global__ void k_row_Z(const uint64_t* __restrict__ rp, const uint8_t* __restrict__ dist, uint32_t n, uint32_t k,
                        Gauss gs, float* __restrict__ Z) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warp0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t i = warp0; i < n; i += nwarps) {
        // class counts by warp ballots: every lane ends with the same totals
        uint32_t c[15];
#pragma unroll
        for (int d = 0; d < 15; ++d) c[d] = 0;
        const uint64_t e0 = rp[i], e1 = rp[i + 1];
        for (uint64_t b = e0; b < e1; b += 32) {
            const uint64_t e = b + lane;
            const uint32_t dd = e < e1 ? dist[e] : 0u;
#pragma unroll
            for (int d = 0; d < 15; ++d)
                if ((uint32_t)d < k) c[d] += __popc(__ballot_sync(0xFFFFFFFFu, dd == (uint32_t)(d + 1)));
        }
        float z = 0.f;
#pragma unroll
        for (int d = 0; d < 15; ++d)
            if ((uint32_t)d < k) z = __fadd_rn(z, __fmul_rn(__uint2float_rn(c[d]), gs.g[d]));
        if (lane == 0) Z[i] = z;
    }
}

// q_e = floor((fl(g/Z_i) + fl(g/Z_j)) * 2^30).
__global__ void k_quantise(const uint32_t* __restrict__ esrc, const uint32_t* __restrict__ col,
                           const uint8_t* __restrict__ dist, const float* __restrict__ Z, Gauss gs, uint64_t nnz,
                           uint32_t* __restrict__ q) {
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < nnz; e += (uint64_t)gridDim.x * blockDim.x) {
        const float gd = gs.g[dist[e] - 1];
        const float s = __fadd_rn(__fdiv_rn(gd, Z[esrc[e]]), __fdiv_rn(gd, Z[col[e]]));
        q[e] = __float2uint_rz(__fmul_rn(s, 1073741824.0f));
    }
}

// r_i = sum of q over row i (exact, one warp per row); also the maximum.
__global__ void k_row_r(const uint64_t* __restrict__ rp, const uint32_t* __restrict__ q, uint32_t n,
                        uint64_t* __restrict__ r, unsigned long long* __restrict__ rmax) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warp0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t i = warp0; i < n; i += nwarps) {
        uint64_t s = 0;
        for (uint64_t e = rp[i] + lane; e < rp[i + 1]; e += 32) s += q[e];
#pragma unroll
        for (int off = 16; off; off >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, off);
        if (lane == 0) {
            r[i] = s;
            atomicMax(rmax, (unsigned long long)s);
        }
    }
}

__global__ void k_shift_u32(const uint64_t* __restrict__ r, uint32_t n, uint32_t s, uint32_t* __restrict__ out) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        out[i] = (uint32_t)(r[i] >> s);
}

// ------------------------------------------------------------------ alias tables
// Exact integer "sweep" construction (Huebschle-Schneider & Sanders 2019) in
// its merge form: with a_i = q_i N and bucket capacity W = sum q, lights
// (a < W) and heavies (a >= W) keep index order; Dl(x) is the lights'
// cumulative deficit before light x, S(y) the heavies' cumulative excess up to
// and including heavy y.  Merging Dl and S (a light precedes a heavy iff
// Dl < S) gives every light the number of heavies before it -- its alias is
// the next heavy -- and every heavy the number of lights before it, from
// which its own remaining mass follows.
struct LightDeficit {
    const uint32_t* q; const uint32_t* L; uint64_t N, W;
    __device__ __forceinline__ u128 operator()(size_t x) const { return (u128)(W - (uint64_t)q[L[x]] * N); }
};
struct HeavyExcess {
    const uint32_t* q; const uint32_t* H; uint64_t N, W;
    __device__ __forceinline__ u128 operator()(size_t y) const { return (u128)((uint64_t)q[H[y]] * N - W); }
};
struct LightFlag {
    const uint32_t* q; uint64_t N, W;
    __device__ __forceinline__ uint32_t operator()(size_t i) const { return (uint64_t)q[i] * N < W ? 1u : 0u; }
};

__global__ void k_split(const uint32_t* __restrict__ q, const uint32_t* __restrict__ lpos, uint64_t N, uint64_t W,
                        uint32_t* __restrict__ L, uint32_t* __restrict__ H) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < N; i += (uint64_t)gridDim.x * blockDim.x) {
        if ((uint64_t)q[i] * N < W) L[lpos[i]] = (uint32_t)i;
        else H[i - lpos[i]] = (uint32_t)i;
    }
}

__device__ __forceinline__ uint64_t merge_path(const u128* A, uint64_t nA, const u128* B, uint64_t nB, uint64_t diag) {
    uint64_t lo = diag > nB ? diag - nB : 0;
    uint64_t hi = diag < nA ? diag : nA;
    while (lo < hi) {
        const uint64_t mid = (lo + hi) >> 1;
        if (A[mid] < B[diag - mid - 1]) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

constexpr int MERGE_THREADS = 256, MERGE_ITEMS = 8, MERGE_TILE = MERGE_THREADS * MERGE_ITEMS;

// Merge-path split of every tile boundary (diagonal t * MERGE_TILE, and the
// end): one thread per boundary, all searches in flight together.
__global__ void k_merge_partition(const u128* __restrict__ A, uint64_t nA, const u128* __restrict__ B, uint64_t nB,
                                  uint64_t tiles, uint64_t* __restrict__ part) {
    const uint64_t total = nA + nB;
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t <= tiles; t += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t d = t * MERGE_TILE < total ? t * MERGE_TILE : total;
        part[t] = merge_path(A, nA, B, nB, d);
    }
}

__global__ void __launch_bounds__(MERGE_THREADS) k_merge_ranks(const u128* __restrict__ A, uint64_t nA,
                                                               const u128* __restrict__ B, uint64_t nB,
                                                               const uint64_t* __restrict__ part,
                                                               uint32_t* __restrict__ a_rank,
                                                               uint32_t* __restrict__ b_rank) {
    __shared__ u128 s[MERGE_TILE];
    const uint64_t total = nA + nB;
    const uint64_t d0 = (uint64_t)blockIdx.x * MERGE_TILE;
    const uint64_t d1 = d0 + MERGE_TILE < total ? d0 + MERGE_TILE : total;
    const uint64_t x0 = part[blockIdx.x], x1 = part[blockIdx.x + 1], y0 = d0 - x0, y1 = d1 - x1;
    const uint32_t na = (uint32_t)(x1 - x0), nb = (uint32_t)(y1 - y0);
    for (uint32_t t = threadIdx.x; t < na; t += MERGE_THREADS) s[t] = A[x0 + t];
    for (uint32_t t = threadIdx.x; t < nb; t += MERGE_THREADS) s[na + t] = B[y0 + t];
    __syncthreads();
    const u128* As = s;
    const u128* Bs = s + na;
    const uint32_t dl = threadIdx.x * MERGE_ITEMS;
    if (dl >= na + nb) return;
    uint32_t xa = (uint32_t)merge_path(As, na, Bs, nb, dl);
    uint32_t yb = dl - xa;
#pragma unroll
    for (int it = 0; it < MERGE_ITEMS; ++it) {
        if (xa + yb >= na + nb) break;
        if (xa < na && (yb >= nb || As[xa] < Bs[yb])) {
            a_rank[x0 + xa] = (uint32_t)(y0 + yb);
            ++xa;
        } else {
            b_rank[y0 + yb] = (uint32_t)(x0 + xa);
            ++yb;
        }
    }
}

// floor(own * 2^32 / W) for own < W and a fixed W: division by an invariant
// integer with a precomputed reciprocal (Moeller & Granlund, "Improved
// division by invariant integers", IEEE Trans. Computers 2011, 2-by-1
// division).  W is normalised to d = W << s (top bit set), v = floor((2^128 -
// 1) / d) - 2^64; the numerator own * 2^(32 + s) splits into words (u1, u0).
struct InvDiv {
    uint64_t d, v;
    int s;
};

static InvDiv make_invdiv(uint64_t W) {
    const int s = __builtin_clzll(W);
    const uint64_t d = W << s;
    const u128 v = (~(u128)0) / d - ((u128)1 << 64);
    return InvDiv{d, (uint64_t)v, s};
}

__device__ __forceinline__ uint32_t frac32(uint64_t own, const InvDiv& D) {
    const int sh = 32 + D.s;
    uint64_t u1, u0;
    if (sh >= 64) {
        u1 = own << (sh - 64);
        u0 = 0;
    } else {
        u1 = own >> (64 - sh);
        u0 = own << sh;
    }
    uint64_t q0 = D.v * u1;
    uint64_t q1 = __umul64hi(D.v, u1);
    q0 += u0;
    q1 += u1 + (q0 < u0 ? 1u : 0u);
    q1 += 1;
    uint64_t r = u0 - q1 * D.d;
    if (r > q0) {
        q1 -= 1;
        r += D.d;
    }
    if (r >= D.d) q1 += 1;
    return (uint32_t)q1;
}

__global__ void k_alias_lights(const uint32_t* __restrict__ q, const uint32_t* __restrict__ L, uint64_t nL,
                               const uint32_t* __restrict__ H, const uint32_t* __restrict__ a_rank, uint64_t N,
                               uint64_t W, InvDiv D, uint32_t* __restrict__ thresh, uint32_t* __restrict__ alias) {
    for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < nL; x += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t b = L[x];
        thresh[b] = frac32((uint64_t)q[b] * N, D);
        alias[b] = H[a_rank[x]];
    }
}

__global__ void k_alias_heavies(const uint32_t* __restrict__ H, uint64_t nH, const u128* __restrict__ S,
                                const u128* __restrict__ Dl, const uint32_t* __restrict__ b_rank, uint64_t W,
                                InvDiv D, uint32_t* __restrict__ thresh, uint32_t* __restrict__ alias) {
    for (uint64_t y = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; y < nH; y += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t b = H[y];
        const uint64_t own = (uint64_t)(S[y] + (u128)W - Dl[b_rank[y]]);
        // exact totals make the last heavy full; the index guard only keeps a
        // violated invariant from reading past H
        if (own >= W || y + 1 >= nH) {
            thresh[b] = 0xFFFFFFFFu;
            alias[b] = b;
        } else {
            thresh[b] = frac32(own, D);
            alias[b] = H[y + 1];
        }
    }
}

struct Sum64 {
    const uint32_t* q;
    __device__ __forceinline__ uint64_t operator()(size_t i) const { return q[i]; }
};

// Alias table over N items with 32-bit weights q; thresh/alias are [N].
// Returns false (tables untouched) when the weights sum to zero.
bool build_alias(drg_ctx* ctx, const uint32_t* q, uint64_t N, uint32_t* thresh, uint32_t* alias) {
    DRG_CHECK(N > 0 && N < (1ull << 32), DRG_EUNSUPPORTED, "alias table size must be in [1, 2^32)");
    DBuf<uint64_t> Wd(ctx, 1);
    {
        DBuf<uint64_t> tmp(ctx, 1);
        // reduce via the scan machinery (exclusive output discarded in a small buffer per block)
        DBuf<uint64_t> sums(ctx, (N + ScanShape<uint64_t>::TILE - 1) / ScanShape<uint64_t>::TILE);
        const uint32_t nb = (uint32_t)sums.n;
        DRG_LAUNCH(ctx, (k_scan_reduce<uint64_t, Sum64>), nb, 256, 0, Sum64{q}, (size_t)N, sums.p);
        scan<uint64_t>(ctx, LoadArr<uint64_t>{sums.p}, nb, sums.p, false, Wd.p);
    }
    const uint64_t W = read1(ctx, Wd.p);
    if (W == 0) return false;
    DBuf<uint32_t> lpos(ctx, N), nLd(ctx, 1);
    scan<uint32_t>(ctx, LightFlag{q, N, W}, N, lpos.p, false, nLd.p);
    const uint64_t nL = read1(ctx, nLd.p);
    const uint64_t nH = N - nL;
    DBuf<uint32_t> L(ctx, nL), H(ctx, nH);
    const uint32_t g = grid_for(N, 256, 65536);
    DRG_LAUNCH(ctx, k_split, g, 256, 0, q, lpos.p, N, W, L.p, H.p);
    lpos.reset();
    DBuf<u128> Dl(ctx, nL + 1), S(ctx, nH);
    scan<u128>(ctx, LightDeficit{q, L.p, N, W}, nL, Dl.p, false, Dl.p + nL);
    scan<u128>(ctx, HeavyExcess{q, H.p, N, W}, nH, S.p, true, nullptr);
    DBuf<uint32_t> a_rank(ctx, nL), b_rank(ctx, nH);
    const uint64_t tiles = (N + MERGE_TILE - 1) / MERGE_TILE;
    {
        DBuf<uint64_t> part(ctx, tiles + 1);
        DRG_LAUNCH(ctx, k_merge_partition, grid_for(tiles + 1, 256, 65536), 256, 0, Dl.p, nL, S.p, nH, tiles, part.p);
        DRG_LAUNCH(ctx, k_merge_ranks, (uint32_t)tiles, MERGE_THREADS, 0, Dl.p, nL, S.p, nH, part.p, a_rank.p,
                   b_rank.p);
    }
    DRG_LAUNCH(ctx, k_alias_lights, grid_for(nL, 256, 65536), 256, 0, q, L.p, nL, H.p, a_rank.p, N, W, make_invdiv(W), thresh, alias);
    DRG_LAUNCH(ctx, k_alias_heavies, grid_for(nH, 256, 65536), 256, 0, H.p, nH, S.p, Dl.p, b_rank.p, W, make_invdiv(W), thresh,
               alias);
    return true;
}

template <bool PACKED>
__global__ void k_edge_records(const uint32_t* __restrict__ thresh, const uint32_t* __restrict__ alias,
                               const uint32_t* __restrict__ esrc, const uint32_t* __restrict__ col, uint64_t nnz,
                               void* __restrict__ out) {
    for (uint64_t b = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; b < nnz; b += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t al = alias[b];
        if constexpr (PACKED) {
            static_cast<uint4*>(out)[b] = pack_edge16(thresh[b], esrc[b], col[b], esrc[al], col[al]);
        } else {
            EdgeRec r;
            r.thresh = thresh[b];
            r.i0 = esrc[b];
            r.j0 = col[b];
            r.i1 = esrc[al];
            r.j1 = col[al];
            r.pad0 = r.pad1 = r.pad2 = 0;
            static_cast<EdgeRec*>(out)[b] = r;
        }
    }
}

__global__ void k_node_records(const uint32_t* __restrict__ thresh, const uint32_t* __restrict__ alias, uint32_t n,
                               uint2* __restrict__ out) {
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x)
        out[v] = make_uint2(thresh[v], alias[v]);
}

void dmat_free(drg_dmat* d) {
    if (!d) return;
    drg_ctx* c = d->ctx;
    void* ps[] = {d->rp, d->col, d->dist, d->q, d->r, d->Z, d->etab, d->e_alias, d->vtab};
    for (void* p : ps)
        if (p) dfree(c, p);
    delete d;
}

drg_dmat* build_dmat(drg_ctx* ctx, const drg_graph* g, uint32_t k, float sigma) {
    DRG_CHECK(g, DRG_EINVAL, "null graph");
    DRG_CHECK(k >= 1 && k <= 15, DRG_EINVAL, "k must be in [1, 15]");
    DRG_CHECK(sigma > 0.f, DRG_EINVAL, "sigma must be positive");
    drg_dmat* d = new drg_dmat();
    d->ctx = ctx;
    d->n = g->n;
    d->k = k;
    d->sigma = sigma;
    try {
        DRG_CHECK(g->nnz > 0, DRG_EEMPTY, "graph has no edges");
        ProfSpan span(ctx, DRG_PROF_DMAT, 0);
        build_korder(ctx, g, k, d);
        span.units = d->nnz;
        const uint32_t n = d->n;
        const uint64_t nnz = d->nnz;
        ProfSpan ss(ctx, DRG_PROF_SIM, nnz);
        Gauss gs{};
        for (uint32_t x = 1; x <= k; ++x)
            gs.g[x - 1] = (float)std::exp(-(double)(x * x) / (2.0 * (double)sigma * (double)sigma));
        d->Z = static_cast<float*>(dalloc(ctx, sizeof(float) * n));
        d->q = static_cast<uint32_t*>(dalloc(ctx, sizeof(uint32_t) * nnz));
        d->r = static_cast<uint64_t*>(dalloc(ctx, sizeof(uint64_t) * n));
        const uint32_t gw = grid_for((size_t)n * 32, 256, (uint32_t)ctx->num_sms * 16);
        DRG_LAUNCH(ctx, k_row_Z, gw, 256, 0, d->rp, d->dist, n, k, gs, d->Z);
        DBuf<uint32_t> esrc(ctx, nnz);
        DRG_LAUNCH(ctx, k_expand_rows, gw, 256, 0, d->rp, n, esrc.p);
        DRG_LAUNCH(ctx, k_quantise, grid_for(nnz, 256, 65536), 256, 0, esrc.p, d->col, d->dist, d->Z, gs, nnz, d->q);
        DBuf<unsigned long long> rmax(ctx, 1);
        DRG_CUDA(cudaMemsetAsync(rmax.p, 0, 8, ctx->stream));
        DRG_LAUNCH(ctx, k_row_r, gw, 256, 0, d->rp, d->q, n, d->r, rmax.p);
        const uint64_t mx = read1(ctx, rmax.p);
        const int bits = bitlen(mx);
        d->shift = bits > 32 ? (uint32_t)(bits - 32) : 0u;
        ss.reopen(DRG_PROF_ALIAS, nnz + n);
        // edge table over the entries (positive samples)
        {
            DBuf<uint32_t> th(ctx, nnz);
            d->e_alias = static_cast<uint32_t*>(dalloc(ctx, sizeof(uint32_t) * nnz));
            DRG_CHECK(build_alias(ctx, d->q, nnz, th.p, d->e_alias), DRG_EEMPTY, "all edge weights are zero");
            const bool packed = n <= kPackedIdLimit;
            d->erec_bytes = packed ? 16u : (uint32_t)sizeof(EdgeRec);
            d->etab = dalloc(ctx, (size_t)d->erec_bytes * nnz);
            DRG_LAUNCH(ctx, packed ? k_edge_records<true> : k_edge_records<false>, grid_for(nnz, 256, 65536), 256, 0,
                       th.p, d->e_alias, esrc.p, d->col, nnz, d->etab);
        }
        // node table (negative samples)
        {
            DBuf<uint32_t> r32(ctx, n), th(ctx, n), al(ctx, n);
            DRG_LAUNCH(ctx, k_shift_u32, grid_for(n, 256, 65536), 256, 0, d->r, n, d->shift, r32.p);
            DRG_CHECK(build_alias(ctx, r32.p, n, th.p, al.p), DRG_EEMPTY, "all node weights are zero");
            d->vtab = static_cast<uint2*>(dalloc(ctx, sizeof(uint2) * n));
            DRG_LAUNCH(ctx, k_node_records, grid_for(n, 256, 65536), 256, 0, th.p, al.p, n, d->vtab);
        }
        sync(ctx);
    } catch (...) {
        dmat_free(d);
        throw;
    }
    return d;
}

}  // namespace drg
