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
// touched words in increasing order; each warp takes a contiguous range of
// them and prefix-sums their popcounts with shuffles) -- no global sort.  Hop
// distances: for k = 2 a node is at distance 1 exactly when it is in the
// source's adjacency; after the row is written, each adjacency node finds its
// word in the (shared) word list, whose output offsets were recorded, and
// marks its entry (rows with more touched words than the shared list holds
// search the emitted row instead); for k > 2 the block records each
// discovered node's level.
// Staged mode writes each row into a staging area at an offset reserved with
// an atomic cursor (one traversal gives the counts and the rows); direct mode
// writes at the final row offsets and is the fallback when the staging area
// overflows.
// Block sizes of the block kernel: 1024 threads when the bitmap leaves room
// for one block per SM (large graphs), else 512 (several blocks per SM).
constexpr int BFS_THREADS_BIG = 1024, BFS_THREADS_SMALL = 512;

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
    const uint32_t* rows;     // rows to traverse (nullptr: all rows 0 .. n-1)
    uint32_t nrows;
    uint64_t* counts;         // row sizes (written in both modes)
    int staged;               // 1: write at a reserved staging offset
    unsigned long long* cursor;  // staged: next free staging entry
    uint64_t cap;             // staged: staging capacity
    uint64_t* row_off;        // staged: staging offset of each row
    uint32_t* overflow;       // staged: set when a row did not fit
    uint32_t row_cap;         // > 0: each row keeps its row_cap nearest nodes (k_cap_rows only)
    const uint32_t* tcol;     // k_cap_rows: each row's adjacency as tie values, ascending
    const uint64_t* gd_rp;    // direct: row offsets
    uint32_t* out_col;        // staging or final column array
    uint8_t* out_dist;        // staging or final distance array
};

// Counts the warp's new nodes in s_len and, when `store`, appends them to the
// discovered list (the last level's nodes are only counted).
__device__ __forceinline__ void bfs_append(uint32_t v, bool isnew, uint32_t* list, uint32_t* s_len, bool store) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t ballot = __ballot_sync(0xFFFFFFFFu, isnew);
    if (!ballot) return;
    uint32_t base = 0;
    if (lane == (uint32_t)(__ffs(ballot) - 1)) base = atomicAdd(s_len, (uint32_t)__popc(ballot));
    if (!store) return;
    base = __shfl_sync(0xFFFFFFFFu, base, __ffs(ballot) - 1);
    if (isnew) list[base + __popc(ballot & lanemask_lt())] = v;
}

constexpr int BFS_UNROLL = 4;          // adjacency loads in flight per thread
constexpr uint32_t BFS_WL_SMEM = 4096;  // touched-word list (and offsets) in shared memory up to this length

// Dynamic shared memory besides the bitmap: summary, word list, word offsets.
static size_t bfs_extra_smem(uint32_t swords) { return (size_t)(swords + 2 * BFS_WL_SMEM) * 4; }

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

// Marks v visited and its word touched, without asking who was first.
__device__ __forceinline__ void mark(uint32_t* bm, uint32_t* summ, uint32_t v) {
    const uint32_t w = v >> 5, bit = 1u << (v & 31);
    if (*(volatile uint32_t*)&bm[w] & bit) return;
    atomicOr(&bm[w], bit);
    const uint32_t sbit = 1u << (w & 31);
    if (!(*(volatile uint32_t*)&summ[w >> 5] & sbit)) atomicOr(&summ[w >> 5], sbit);
}

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v, uint32_t lane) {
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, v, off);
        if (lane >= (uint32_t)off) v += t;
    }
    return v;
}

template <bool K2, int BFS_THREADS>
__global__ void __launch_bounds__(BFS_THREADS, BFS_THREADS == 512 ? 3 : 1) k_bfs(BfsArgs a) {
    extern __shared__ uint32_t dsm[];
    __shared__ uint64_t s_off[BFS_THREADS];
    __shared__ uint64_t s_start[BFS_THREADS];
    __shared__ uint64_t s_wt[BFS_THREADS / 32];
    __shared__ uint32_t s_row, s_len, s_next;
    __shared__ uint64_t s_base;
    __shared__ int s_skip;
    __shared__ uint32_t s_wcnt[BFS_THREADS / 32];
    uint32_t* bm = a.gbitmaps ? a.gbitmaps + (size_t)blockIdx.x * a.words : dsm;
    uint32_t* summ = a.gbitmaps ? dsm : dsm + a.words;
    uint32_t* s_wl = summ + a.swords;
    uint32_t* s_woff = s_wl + BFS_WL_SMEM;  // output offset of each listed word, relative to the row
    uint32_t* list = a.lists + (size_t)blockIdx.x * a.n;
    uint32_t* wl = a.wlists + (size_t)blockIdx.x * a.words;
    uint8_t* dl = K2 ? nullptr : a.dlev + (size_t)blockIdx.x * a.n;
    for (uint32_t w = threadIdx.x; w < a.words; w += BFS_THREADS) bm[w] = 0;
    for (uint32_t w = threadIdx.x; w < a.swords; w += BFS_THREADS) summ[w] = 0;
    if (threadIdx.x == 0) s_next = atomicAdd(a.next_row, 1u);
    __syncthreads();
    for (;;) {
        if (threadIdx.x == 0) {
            s_row = s_next < a.nrows ? (a.rows ? a.rows[s_next] : s_next) : 0xFFFFFFFFu;
            s_len = 0;
        }
        __syncthreads();
        const uint32_t row = s_row;
        if (row == 0xFFFFFFFFu) break;
        // the next row's index, taken now and stored once this row is done
        uint32_t next = 0;
        if (threadIdx.x == 0) {
            next = atomicAdd(a.next_row, 1u);
            visit(bm, summ, row);
        }
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
            bfs_append(v, isnew, list, &s_len, a.k > 1);
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
                const bool store = d < a.k;
                for (uint64_t x0 = 0; x0 < tot; x0 += (uint64_t)BFS_UNROLL * BFS_THREADS) {
                    // each thread takes BFS_UNROLL consecutive slots of the
                    // concatenated adjacency: one search for the owner of the
                    // first (the last frontier slot whose offset is <= x),
                    // then a walk forward for the others
                    uint32_t v[BFS_UNROLL];
                    const uint64_t xb = x0 + (uint64_t)threadIdx.x * BFS_UNROLL;
                    uint32_t own = 0;
                    if (xb < tot) {
                        uint32_t hi2 = cnt;
                        while (hi2 - own > 1) {
                            const uint32_t mid = (own + hi2) >> 1;
                            if (s_off[mid] <= xb) own = mid; else hi2 = mid;
                        }
                    }
#pragma unroll
                    for (int u = 0; u < BFS_UNROLL; ++u) {
                        const uint64_t x = xb + u;
                        v[u] = 0xFFFFFFFFu;
                        if (x < tot) {
                            while (own + 1 < cnt && s_off[own + 1] <= x) ++own;
                            v[u] = a.col[s_start[own] + (x - s_off[own])];
                        }
                    }
                    if (K2 && !store) {
                        // last level of k = 2: only mark (the row is counted from the
                        // bitmap when it is written)
#pragma unroll
                        for (int u = 0; u < BFS_UNROLL; ++u)
                            if (v[u] != 0xFFFFFFFFu) mark(bm, summ, v[u]);
                    } else {
#pragma unroll
                        for (int u = 0; u < BFS_UNROLL; ++u) {
                            const bool isnew = v[u] != 0xFFFFFFFFu && visit(bm, summ, v[u]);
                            if (!K2 && isnew) dl[v[u]] = (uint8_t)d;
                            bfs_append(v[u], isnew, list, &s_len, store);
                        }
                    }
                }
                __syncthreads();
            }
            lo = hi;
            hi = s_len;
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            s_next = next;
            bm[row >> 5] &= ~(1u << (row & 31));  // the source is not its own neighbour
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
        const bool wl_smem = nw <= BFS_WL_SMEM;
        uint32_t* wlist = wl_smem ? s_wl : wl;
        for (uint32_t s = s0; s < s1; ++s) {
            uint32_t m = summ[s];
            summ[s] = 0;
            while (m) {
                const uint32_t b = __ffs(m) - 1;
                m &= m - 1;
                wlist[pos++] = 32 * s + b;
            }
        }
        __syncthreads();
        // every touched word's bits, in order: warp w takes words [w0, w1)
        const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        constexpr uint32_t NW = BFS_THREADS / 32;
        const uint64_t wper = (nw + NW - 1) / NW;
        const uint64_t w0 = (uint64_t)warp * wper < nw ? (uint64_t)warp * wper : nw;
        const uint64_t w1 = w0 + wper < nw ? w0 + wper : nw;
        uint32_t cw = 0;
        for (uint64_t x = w0 + lane; x < w1; x += 32) cw += __popc(bm[wlist[x]]);
#pragma unroll
        for (int off = 16; off; off >>= 1) cw += __shfl_xor_sync(0xFFFFFFFFu, cw, off);
        if (lane == 0) s_wcnt[warp] = cw;
        __syncthreads();
        uint64_t out = 0;  // relative to the row
        for (uint32_t w = 0; w < warp; ++w) out += s_wcnt[w];
        // the row's size, and its place
        if (threadIdx.x == 0) {
            uint32_t total = 0;
            for (uint32_t w = 0; w < NW; ++w) total += s_wcnt[w];
            s_len = total;
            a.counts[row] = total;
            uint64_t base = 0;
            int skip = 0;
            if (a.staged) {
                // staged rows start at multiples of 16 entries (aligned copies later)
                const uint64_t span = ((uint64_t)total + 15) & ~15ull;
                base = atomicAdd(a.cursor, (unsigned long long)span);
                if (base + span > a.cap) {
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
        const uint32_t total = s_len;
        const bool emit = !s_skip;
        for (uint64_t x0 = w0; x0 < w1; x0 += 32) {
            const uint64_t x = x0 + lane;
            uint32_t wi = 0, w = 0;
            if (x < w1) {
                wi = wlist[x];
                w = bm[wi];
            }
            const uint32_t c = __popc(w);
            uint32_t incl = c;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, off);
                if (lane >= (uint32_t)off) incl += t;
            }
            const uint32_t excl = incl - c;
            const uint32_t ctot = __shfl_sync(0xFFFFFFFFu, incl, 31);
            if (wl_smem && x < w1) s_woff[x] = (uint32_t)(out + excl);
            if (emit) {
                uint64_t o = out + excl;
                while (w) {
                    const uint32_t b = __ffs(w) - 1;
                    w &= w - 1;
                    const uint32_t v = 32 * wi + b;
                    a.out_col[s_base + o] = v;
                    if (!K2) a.out_dist[s_base + o] = dl[v];
                    ++o;
                }
            }
            out += ctot;
        }
        if (K2 && emit) {
            // every distance 2 (aligned 16-byte stores), then the adjacency's 1s
            uint8_t* dd = a.out_dist + s_base;
            const uint64_t head = ((16 - ((uintptr_t)dd & 15)) & 15) < total ? ((16 - ((uintptr_t)dd & 15)) & 15) : total;
            if (threadIdx.x < head) dd[threadIdx.x] = 2;
            const uint64_t body = (total - head) / 16;
            uint4* dv = reinterpret_cast<uint4*>(dd + head);
            for (uint64_t t = threadIdx.x; t < body; t += BFS_THREADS)
                dv[t] = make_uint4(0x02020202u, 0x02020202u, 0x02020202u, 0x02020202u);
            for (uint64_t t = head + 16 * body + threadIdx.x; t < total; t += BFS_THREADS) dd[t] = 2;
        }
        __syncthreads();
        if (K2 && emit) {
            // distance 1: the source's adjacency
            for (uint64_t x = ab + threadIdx.x; x < ae; x += BFS_THREADS) {
                const uint32_t v = a.col[x];
                uint64_t at;
                if (wl_smem) {
                    // its word in the list, then its bit within the word
                    uint32_t lo3 = 0, hi3 = (uint32_t)nw;
                    while (lo3 < hi3) {
                        const uint32_t mid = (lo3 + hi3) >> 1;
                        if (s_wl[mid] < (v >> 5)) lo3 = mid + 1; else hi3 = mid;
                    }
                    at = s_woff[lo3] + __popc(bm[v >> 5] & ((1u << (v & 31)) - 1u));
                } else {
                    // in the emitted (sorted) row
                    const uint32_t* rowc = a.out_col + s_base;
                    uint32_t lo3 = 0, hi3 = total;
                    while (lo3 < hi3) {
                        const uint32_t mid = (lo3 + hi3) >> 1;
                        if (rowc[mid] < v) lo3 = mid + 1; else hi3 = mid;
                    }
                    at = lo3;
                }
                a.out_dist[s_base + at] = 1;
            }
            __syncthreads();
        }
        for (uint64_t x = threadIdx.x; x < nw; x += BFS_THREADS) bm[wlist[x]] = 0;
        __syncthreads();
    }
}

// Ascending bitonic sort of buf[0, m) by one warp; pads to a power of two with
// all-ones keys (buf must hold that power of two).
__device__ __forceinline__ void warp_bitonic(uint32_t* buf, uint32_t m, uint32_t lane) {
    uint32_t P = 1, lp = 0;
    while (P < m) {
        P <<= 1;
        ++lp;
    }
    for (uint32_t x = m + lane; x < P; x += 32) buf[x] = 0xFFFFFFFFu;
    __syncwarp();
    for (uint32_t lk = 1; lk <= lp; ++lk) {
        for (int lj = (int)lk - 1; lj >= 0; --lj) {
            const uint32_t j = 1u << lj;
            for (uint32_t t = lane; t < P / 2; t += 32) {
                const uint32_t i = ((t >> lj) << (lj + 1)) | (t & (j - 1)), l = i + j;
                const uint32_t u = buf[i], w = buf[l];
                if ((u > w) == (((i >> lk) & 1u) == 0)) {
                    buf[i] = w;
                    buf[l] = u;
                }
            }
            __syncwarp();
        }
    }
}

// ------------------------------------------------------------------ small rows, k = 2
// Rows whose candidate count (the source's degree plus its neighbours'
// degrees) is at most SMALL_CAP are built by one warp each, with no block
// barrier: the warp copies the source's adjacency (key v << 1) and every
// neighbour's adjacency except the source (key v << 1 | 1) into shared
// memory, load-balanced over its lanes; sorts the keys (bitonic); keeps the
// first key of each node -- its distance is 1 + its low bit -- and writes the
// row to the staging area.
constexpr uint32_t SMALL_CAP = 2048;
constexpr int SMALL_WARPS = 8;


__global__ void __launch_bounds__(SMALL_WARPS * 32) k_bfs_small(BfsArgs a) {
    extern __shared__ uint32_t small_smem[];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t* buf = small_smem + (size_t)warp * SMALL_CAP;
    for (;;) {
        uint32_t idx = 0;
        if (lane == 0) idx = atomicAdd(a.next_row, 1u);
        idx = __shfl_sync(0xFFFFFFFFu, idx, 0);
        if (idx >= a.nrows) break;
        const uint32_t row = a.rows[idx];
        const uint64_t ab = a.rp[row], ae = a.rp[row + 1];
        const uint32_t deg = (uint32_t)(ae - ab);
        for (uint32_t x = lane; x < deg; x += 32) buf[x] = a.col[ab + x] << 1;
        uint32_t m = deg;
        // neighbours' adjacencies, 32 neighbours at a time
        for (uint32_t c = 0; c < deg; c += 32) {
            uint64_t st = 0;
            uint32_t d = 0;
            if (c + lane < deg) {
                const uint32_t u = a.col[ab + c + lane];
                st = a.rp[u];
                d = (uint32_t)(a.rp[u + 1] - st);
            }
            const uint32_t incl = warp_incl_scan(d, lane);
            const uint32_t tot = __shfl_sync(0xFFFFFFFFu, incl, 31);
            const uint32_t excl = incl - d;
            for (uint32_t x0 = 0; x0 < tot; x0 += 32) {
                const uint32_t x = x0 + lane;
                // owner: last lane whose exclusive offset is <= x (five steps on every lane)
                uint32_t lo = 0, hi = 32;
                while (hi - lo > 1) {
                    const uint32_t mid = (lo + hi) >> 1;
                    if (__shfl_sync(0xFFFFFFFFu, excl, mid) <= x) lo = mid; else hi = mid;
                }
                const uint64_t so = __shfl_sync(0xFFFFFFFFu, st, lo);
                const uint32_t eo = __shfl_sync(0xFFFFFFFFu, excl, lo);
                uint32_t key = 0xFFFFFFFFu;
                if (x < tot) {
                    const uint32_t v = a.col[so + (x - eo)];
                    if (v != row) key = (v << 1) | 1u;
                }
                const uint32_t keep = __ballot_sync(0xFFFFFFFFu, key != 0xFFFFFFFFu);
                if (key != 0xFFFFFFFFu) buf[m + __popc(keep & lanemask_lt())] = key;
                m += __popc(keep);
            }
        }
        // keys v << 1 | 1 stay below the all-ones padding (ids < 2^31 - 1)
        __syncwarp();
        warp_bitonic(buf, m, lane);
        // first key of each node, counted and written in order
        uint32_t total = 0;
        for (uint32_t x0 = 0; x0 < m; x0 += 32) {
            const uint32_t x = x0 + lane;
            const bool first = x < m && (x == 0 || (buf[x] >> 1) != (buf[x - 1] >> 1));
            total += __popc(__ballot_sync(0xFFFFFFFFu, first));
        }
        uint64_t base = 0;
        int skip = 0;
        if (lane == 0) {
            a.counts[row] = total;
            const uint64_t span = ((uint64_t)total + 15) & ~15ull;
            base = atomicAdd(a.cursor, (unsigned long long)span);
            if (base + span > a.cap) {
                skip = 1;
                atomicExch(a.overflow, 1u);
            }
            a.row_off[row] = base;
        }
        base = __shfl_sync(0xFFFFFFFFu, base, 0);
        skip = __shfl_sync(0xFFFFFFFFu, skip, 0);
        if (!skip) {
            uint64_t o = base;
            for (uint32_t x0 = 0; x0 < m; x0 += 32) {
                const uint32_t x = x0 + lane;
                const bool first = x < m && (x == 0 || (buf[x] >> 1) != (buf[x - 1] >> 1));
                const uint32_t bal = __ballot_sync(0xFFFFFFFFu, first);
                if (first) {
                    const uint64_t at = o + __popc(bal & lanemask_lt());
                    a.out_col[at] = buf[x] >> 1;
                    a.out_dist[at] = (uint8_t)(1 + (buf[x] & 1u));
                }
                o += __popc(bal);
            }
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------------ capped rows, one warp each
// Rows of the capped matrix (R24), one warp each: row i keeps K_i, its
// row_cap nearest nodes by (hop distance, tie order of the id).  The tie
// order is a fixed bijection of [0, 2^28): an xor with a constant, a
// multiplication by an odd constant mod 2^28, an xor-shift, again, again; it
// keeps the choice among equally near nodes independent of how the ids were
// assigned.  The traversal reads a copy of the adjacency that holds each
// row's neighbours as tie values in ascending order (tcol).  A source of
// degree >= row_cap keeps the first row_cap of its list.  Otherwise the warp
// holds the row's known nodes as keys (tie << 4 | d - 1, below the all-ones
// padding key even at k = 15) in shared memory and grows them a level at a
// time while fewer than row_cap nodes are known: the lists of the previous
// level's nodes stream through the buffer; whenever it fills, and at the end
// of the level, the keys are sorted (bitonic), only the first key of each
// node is kept (its smallest distance) and, once more than row_cap nodes are
// known, the level is cut to its row_cap - (nodes before it) first keys.  A
// node cut that way never returns: at least that many keys of the level
// before it are kept.  From the first cut on, the largest kept tie value of
// the level bounds what can still enter: later candidates above it are
// dropped, and each list is read only up to it.  The row is then re-keyed by
// id, sorted and written to the staging area (staged) or at its final offset
// (direct).
constexpr uint32_t kTieMask = (1u << 28) - 1;

__device__ __forceinline__ uint32_t tie_of(uint32_t v) {
    uint32_t x = (v ^ 0x2545F49u) & kTieMask;
    x = (x * 0x9E3779Bu) & kTieMask;
    x ^= x >> 14;
    x = (x * 0x85EBCA7u) & kTieMask;
    x ^= x >> 13;
    return x;
}

// The inverse: each step undone in reverse order (the xor-shifts by their
// repeated application within 28 bits, the multiplications by the inverses
// of the odd constants mod 2^28).
__device__ __forceinline__ uint32_t id_of_tie(uint32_t x) {
    x ^= (x >> 13) ^ (x >> 26);
    x = (x * 0x46B2B17u) & kTieMask;
    x ^= x >> 14;
    x = (x * 0x3811693u) & kTieMask;
    return x ^ 0x2545F49u;
}

// Sorts buf[0, m), keeps the first key of each node and, when more than cap
// nodes remain, only the first cap - lower keys of the level whose code (the
// key's low 4 bits) is d (lower = nodes of the levels before it, all kept);
// *tau becomes the largest tie value of that level kept after such a cut.
// Returns the new size (cap when cut).
__device__ __forceinline__ uint32_t capw_flush(uint32_t* buf, uint32_t m, uint32_t lower, uint32_t cap, uint32_t d,
                                               uint32_t lane, uint32_t* tau) {
    warp_bitonic(buf, m, lane);
    // first key of each node (in place)
    uint32_t out = 0, prev = 0xFFFFFFFFu;
    for (uint32_t x0 = 0; x0 < m; x0 += 32) {
        const uint32_t x = x0 + lane;
        const uint32_t key = x < m ? buf[x] : 0xFFFFFFFFu;
        uint32_t before = __shfl_up_sync(0xFFFFFFFFu, key, 1);
        if (lane == 0) before = prev;
        const bool first = x < m && (x == 0 || (key >> 4) != (before >> 4));
        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, first);
        prev = __shfl_sync(0xFFFFFFFFu, key, 31);
        __syncwarp();
        if (first) buf[out + __popc(bal & lanemask_lt())] = key;
        out += __popc(bal);
        __syncwarp();
    }
    if (out <= cap) return out;
    // keep the levels before d and the first cap - lower nodes of level d (in place)
    const uint32_t keep_d = cap - lower;
    uint32_t kept = 0, seen_d = 0, last_d = 0;
    for (uint32_t x0 = 0; x0 < out; x0 += 32) {
        const uint32_t x = x0 + lane;
        const uint32_t key = x < out ? buf[x] : 0u;
        const bool at_d = x < out && (key & 15u) == d;
        const uint32_t db = __ballot_sync(0xFFFFFFFFu, at_d);
        const bool take = x < out && (!at_d || seen_d + __popc(db & lanemask_lt()) < keep_d);
        const uint32_t tb = __ballot_sync(0xFFFFFFFFu, take);
        const uint32_t tdb = tb & db;
        if (tdb) last_d = __shfl_sync(0xFFFFFFFFu, key, 31 - __clz(tdb)) >> 4;
        __syncwarp();
        if (take) buf[kept + __popc(tb & lanemask_lt())] = key;
        kept += __popc(tb);
        seen_d += __popc(db);
        __syncwarp();
    }
    *tau = last_d;
    return kept;
}

// First index in [lo, hi) whose entry is >= tau (hi if none); the entries
// are ascending there.
__device__ __forceinline__ uint64_t capw_clip(const uint32_t* __restrict__ t, uint64_t lo, uint64_t hi, uint32_t tau) {
    while (lo < hi) {
        const uint64_t mid = (lo + hi) >> 1;
        if (t[mid] < tau) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// BUF: keys per warp buffer (>= row_cap + 32); the frontier buffer holds BUF/2.
template <uint32_t BUF, int WARPS>
__global__ void __launch_bounds__(WARPS * 32) k_cap_rows(BfsArgs a) {
    extern __shared__ uint32_t capw_smem[];
    constexpr uint32_t FRONT = BUF / 2;
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t* buf = capw_smem + (size_t)warp * (BUF + FRONT);
    uint32_t* fr = buf + BUF;
    const uint32_t C = a.row_cap;
    for (;;) {
        uint32_t row = 0;
        if (lane == 0) row = atomicAdd(a.next_row, 1u);
        row = __shfl_sync(0xFFFFFFFFu, row, 0);
        if (row >= a.nrows) break;
        const uint32_t trow = tie_of(row);
        const uint64_t ab = a.rp[row], ae = a.rp[row + 1];
        const uint32_t deg = (uint32_t)(ae - ab);
        // level 1: the source's list (all of it, or its first C)
        uint32_t m = deg < C ? deg : C;
        for (uint32_t x = lane; x < m; x += 32) buf[x] = a.tcol[ab + x] << 4;
        __syncwarp();
        for (uint32_t d = 2; d <= a.k && m < C; ++d) {
            // the level-(d-1) nodes
            uint32_t nf = 0;
            for (uint32_t x0 = 0; x0 < m; x0 += 32) {
                const uint32_t x = x0 + lane;
                const bool f = x < m && (buf[x] & 15u) == d - 2;
                const uint32_t fb = __ballot_sync(0xFFFFFFFFu, f);
                if (f) fr[nf + __popc(fb & lanemask_lt())] = id_of_tie(buf[x] >> 4);
                nf += __popc(fb);
            }
            __syncwarp();
            if (nf == 0) break;
            const uint32_t lower = m;
            uint32_t mm = m, tau = 0xFFFFFFFFu;
            for (uint32_t c = 0; c < nf; c += 32) {
                // each lane walks one frontier node's adjacency [cur, end)
                uint64_t cur = 0, end = 0;
                if (c + lane < nf) {
                    const uint32_t u = fr[c + lane];
                    cur = a.rp[u];
                    end = a.rp[u + 1];
                }
                if (tau != 0xFFFFFFFFu) end = capw_clip(a.tcol, cur, end, tau);
                for (;;) {
                    const uint64_t r64 = end - cur;
                    const uint32_t rem = r64 > (1ull << 26) ? (1u << 26) : (uint32_t)r64;
                    const uint32_t incl = warp_incl_scan(rem, lane);
                    const uint32_t tot = __shfl_sync(0xFFFFFFFFu, incl, 31);
                    if (tot == 0) break;
                    const uint32_t excl = incl - rem;
                    const uint32_t take = min(tot, BUF - mm);
                    for (uint32_t x0 = 0; x0 < take; x0 += 32) {
                        const uint32_t x = x0 + lane;
                        uint32_t lo = 0, hi = 32;
                        while (hi - lo > 1) {
                            const uint32_t mid = (lo + hi) >> 1;
                            if (__shfl_sync(0xFFFFFFFFu, excl, mid) <= x) lo = mid; else hi = mid;
                        }
                        const uint64_t so = __shfl_sync(0xFFFFFFFFu, cur, lo);
                        const uint32_t eo = __shfl_sync(0xFFFFFFFFu, excl, lo);
                        uint32_t key = 0xFFFFFFFFu;
                        if (x < take) {
                            const uint32_t tv = a.tcol[so + (x - eo)];
                            if (tv != trow && tv < tau) key = (tv << 4) | (d - 1);
                        }
                        const uint32_t keep = __ballot_sync(0xFFFFFFFFu, key != 0xFFFFFFFFu);
                        if (key != 0xFFFFFFFFu) buf[mm + __popc(keep & lanemask_lt())] = key;
                        mm += __popc(keep);
                        __syncwarp();
                    }
                    cur += min(rem, take > excl ? take - excl : 0u);
                    if (take < tot) {  // the buffer is full
                        mm = capw_flush(buf, mm, lower, C, d - 1, lane, &tau);
                        if (tau != 0xFFFFFFFFu) end = capw_clip(a.tcol, cur, end, tau);
                    }
                }
            }
            m = capw_flush(buf, mm, lower, C, d - 1, lane, &tau);
            if (m == lower) break;  // no new node: nothing further either
        }
        // the kept nodes in id order
        for (uint32_t x = lane; x < m; x += 32) buf[x] = (id_of_tie(buf[x] >> 4) << 4) | (buf[x] & 15u);
        __syncwarp();
        warp_bitonic(buf, m, lane);
        uint64_t base = 0;
        int skip = 0;
        if (lane == 0) {
            a.counts[row] = m;
            if (a.staged) {
                const uint64_t span = ((uint64_t)m + 15) & ~15ull;
                base = atomicAdd(a.cursor, (unsigned long long)span);
                if (base + span > a.cap) {
                    skip = 1;
                    atomicExch(a.overflow, 1u);
                }
                a.row_off[row] = base;
            } else {
                base = a.gd_rp[row];
            }
        }
        base = __shfl_sync(0xFFFFFFFFu, base, 0);
        skip = __shfl_sync(0xFFFFFFFFu, skip, 0);
        if (!skip) {
            for (uint32_t x = lane; x < m; x += 32) {
                a.out_col[base + x] = buf[x] >> 4;
                a.out_dist[base + x] = (uint8_t)((buf[x] & 15u) + 1);
            }
        }
        __syncwarp();
    }
}

// Keys (row << 28 | tie(v)) of the adjacency entries, for the tie-ordered copy.
__global__ void k_tie_keys(const uint32_t* __restrict__ esrc, const uint32_t* __restrict__ col, uint64_t m,
                           uint64_t* __restrict__ keys) {
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < m; e += (uint64_t)gridDim.x * blockDim.x)
        keys[e] = ((uint64_t)esrc[e] << 28) | tie_of(col[e]);
}

__global__ void k_tie_values(const uint64_t* __restrict__ keys, uint64_t m, uint32_t* __restrict__ t) {
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < m; e += (uint64_t)gridDim.x * blockDim.x)
        t[e] = (uint32_t)keys[e] & kTieMask;
}

// The two shapes: caps up to 480 (1024-key buffers, 8 warps per block) and up
// to 2016 (4096-key buffers, 4 warps per block).
constexpr uint32_t CAPW_MAX_SMALL = 1024 / 2 - 32, CAPW_MAX = 4096 / 2 - 32;

static void launch_cap_rows(drg_ctx* ctx, const BfsArgs& a) {
    auto run = [&](auto kern, uint32_t buf, int warps) {
        const size_t smem = (size_t)warps * (buf + buf / 2) * 4;
        DRG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int per = 0;
        DRG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, warps * 32, smem));
        DRG_LAUNCH(ctx, kern, (uint32_t)ctx->num_sms * (uint32_t)(per > 0 ? per : 1), warps * 32, smem, a);
    };
    if (a.row_cap <= CAPW_MAX_SMALL) run(k_cap_rows<1024, 8>, 1024, 8);
    else run(k_cap_rows<4096, 4>, 4096, 4);
}

// Splits the rows into those of at most SMALL_CAP candidates (small) and the
// rest (big), as two lists (in no particular order).
__global__ void k_bfs_classify(const uint64_t* __restrict__ rp, const uint32_t* __restrict__ col, uint32_t n,
                               uint32_t* __restrict__ small, uint32_t* __restrict__ big,
                               uint32_t* __restrict__ counters) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warp0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t i = warp0; i < n; i += nwarps) {
        const uint64_t ab = rp[i], ae = rp[i + 1];
        uint64_t w = 0;
        for (uint64_t x = ab + lane; x < ae; x += 32) {
            const uint32_t u = col[x];
            w += rp[u + 1] - rp[u];
        }
#pragma unroll
        for (int off = 16; off; off >>= 1) w += __shfl_xor_sync(0xFFFFFFFFu, w, off);
        w += ae - ab;
        if (lane == 0) {
            if (w <= SMALL_CAP) small[atomicAdd(&counters[0], 1u)] = (uint32_t)i;
            else big[atomicAdd(&counters[1], 1u)] = (uint32_t)i;
        }
    }
}

// Moves staged rows to their final place, one warp per row.  A staged row
// starts at a multiple of 16 entries; the destination does not, so each
// lane writes aligned 16-byte groups of the destination, assembled from two
// aligned 16-byte loads of the source shifted by the row's phase (the same
// for every group of a row).  Head and tail entries are copied one by one.
__device__ __forceinline__ uint32_t pick4(uint4 a, uint4 b, uint32_t k) {
    switch (k) {
        case 0: return a.x;
        case 1: return a.y;
        case 2: return a.z;
        case 3: return a.w;
        case 4: return b.x;
        case 5: return b.y;
        case 6: return b.z;
        default: return b.w;
    }
}

__global__ void k_unstage(const uint64_t* __restrict__ row_off, const uint64_t* __restrict__ rp, uint32_t n,
                          const uint32_t* __restrict__ scol, const uint8_t* __restrict__ sdist,
                          uint32_t* __restrict__ col, uint8_t* __restrict__ dist) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warp0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t r = warp0; r < n; r += nwarps) {
        const uint64_t src = row_off[r], dst = rp[r], cnt = rp[r + 1] - dst;
        // columns: groups of 4 entries
        {
            const uint64_t head = ((4 - (dst & 3)) & 3) < cnt ? ((4 - (dst & 3)) & 3) : cnt;
            const uint64_t groups = (cnt - head) / 4;
            const uint64_t done = head + 4 * groups;
            if (lane < head) col[dst + lane] = scol[src + lane];
            if (lane < cnt - done) col[dst + done + lane] = scol[src + done + lane];
            const uint32_t ph = (uint32_t)((src + head) & 3);
            for (uint64_t g = lane; g < groups; g += 32) {
                const uint64_t sx = src + head + 4 * g, al = sx & ~3ull;
                const uint4 a = __ldg(reinterpret_cast<const uint4*>(scol + al));
                const uint4 b = ph ? __ldg(reinterpret_cast<const uint4*>(scol + al + 4)) : a;
                *reinterpret_cast<uint4*>(col + dst + head + 4 * g) =
                    make_uint4(pick4(a, b, ph), pick4(a, b, ph + 1), pick4(a, b, ph + 2), pick4(a, b, ph + 3));
            }
        }
        // distances: groups of 16 bytes
        {
            const uint64_t head = ((16 - (dst & 15)) & 15) < cnt ? ((16 - (dst & 15)) & 15) : cnt;
            const uint64_t groups = (cnt - head) / 16;
            const uint64_t done = head + 16 * groups;
            if (lane < head) dist[dst + lane] = sdist[src + lane];
            if (lane < cnt - done) dist[dst + done + lane] = sdist[src + done + lane];
            const uint32_t ph = (uint32_t)((src + head) & 15), wsh = ph >> 2, bsh = 8 * (ph & 3);
            for (uint64_t g = lane; g < groups; g += 32) {
                const uint64_t sx = src + head + 16 * g, al = sx & ~15ull;
                const uint4 a = __ldg(reinterpret_cast<const uint4*>(sdist + al));
                const uint4 b = ph ? __ldg(reinterpret_cast<const uint4*>(sdist + al + 16)) : a;
                uint32_t o[4];
#pragma unroll
                for (uint32_t k = 0; k < 4; ++k)
                    o[k] = __funnelshift_r(pick4(a, b, wsh + k), pick4(a, b, wsh + k + 1), bsh);
                *reinterpret_cast<uint4*>(dist + dst + head + 16 * g) = make_uint4(o[0], o[1], o[2], o[3]);
            }
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

// The distance array is padded to whole 16-byte words: k_row_Z reads rows in
// aligned 16-byte pieces (bytes outside the row are masked).
static size_t dist_bytes(uint64_t nnz) { return (size_t)((nnz + 15) / 16 + 1) * 16; }

static void build_korder(drg_ctx* ctx, const drg_graph* g, uint32_t k, drg_dmat* d, uint32_t row_cap) {
    const uint32_t n = g->n;
    // a cap that no row can reach (n - 1 nodes besides the source) keeps every row whole
    if (row_cap && (uint64_t)row_cap >= (uint64_t)(n > 0 ? n - 1 : 0)) row_cap = 0;
    if (row_cap) {
        DRG_CHECK(n <= (1u << 28), DRG_EUNSUPPORTED, "capped rows need fewer than 2^28 nodes");
        DRG_CHECK(row_cap <= CAPW_MAX, DRG_EUNSUPPORTED, "a row cap above 2016 (and below n - 1) is not supported");
    }
    d->rp = static_cast<uint64_t*>(dalloc(ctx, sizeof(uint64_t) * ((size_t)n + 1)));
    if (k == 1 && row_cap == 0) {
        // NNG(v_i, 1) is the adjacency itself, already sorted by column
        d->nnz = g->nnz;
        d->col = static_cast<uint32_t*>(dalloc(ctx, sizeof(uint32_t) * (d->nnz ? d->nnz : 1)));
        d->dist = static_cast<uint8_t*>(dalloc(ctx, dist_bytes(d->nnz)));
        d2d(ctx, d->rp, g->rp, (size_t)n + 1);
        d2d(ctx, d->col, g->col, d->nnz);
        DRG_LAUNCH(ctx, k_fill_u8, grid_for(d->nnz, 256, 65536), 256, 0, d->dist, d->nnz, (uint8_t)1);
        return;
    }
    const bool k2 = k == 2 && row_cap == 0;
    const uint32_t words = (n + 31) / 32;
    const uint32_t swords = (words + 31) / 32;
    const size_t bm_bytes = (size_t)words * 4, extra = bfs_extra_smem(swords);
    const bool smem_bm = bm_bytes + extra + 16384 <= (size_t)ctx->max_smem_optin;
    DRG_CHECK(extra + 16384 <= (size_t)ctx->max_smem_optin, DRG_EUNSUPPORTED, "graph too large for the BFS");
    const size_t dyn = (smem_bm ? bm_bytes : 0) + extra;
    // 512-thread blocks when three of them fit an SM's shared memory, else 1024
    const bool small_blocks = 3 * (dyn + 8 * 1024) <= (size_t)ctx->max_smem_optin;
    const int bfs_threads = small_blocks ? BFS_THREADS_SMALL : BFS_THREADS_BIG;
    auto kern = k2 ? (small_blocks ? k_bfs<true, BFS_THREADS_SMALL> : k_bfs<true, BFS_THREADS_BIG>)
                   : (small_blocks ? k_bfs<false, BFS_THREADS_SMALL> : k_bfs<false, BFS_THREADS_BIG>);
    // The limit is process-wide per kernel and graphs differ in size (and may
    // be built by several host threads at once): allow the kernel's maximum
    // always; each launch passes its own size, which sets the occupancy.
    {
        cudaFuncAttributes fa;
        DRG_CUDA(cudaFuncGetAttributes(&fa, kern));
        DRG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      ctx->max_smem_optin - (int)fa.sharedSizeBytes));
    }
    int per_sm = 0;
    DRG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, bfs_threads, dyn));
    if (per_sm < 1) per_sm = 1;
    uint32_t blocks = (uint32_t)ctx->num_sms * (uint32_t)per_sm;
    if (blocks > n) blocks = n;
    // per-block discovered lists, touched words, word offsets / hop distances
    // (and bitmaps when they live in global memory); capped rows use none
    const size_t per_block = row_cap ? 0 : (size_t)blocks;
    DBuf<uint32_t> lists(ctx, per_block * n);
    DBuf<uint32_t> wlists(ctx, per_block * words);
    DBuf<uint8_t> dlev(ctx, k2 ? 1 : per_block * n);
    DBuf<uint32_t> gbm(ctx, smem_bm ? 1 : per_block * words);
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
    if (row_cap) cap = std::min<uint64_t>(cap, (uint64_t)n * row_cap);  // no row holds more
    if (cap > 0xFFFFFFFFull) cap = 0xFFFFFFFFull;
    cap += 16ull * n;  // each staged row is padded to a multiple of 16 entries
    if (ctx->bfs_stage_limit >= 0 && (uint64_t)ctx->bfs_stage_limit < cap) cap = (uint64_t)ctx->bfs_stage_limit;
    DBuf<uint32_t> scol;
    DBuf<uint8_t> sdist;
    try {
        // 32 spare entries: the aligned copies read up to one group past a row
        scol = DBuf<uint32_t>(ctx, cap + 32);
        sdist = DBuf<uint8_t>(ctx, cap + 32);
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
    a.rows = nullptr; a.nrows = n;
    a.gbitmaps = smem_bm ? nullptr : gbm.p;
    a.lists = lists.p; a.wlists = wlists.p; a.dlev = dlev.p;
    a.next_row = counter.p; a.counts = counts.p;
    a.staged = 1; a.cursor = cursor.p; a.cap = cap; a.row_off = row_off.p; a.overflow = overflow.p;
    a.out_col = scol.p; a.out_dist = sdist.p;
    a.row_cap = row_cap;
    // capped rows read every row's adjacency as tie values, ascending: one
    // sort of the entries by (row, tie)
    DBuf<uint32_t> tcol;
    if (row_cap) {
        const uint64_t m = g->nnz;
        tcol = DBuf<uint32_t>(ctx, m);
        DBuf<uint32_t> esrc(ctx, m);
        DBuf<uint64_t> keys(ctx, m), kalt(ctx, m);
        DRG_LAUNCH(ctx, k_expand_rows, grid_for((size_t)n * 32, 256, (uint32_t)ctx->num_sms * 16), 256, 0, g->rp, n,
                   esrc.p);
        DRG_LAUNCH(ctx, k_tie_keys, grid_for(m, 256, 65536), 256, 0, esrc.p, g->col, m, keys.p);
        uint64_t* kp = keys.p;
        uint64_t* ap = kalt.p;
        uint32_t* vnull = nullptr;
        uint32_t* vnull2 = nullptr;
        radix_sort(ctx, kp, ap, vnull, vnull2, m, 0, 28 + std::max(1, bitlen(n > 1 ? n - 1 : 1)));
        DRG_LAUNCH(ctx, k_tie_values, grid_for(m, 256, 65536), 256, 0, kp, m, tcol.p);
        a.tcol = tcol.p;
    }
    DRG_CUDA(cudaMemsetAsync(counter.p, 0, 4, ctx->stream));
    DRG_CUDA(cudaMemsetAsync(overflow.p, 0, 4, ctx->stream));
    DRG_CUDA(cudaMemsetAsync(cursor.p, 0, 8, ctx->stream));
    {
        ProfSpan sb(ctx, DRG_PROF_BFS, 0, 3);
        DBuf<uint32_t> small, big;
        if (k2 && n < 0x80000000u && cap > 0) {  // keys v << 1 | 1 stay below 0xFFFFFFFF
            // k = 2: rows of few candidates by one warp each, the rest by blocks
            small = DBuf<uint32_t>(ctx, n);
            big = DBuf<uint32_t>(ctx, n);
            DBuf<uint32_t> ctr(ctx, 2);
            DRG_CUDA(cudaMemsetAsync(ctr.p, 0, 8, ctx->stream));
            DRG_LAUNCH(ctx, k_bfs_classify, grid_for((size_t)n * 32, 256, (uint32_t)ctx->num_sms * 16), 256, 0, g->rp,
                       g->col, n, small.p, big.p, ctr.p);
            uint32_t nc[2];
            d2h(ctx, nc, ctr.p, 2);
            sync(ctx);
            const size_t ssm = (size_t)SMALL_WARPS * SMALL_CAP * 4;
            DRG_CUDA(cudaFuncSetAttribute(k_bfs_small, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ssm));
            int sper = 0;
            DRG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&sper, k_bfs_small, SMALL_WARPS * 32, ssm));
            BfsArgs as = a;
            as.rows = small.p;
            as.nrows = nc[0];
            DRG_LAUNCH(ctx, k_bfs_small, (uint32_t)ctx->num_sms * (uint32_t)(sper > 0 ? sper : 1), SMALL_WARPS * 32,
                       ssm, as);
            DRG_CUDA(cudaMemsetAsync(counter.p, 0, 4, ctx->stream));
            a.rows = big.p;
            a.nrows = nc[1];
        } else if (row_cap) {
            // capped rows: every row by one warp, on the tie-ordered adjacency
            launch_cap_rows(ctx, a);
            a.nrows = 0;
        }
        if (a.nrows) DRG_LAUNCH(ctx, kern, blocks, bfs_threads, dyn, a);
    }
    DBuf<uint64_t> tot(ctx, 1);
    scan<uint64_t>(ctx, LoadArr<uint64_t>{counts.p}, n, d->rp, false, tot.p);
    d2d(ctx, d->rp + n, tot.p, 1);
    d->nnz = read1(ctx, tot.p);
    DRG_CHECK(d->nnz < (1ull << 32), DRG_EUNSUPPORTED, "distance matrix has 2^32 entries or more");
    const bool overflowed = read1(ctx, overflow.p) != 0;
    d->col = static_cast<uint32_t*>(dalloc(ctx, sizeof(uint32_t) * (d->nnz ? d->nnz : 1)));
    d->dist = static_cast<uint8_t*>(dalloc(ctx, dist_bytes(d->nnz)));
    if (!overflowed) {
        DRG_LAUNCH(ctx, k_unstage, grid_for((size_t)n * 32, 256, (uint32_t)ctx->num_sms * 16), 256, 0, row_off.p,
                   d->rp, n, scol.p, sdist.p, d->col, d->dist);
        return;
    }
    // the staging area was too small: traverse again, writing at the final offsets
    scol.reset();
    sdist.reset();
    a.staged = 0;
    a.rows = nullptr;
    a.nrows = n;
    a.gd_rp = d->rp;
    a.out_col = d->col;
    a.out_dist = d->dist;
    DRG_CUDA(cudaMemsetAsync(counter.p, 0, 4, ctx->stream));
    ProfSpan sb(ctx, DRG_PROF_BFS, 0);
    if (row_cap) launch_cap_rows(ctx, a);
    else DRG_LAUNCH(ctx, kern, blocks, bfs_threads, dyn, a);
}

struct Gauss {
    float g[16];
};

// ------------------------------------------------------------------ row cap: the union pattern
// Kept rows K (each row's row_cap nearest nodes, sorted by (row, column)) ->
// the sampling pattern K u K^T, sorted by (row, column); each entry carries
// flag 1 (j in K_i, "own") and / or flag 2 (i in K_j, "back").  T = K^T is
// K's entries sorted stably by their column, so T_i lists, in ascending j,
// the rows j that kept i.  A pair kept on both sides appears once in K_i and
// once in T_i ("dup"); row i of the union is K_i merged with T_i \ K_i, and
// the place of each entry in it is the count of union entries below it:
//   j in K_i at index a:       a + #{T_i < j} - #{dups of K_i before a}
//   j in T_i \ K_i at index b: b + #{K_i < j} - #{dups of K_i below j}

// T's keys: row j of the transposed entry in the low 32 bits, hop distance
// above; values: the column (= the kept row's source).
__global__ void k_cap_transpose(const uint32_t* __restrict__ esrc, const uint32_t* __restrict__ col,
                                const uint8_t* __restrict__ dist, uint64_t nK, uint64_t* __restrict__ tkey,
                                uint32_t* __restrict__ tval) {
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < nK; e += (uint64_t)gridDim.x * blockDim.x) {
        tkey[e] = (uint64_t)col[e] | ((uint64_t)dist[e] << 32);
        tval[e] = esrc[e];
    }
}

// Row pointers of keys sorted by row (low 32 bits): the first entry of each
// row writes the pointers of the rows after the previous entry's row up to
// its own, the last entry those of the rows after it.
__global__ void k_rows_of_sorted(const uint64_t* __restrict__ key, uint64_t m, uint32_t n, uint32_t* __restrict__ rp) {
    for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < m; x += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t i = (uint32_t)key[x];
        if (x + 1 == m)
            for (uint64_t t = i + 1; t <= n; ++t) rp[t] = (uint32_t)m;
        const uint64_t from = x == 0 ? 0 : (uint64_t)(uint32_t)key[x - 1] + 1;
        for (uint64_t t = from; t <= i; ++t) rp[t] = (uint32_t)x;
    }
}

// First index in [lo, hi) of a sorted u32 array holding a value >= v.
__device__ __forceinline__ uint64_t lower_bound_u32(const uint32_t* __restrict__ a, uint64_t lo, uint64_t hi,
                                                    uint32_t v) {
    while (lo < hi) {
        const uint64_t mid = (lo + hi) >> 1;
        if (a[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// For each entry e = (i, j) of K: tlo[e] = #{T_i < j} and dup[e] = (j in T_i).
__global__ void k_cap_dups(const uint64_t* __restrict__ rpK, const uint32_t* __restrict__ esrc,
                           const uint32_t* __restrict__ col, const uint32_t* __restrict__ rpT,
                           const uint32_t* __restrict__ tval, uint64_t nK, uint32_t* __restrict__ tlo,
                           uint32_t* __restrict__ dup) {
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < nK; e += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t i = esrc[e], j = col[e];
        const uint64_t t0 = rpT[i], t1 = rpT[i + 1];
        const uint64_t lb = lower_bound_u32(tval, t0, t1, j);
        tlo[e] = (uint32_t)(lb - t0);
        dup[e] = (lb < t1 && tval[lb] == j) ? 1u : 0u;
    }
}

// Union row sizes |K_i| + |T_i| - dups_i (dpre: exclusive prefix of dup over
// K, with the total at index nK).
__global__ void k_cap_rowsize(const uint64_t* __restrict__ rpK, const uint32_t* __restrict__ rpT,
                              const uint32_t* __restrict__ dpre, uint32_t n, uint64_t* __restrict__ cnt) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        cnt[i] = (rpK[i + 1] - rpK[i]) + (rpT[i + 1] - rpT[i]) - (dpre[rpK[i + 1]] - dpre[rpK[i]]);
}

__global__ void k_cap_write_own(const uint64_t* __restrict__ rpK, const uint32_t* __restrict__ esrc,
                                const uint32_t* __restrict__ col, const uint8_t* __restrict__ dist,
                                const uint32_t* __restrict__ tlo, const uint32_t* __restrict__ dup,
                                const uint32_t* __restrict__ dpre, const uint64_t* __restrict__ rpU, uint64_t nK,
                                uint32_t* __restrict__ ucol, uint8_t* __restrict__ udist, uint8_t* __restrict__ uflag) {
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < nK; e += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t i = esrc[e];
        const uint64_t k0 = rpK[i];
        const uint64_t p = rpU[i] + (e - k0) + tlo[e] - (dpre[e] - dpre[k0]);
        ucol[p] = col[e];
        udist[p] = dist[e];
        uflag[p] = (uint8_t)(1u | (dup[e] << 1));
    }
}

__global__ void k_cap_write_back(const uint64_t* __restrict__ rpK, const uint32_t* __restrict__ col,
                                 const uint32_t* __restrict__ rpT, const uint64_t* __restrict__ tkey,
                                 const uint32_t* __restrict__ tval, const uint32_t* __restrict__ dpre,
                                 const uint64_t* __restrict__ rpU, uint64_t nK, uint32_t* __restrict__ ucol,
                                 uint8_t* __restrict__ udist, uint8_t* __restrict__ uflag) {
    for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < nK; x += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t key = tkey[x];
        const uint32_t i = (uint32_t)key, j = tval[x];
        const uint64_t k0 = rpK[i], k1 = rpK[i + 1];
        const uint64_t ub = lower_bound_u32(col, k0, k1, j);
        if (ub < k1 && col[ub] == j) continue;  // kept by both: written as i's own entry
        const uint64_t p = rpU[i] + (x - rpT[i]) + (ub - k0) - (dpre[ub] - dpre[k0]);
        ucol[p] = j;
        udist[p] = (uint8_t)(key >> 32);
        uflag[p] = 2u;
    }
}

// Z_i of the kept set K_i: sum over d = 1..k of fl32(count of own entries at
// distance d) * g(d), in that order, FP32 correctly rounded, no fused
// multiply-add (one warp per row).
__global__ void k_row_Z_own(const uint64_t* __restrict__ rp, const uint8_t* __restrict__ dist,
                            const uint8_t* __restrict__ flag, uint32_t n, uint32_t k, Gauss gs, float* __restrict__ Z) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t i = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; i < n; i += nw) {
        uint32_t cnt[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) cnt[c] = 0;
        for (uint64_t e = rp[i] + lane; e < rp[i + 1]; e += 32) {
            if (!(flag[e] & 1u)) continue;
            const uint32_t dd = dist[e];
#pragma unroll
            for (int c = 0; c < 16; ++c) cnt[c] += (dd == (uint32_t)(c + 1)) ? 1u : 0u;
        }
        float z = 0.f;
        for (uint32_t c = 0; c < k; ++c) {
            uint32_t t = cnt[c];
#pragma unroll
            for (int off = 16; off; off >>= 1) t += __shfl_xor_sync(0xFFFFFFFFu, t, off);
            z = __fadd_rn(z, __fmul_rn((float)t, gs.g[c]));
        }
        if (lane == 0) Z[i] = z;
    }
}

// ------------------------------------------------------------------ similarity

// Bytes [lo, hi) of a 16-byte piece, as a mask per 32-bit word q.
__device__ __forceinline__ uint32_t byte_mask(uint32_t q, uint32_t lo, uint32_t hi) {
    const uint32_t b0 = 4 * q;
    const uint32_t a = lo > b0 ? (lo - b0 < 4 ? lo - b0 : 4) : 0;   // bytes cut at the front
    const uint32_t e = hi > b0 ? (hi - b0 < 4 ? hi - b0 : 4) : 0;   // bytes kept up to here
    const uint64_t keep_hi = (1ull << (8 * e)) - 1;
    const uint64_t cut_lo = (1ull << (8 * a)) - 1;
    return (uint32_t)(keep_hi & ~cut_lo);
}

// Z_i = sum over d = 1..k of count_i(d) * g(d), in that order, FP32
// correctly rounded with no fused multiply-add.  One warp per row; each lane
// reads aligned 16-byte pieces of the row's distances and counts the bytes
// of each class with byte-wise compares.
// With COUNTS the row's class counts go to cnt[i k + d - 1] instead (the
// perplexity calibration needs them, not Z).
template <bool COUNTS>
__global__ void k_row_Z(const uint64_t* __restrict__ rp, const uint8_t* __restrict__ dist, uint32_t n, uint32_t k,
                        Gauss gs, float* __restrict__ Z, uint32_t* __restrict__ cnt) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warp0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t i = warp0; i < n; i += nwarps) {
        uint32_t c[15];
#pragma unroll
        for (int d = 0; d < 15; ++d) c[d] = 0;
        const uint64_t e0 = rp[i], e1 = rp[i + 1];
        for (uint64_t b = (e0 & ~15ull) + 16 * lane; b < e1; b += 512) {
            const uint4 v = *reinterpret_cast<const uint4*>(dist + b);
            const uint32_t lo = b < e0 ? (uint32_t)(e0 - b) : 0u;
            const uint32_t hi = e1 - b < 16 ? (uint32_t)(e1 - b) : 16u;
            const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint32_t m = byte_mask(q, lo, hi);
#pragma unroll
                for (int d = 0; d < 15; ++d)
                    if ((uint32_t)d < k) c[d] += __popc(__vcmpeq4(w[q], (uint32_t)(d + 1) * 0x01010101u) & m) >> 3;
            }
        }
        float z = 0.f;
#pragma unroll
        for (int d = 0; d < 15; ++d) {
            if ((uint32_t)d < k) {
                uint32_t t = c[d];
#pragma unroll
                for (int off = 16; off; off >>= 1) t += __shfl_xor_sync(0xFFFFFFFFu, t, off);
                if (COUNTS) {
                    if (lane == 0) cnt[i * k + d] = t;
                } else {
                    z = __fadd_rn(z, __fmul_rn(__uint2float_rn(t), gs.g[d]));
                }
            }
        }
        if (!COUNTS && lane == 0) Z[i] = z;
    }
}

// ------------------------------------------------------------------ perplexity calibration
// Eq. 9's sigma_i per node by the perplexity rule: row i holds c_d nodes at
// hop distance d; with beta = 1/(2 sigma_i^2) and w_d = e^{-beta (d^2 - 1)},
// exp(H_i) = Z' exp(beta S'/Z') (Z' = sum c_d w_d, S' = sum c_d (d^2 - 1) w_d)
// falls from the row size to c_1 as beta grows; 60 bisection steps on
// [0, 512] give beta_i.  All FP64 with separately rounded operations and the
// exponential below, so beta_i is a fixed function of the counts; then
// g_i(d) = fl32(e^{-beta_i (d^2 - 1)}), Z_i as for a global sigma, and the
// per-node table W_i(d) = fl32(g_i(d) / Z_i) that the quantisation reads.
struct ExpPoly {
    double c[14];  // 1/n!, n = 0..13
};

// e^x: Cody & Waite's reduction x = m ln2 + r (ln 2 as a 32-significant-bit
// head and a tail, so m * head is exact), degree-13 Taylor polynomial of e^r
// by Horner's rule, times 2^m from its bits; 0 below -700.
__device__ __forceinline__ double cal_exp(double x, const ExpPoly& P) {
    if (x < -700.0) return 0.0;
    const double m = floor(__dadd_rn(__dmul_rn(x, 1.4426950408889634), 0.5));
    const double r = __dsub_rn(__dsub_rn(x, __dmul_rn(m, 0.6931471803691238)), __dmul_rn(m, 1.9082149292705877e-10));
    double p = P.c[13];
#pragma unroll
    for (int i = 12; i >= 0; --i) p = __dadd_rn(__dmul_rn(p, r), P.c[i]);
    const double scale = __longlong_as_double((long long)((int)m + 1023) << 52);
    return __dmul_rn(p, scale);
}

__device__ __forceinline__ double cal_perplexity(const uint32_t* c, uint32_t k, double beta, const ExpPoly& P) {
    double z = 0.0, s = 0.0;
    for (uint32_t d = 1; d <= k; ++d) {
        const double dd = (double)(d * d - 1);
        const double w = cal_exp(-__dmul_rn(beta, dd), P);
        const double cd = (double)c[d - 1];
        z = __dadd_rn(z, __dmul_rn(cd, w));
        s = __dadd_rn(s, __dmul_rn(__dmul_rn(cd, dd), w));
    }
    return __dmul_rn(z, cal_exp(__dmul_rn(beta, __ddiv_rn(s, z)), P));
}

// One thread per node: beta_i, Z_i and W_i(1..k) (all zero for an empty row).
__global__ void k_calibrate(const uint32_t* __restrict__ cnt, uint32_t n, uint32_t k, double perplexity, ExpPoly P,
                            double* __restrict__ beta, float* __restrict__ Z, float* __restrict__ W) {
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t c[15];
        uint64_t size = 0;
        for (uint32_t d = 0; d < k; ++d) {
            c[d] = cnt[v * k + d];
            size += c[d];
        }
        if (size == 0) {
            beta[v] = 0.0;
            Z[v] = 0.f;
            for (uint32_t d = 0; d < k; ++d) W[v * k + d] = 0.f;
            continue;
        }
        double lo = 0.0, hi = 512.0;
        for (int it = 0; it < 60; ++it) {
            const double mid = __dmul_rn(__dadd_rn(lo, hi), 0.5);
            if (cal_perplexity(c, k, mid, P) > perplexity) lo = mid;
            else hi = mid;
        }
        const double b = __dmul_rn(__dadd_rn(lo, hi), 0.5);
        beta[v] = b;
        float g[15];
        float z = 0.f;
        for (uint32_t d = 1; d <= k; ++d) {
            g[d - 1] = __double2float_rn(cal_exp(-__dmul_rn(b, (double)(d * d - 1)), P));
            z = __fadd_rn(z, __fmul_rn(__uint2float_rn(c[d - 1]), g[d - 1]));
        }
        Z[v] = z;
        for (uint32_t d = 0; d < k; ++d) W[v * k + d] = __fdiv_rn(g[d], z);
    }
}

// q_e = floor((fl(g/Z_i) + fl(g/Z_j)) * 2^30).
__device__ __forceinline__ uint32_t quantise1(float gd, float zi, float zj) {
    const float s = __fadd_rn(__fdiv_rn(gd, zi), __fdiv_rn(gd, zj));
    return __float2uint_rz(__fmul_rn(s, 1073741824.0f));
}

// q for every entry, 4 consecutive entries per thread, and the row sums r_i
// = sum of the row's q (exact): along the entries the rows never decrease,
// so a thread adds any run of its own entries that ends inside its four, and
// the warp sums the open runs by row (segmented suffix sums over the lanes)
// and adds each row's total with one atomic.  r must start at zero.
// Kinds: Q_GLOBAL_SIGMA uses g(d) / Z; Q_PER_NODE takes the two conditional
// similarities from the calibrated per-node table W (fl32(g_i(d) / Z_i),
// row-major n x k); Q_CAPPED (the union of kept rows) takes fl32(g/Z_i) only
// where the entry's flag has bit 1 (j in K_i) and fl32(g/Z_j) only where it
// has bit 2 (i in K_j), each else 0.
enum { Q_GLOBAL_SIGMA = 0, Q_PER_NODE = 1, Q_CAPPED = 2 };
template <int KIND>
__global__ void k_quantise_r(const uint32_t* __restrict__ esrc, const uint32_t* __restrict__ col,
                             const uint8_t* __restrict__ dist, const float* __restrict__ Z, Gauss gs, uint64_t nnz,
                             uint32_t* __restrict__ q, unsigned long long* __restrict__ r,
                             const float* __restrict__ W, uint32_t k, const uint8_t* __restrict__ flag) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t nv = (nnz + 3) / 4;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t w0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x - lane; w0 < nv; w0 += stride) {
        const uint64_t v = w0 + lane;
        uint32_t key = 0xFFFFFFFFu;
        unsigned long long sum = 0;
        if (v < nv) {
            const uint64_t e = 4 * v;
            const uint32_t cnt = nnz - e < 4 ? (uint32_t)(nnz - e) : 4u;
            uint32_t ii[4], jj[4], dd[4], ff[4], qq[4];
            if (cnt == 4) {
                const uint4 a4 = __ldg(reinterpret_cast<const uint4*>(esrc + e));
                const uint4 b4 = __ldg(reinterpret_cast<const uint4*>(col + e));
                const uint32_t dw = __ldg(reinterpret_cast<const uint32_t*>(dist + e));
                const uint32_t fw = KIND == Q_CAPPED ? __ldg(reinterpret_cast<const uint32_t*>(flag + e)) : 0u;
                ii[0] = a4.x; ii[1] = a4.y; ii[2] = a4.z; ii[3] = a4.w;
                jj[0] = b4.x; jj[1] = b4.y; jj[2] = b4.z; jj[3] = b4.w;
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    dd[t] = (dw >> (8 * t)) & 0xFFu;
                    ff[t] = (fw >> (8 * t)) & 0xFFu;
                }
            } else {
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const bool ok = (uint32_t)t < cnt;
                    ii[t] = ok ? esrc[e + t] : 0u;
                    jj[t] = ok ? col[e + t] : 0u;
                    dd[t] = ok ? dist[e + t] : 1u;
                    ff[t] = (KIND == Q_CAPPED && ok) ? flag[e + t] : 0u;
                }
            }
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                if (KIND == Q_PER_NODE) {
                    const float s = __fadd_rn(W[(uint64_t)ii[t] * k + dd[t] - 1], W[(uint64_t)jj[t] * k + dd[t] - 1]);
                    qq[t] = __float2uint_rz(__fmul_rn(s, 1073741824.0f));
                } else if (KIND == Q_CAPPED) {
                    const float g = gs.g[dd[t] - 1];
                    const float av = (ff[t] & 1u) ? __fdiv_rn(g, Z[ii[t]]) : 0.f;
                    const float bv = (ff[t] & 2u) ? __fdiv_rn(g, Z[jj[t]]) : 0.f;
                    qq[t] = __float2uint_rz(__fmul_rn(__fadd_rn(av, bv), 1073741824.0f));
                } else {
                    qq[t] = quantise1(gs.g[dd[t] - 1], Z[ii[t]], Z[jj[t]]);
                }
            }
            if (cnt == 4) {
                *reinterpret_cast<uint4*>(q + e) = make_uint4(qq[0], qq[1], qq[2], qq[3]);
            } else {
                for (uint32_t t = 0; t < cnt; ++t) q[e + t] = qq[t];
            }
            key = ii[0];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                if ((uint32_t)t >= cnt) break;
                if (ii[t] != key) {
                    atomicAdd(&r[key], sum);
                    key = ii[t];
                    sum = 0;
                }
                sum += qq[t];
            }
        }
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t ok = __shfl_down_sync(0xFFFFFFFFu, key, off);
            const unsigned long long ov = __shfl_down_sync(0xFFFFFFFFu, sum, off);
            if (lane + off < 32 && ok == key) sum += ov;
        }
        const uint32_t pk = __shfl_up_sync(0xFFFFFFFFu, key, 1);
        if (key != 0xFFFFFFFFu && (lane == 0 || pk != key)) atomicAdd(&r[key], sum);
    }
}

__global__ void k_rmax(const uint64_t* __restrict__ r, uint32_t n, unsigned long long* __restrict__ rmax) {
    unsigned long long m = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        m = r[i] > m ? r[i] : m;
#pragma unroll
    for (int off = 16; off; off >>= 1) {
        const unsigned long long o = __shfl_xor_sync(0xFFFFFFFFu, m, off);
        m = o > m ? o : m;
    }
    if ((threadIdx.x & 31) == 0 && m) atomicMax(rmax, m);
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
//
// One scan over the items in index order carries (lights so far, their
// deficit, the heavies' excess): its exclusive prefix at item i gives i's
// place in the light or heavy list and its Dl or S value, written straight
// into the lists.

// Running sums of the split scan: the lights' count and weight, the heavies'
// weight.  The deficits and excesses follow from them exactly, so the lists
// hold 64-bit weight prefixes instead of 128-bit mass sums:
//   Dl(x) = x W - N QL(x)          QL(x): weight of the lights before light x
//   S(y)  = N QH(y) - (y + 1) W    QH(y): weight of the heavies up to heavy y
struct SplitAcc {
    uint64_t QL, QH;  // lights' weight, heavies' weight
    uint64_t c;       // lights
    SplitAcc() = default;  // trivial, so that it can live in shared memory
    __host__ __device__ SplitAcc(int) : QL(0), QH(0), c(0) {}  // from 0
    __host__ __device__ SplitAcc& operator+=(const SplitAcc& o) {
        QL += o.QL;
        QH += o.QH;
        c += o.c;
        return *this;
    }
    __host__ __device__ SplitAcc operator+(const SplitAcc& o) const { SplitAcc r = *this; r += o; return r; }
    __host__ __device__ SplitAcc operator-(const SplitAcc& o) const {
        SplitAcc r = *this;
        r.QL -= o.QL;
        r.QH -= o.QH;
        r.c -= o.c;
        return r;
    }
};

__device__ __forceinline__ SplitAcc shfl_up(const SplitAcc& v, int d) {
    SplitAcc r;
    r.QL = shfl_up(v.QL, d);
    r.QH = shfl_up(v.QH, d);
    r.c = shfl_up(v.c, d);
    return r;
}

__device__ __forceinline__ SplitAcc split_item(uint32_t qi, uint64_t N, uint64_t W) {
    SplitAcc r(0);
    if ((uint64_t)qi * N < W) {
        r.QL = qi;
        r.c = 1;
    } else {
        r.QH = qi;
    }
    return r;
}

struct SplitLoad {
    const uint32_t* q;
    uint64_t N, W;
    __device__ __forceinline__ SplitAcc operator()(size_t i) const { return split_item(q[i], N, W); }
};

// Tiles of SPLIT_TILE items; the down pass walks a tile in SPLIT_SUB-item
// pieces (8 consecutive items per thread), one piece per tile.
constexpr int SPLIT_THREADS = 256, SPLIT_SUB = 2048, SPLIT_TILE = SPLIT_SUB;

__device__ __forceinline__ SplitAcc warp_sum(SplitAcc v) {
#pragma unroll
    for (int off = 16; off; off >>= 1) {
        SplitAcc o;
        o.QL = __shfl_xor_sync(0xFFFFFFFFu, v.QL, off);
        o.QH = __shfl_xor_sync(0xFFFFFFFFu, v.QH, off);
        o.c = __shfl_xor_sync(0xFFFFFFFFu, v.c, off);
        v += o;
    }
    return v;
}

// Per-tile sums: a block reads SPLIT_REDUCE_TILES tiles with 16-byte loads
// (8 items per thread and tile) and writes each tile's sum.
constexpr int SPLIT_REDUCE_TILES = 4;

__global__ void __launch_bounds__(SPLIT_THREADS, 6) k_split_reduce(const uint32_t* __restrict__ q, uint64_t N,
                                                                uint64_t W, uint64_t tiles,
                                                                SplitAcc* __restrict__ sums) {
    __shared__ SplitAcc wt[SPLIT_REDUCE_TILES][SPLIT_THREADS / 32];
    constexpr int R = SPLIT_TILE / 4 / SPLIT_THREADS;  // 16-byte loads per thread and tile
    SplitAcc acc[SPLIT_REDUCE_TILES];
#pragma unroll
    for (int p = 0; p < SPLIT_REDUCE_TILES; ++p) {
        acc[p] = SplitAcc(0);
        const uint64_t base = ((uint64_t)blockIdx.x * SPLIT_REDUCE_TILES + p) * SPLIT_TILE;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const uint64_t i = base + 4 * ((uint64_t)r * SPLIT_THREADS + threadIdx.x);
            if (i + 4 <= N) {
                const uint4 v = __ldg(reinterpret_cast<const uint4*>(q + i));
                acc[p] += split_item(v.x, N, W);
                acc[p] += split_item(v.y, N, W);
                acc[p] += split_item(v.z, N, W);
                acc[p] += split_item(v.w, N, W);
            } else {
                for (uint64_t t = i; t < N && t < i + 4; ++t) acc[p] += split_item(q[t], N, W);
            }
        }
    }
#pragma unroll
    for (int p = 0; p < SPLIT_REDUCE_TILES; ++p) {
        const SplitAcc w = warp_sum(acc[p]);
        if ((threadIdx.x & 31) == 0) wt[p][threadIdx.x >> 5] = w;
    }
    __syncthreads();
    if (threadIdx.x < SPLIT_REDUCE_TILES) {
        const uint64_t tile = (uint64_t)blockIdx.x * SPLIT_REDUCE_TILES + threadIdx.x;
        SplitAcc t(0);
        for (int w = 0; w < SPLIT_THREADS / 32; ++w) t += wt[threadIdx.x][w];
        if (tile < tiles) sums[tile] = t;
    }
}

// Lists, in index order: light x is item L[x] with QL[x] = weight of the
// lights before it; heavy y is item H[y] with QH[y] = weight of the heavies
// up to and including it.  Each piece's lights and heavies are gathered in
// shared memory (lights first) and written out in order.
constexpr size_t SPLIT_DOWN_SMEM = (size_t)SPLIT_SUB * (4 + 8);

__global__ void __launch_bounds__(SPLIT_THREADS) k_split_down(const uint32_t* __restrict__ q, uint64_t N, uint64_t W,
                                                              const SplitAcc* __restrict__ tile_pre,
                                                              uint64_t* __restrict__ QL, uint32_t* __restrict__ L,
                                                              uint64_t* __restrict__ QH, uint32_t* __restrict__ H) {
    extern __shared__ __align__(16) unsigned char split_smem[];
    uint64_t* s_val = reinterpret_cast<uint64_t*>(split_smem);
    uint32_t* s_idx = reinterpret_cast<uint32_t*>(split_smem + (size_t)SPLIT_SUB * 8);
    __shared__ SplitAcc wt[SPLIT_THREADS / 32];
    constexpr int IT = SPLIT_SUB / SPLIT_THREADS;
    static_assert(IT == 8, "two 16-byte loads per thread");
    const uint64_t base = (uint64_t)blockIdx.x * SPLIT_TILE;
    SplitAcc run0 = tile_pre[blockIdx.x];  // everything before this piece
    for (uint64_t sb = base; sb < base + SPLIT_TILE && sb < N; sb += SPLIT_SUB) {
        const uint32_t cnt = N - sb < (uint64_t)SPLIT_SUB ? (uint32_t)(N - sb) : (uint32_t)SPLIT_SUB;
        const uint32_t t0 = threadIdx.x * IT;
        // the thread's 8 consecutive items, in registers (q is 16-byte aligned
        // and sb + t0 a multiple of 8)
        uint32_t qv[IT];
        if (t0 + IT <= cnt) {
            const uint4 u = __ldg(reinterpret_cast<const uint4*>(q + sb + t0));
            const uint4 v = __ldg(reinterpret_cast<const uint4*>(q + sb + t0 + 4));
            qv[0] = u.x; qv[1] = u.y; qv[2] = u.z; qv[3] = u.w;
            qv[4] = v.x; qv[5] = v.y; qv[6] = v.z; qv[7] = v.w;
        } else {
#pragma unroll
            for (int j = 0; j < IT; ++j) qv[j] = t0 + j < cnt ? q[sb + t0 + j] : 0u;
        }
        SplitAcc mine(0);
#pragma unroll
        for (int j = 0; j < IT; ++j)
            if (t0 + j < cnt) mine += split_item(qv[j], N, W);
        SplitAcc bt;
        SplitAcc run = block_exclusive_scan<SplitAcc, SPLIT_THREADS>(mine, wt, bt);
        const uint32_t nl = (uint32_t)bt.c;  // lights of the piece
#pragma unroll
        for (int j = 0; j < IT; ++j) {
            const uint32_t t = t0 + j;
            if (t >= cnt) break;
            const SplitAcc it = split_item(qv[j], N, W);
            if (it.c) {
                s_idx[run.c] = (uint32_t)(sb + t);
                s_val[run.c] = run0.QL + run.QL;
            } else {
                const uint32_t h = nl + (t - (uint32_t)run.c);
                s_idx[h] = (uint32_t)(sb + t);
                s_val[h] = run0.QH + run.QH + it.QH;
            }
            run += it;
        }
        __syncthreads();
        const uint64_t xb = run0.c, yb = sb - run0.c;  // lights and heavies before the piece
        for (uint32_t t = threadIdx.x; t < cnt; t += SPLIT_THREADS) {
            if (t < nl) {
                QL[xb + t] = s_val[t];
                L[xb + t] = s_idx[t];
            } else {
                QH[yb + t - nl] = s_val[t];
                H[yb + t - nl] = s_idx[t];
            }
        }
        run0 += bt;
        __syncthreads();
    }
}

// The two sorted sequences of the merge, from their weight prefixes.
struct SweepLists {
    const uint64_t* QL;  // [nL + 1] (QL[nL] = all lights' weight)
    const uint64_t* QH;  // [nH]
    uint64_t nL, nH, N, W;
    __device__ __forceinline__ u128 Dl(uint64_t x) const { return (u128)x * W - (u128)N * QL[x]; }
    __device__ __forceinline__ u128 S(uint64_t y) const { return (u128)N * QH[y] - (u128)(y + 1) * W; }
};

// Lights before diagonal `diag` of the merge (a light precedes a heavy iff
// Dl < S), on the sequences in memory ...
__device__ __forceinline__ uint64_t merge_path(const SweepLists& l, uint64_t diag) {
    uint64_t lo = diag > l.nH ? diag - l.nH : 0;
    uint64_t hi = diag < l.nL ? diag : l.nL;
    while (lo < hi) {
        const uint64_t mid = (lo + hi) >> 1;
        if (l.Dl(mid) < l.S(diag - mid - 1)) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// ... and on a tile's values in shared memory.
__device__ __forceinline__ uint32_t merge_path(const u128* A, uint32_t nA, const u128* B, uint32_t nB, uint32_t diag) {
    uint32_t lo = diag > nB ? diag - nB : 0;
    uint32_t hi = diag < nA ? diag : nA;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (A[mid] < B[diag - mid - 1]) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

constexpr int MERGE_THREADS = 256, MERGE_ITEMS = 8, MERGE_TILE = MERGE_THREADS * MERGE_ITEMS;

// Merge-path split of every tile boundary (diagonal t * MERGE_TILE, and the
// end): one thread per boundary, all searches in flight together.
__global__ void k_merge_partition(SweepLists l, uint64_t tiles, uint64_t* __restrict__ part) {
    const uint64_t total = l.nL + l.nH;
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t <= tiles; t += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t d = t * MERGE_TILE < total ? t * MERGE_TILE : total;
        part[t] = merge_path(l, d);
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

// Where the table goes: the node table as {thresh, alias} pairs, or the edge
// table as packed 16-byte or wide 32-byte records with the endpoints of the
// bucket's own entry and of its alias.
enum AliasOutKind { kOutNodes = 0, kOutEdges16 = 1, kOutEdges32 = 2 };

struct AliasOut {
    int kind;
    uint2* nodes;            // kOutNodes: [N]
    void* edges;             // kOutEdges*: [N] records
    const uint32_t* esrc;    // kOutEdges*: row of each entry
    const uint32_t* col;     // kOutEdges*: column of each entry
};


__device__ __forceinline__ void emit_entry(const AliasOut& o, int kind, uint32_t i, uint32_t th, uint32_t al) {
    if (kind == kOutNodes) {
        o.nodes[i] = make_uint2(th, al);
    } else {
        const uint32_t i0 = o.esrc[i], j0 = o.col[i], i1 = o.esrc[al], j1 = o.col[al];
        if (kind == kOutEdges16) {
            static_cast<uint4*>(o.edges)[i] = pack_edge16(th, i0, j0, i1, j1);
        } else {
            EdgeRec r;
            r.thresh = th;
            r.i0 = i0;
            r.j0 = j0;
            r.i1 = i1;
            r.j1 = j1;
            r.pad0 = r.pad1 = r.pad2 = 0;
            static_cast<EdgeRec*>(o.edges)[i] = r;
        }
    }
}

struct EmitArgs {
    SweepLists l;
    const uint32_t* L;     // [nL] item of each light
    const uint32_t* H;     // [nH] item of each heavy
    InvDiv D;
    const uint64_t* part;  // [tiles + 1] merge-path splits
};

// The merge, tile by tile, and each item's table entry from it.  Phase 1
// merges the tile's Dl and S values in shared memory and records each
// element's cross rank: light x placed after y heavies, heavy y after x
// lights.  Phase 2 writes the entries, lights then heavies, each in list
// (= item) order: light x has threshold a_x / W (a_x = W - (Dl(x + 1) -
// Dl(x)) = q N) and alias H[y]; heavy y has own mass S(y) + W - Dl(x), which
// fills the bucket (threshold all ones, alias itself) or leaves the rest to
// the next heavy H[y + 1].
template <int KIND>
__global__ void __launch_bounds__(MERGE_THREADS, 6) k_alias_emit(EmitArgs m, AliasOut o) {
    __shared__ u128 s[MERGE_TILE + 1];
    __shared__ uint16_t rank[MERGE_TILE];
    const SweepLists& l = m.l;
    const uint64_t total = l.nL + l.nH;
    const uint64_t d0 = (uint64_t)blockIdx.x * MERGE_TILE;
    const uint64_t d1 = d0 + MERGE_TILE < total ? d0 + MERGE_TILE : total;
    const uint64_t x0 = m.part[blockIdx.x], x1 = m.part[blockIdx.x + 1], y0 = d0 - x0, y1 = d1 - x1;
    const uint32_t na = (uint32_t)(x1 - x0), nb = (uint32_t)(y1 - y0);
    // Dl(x0 .. x1) inclusive (the value after the tile's last light closes
    // it), then S(y0 .. y1 - 1): slot u < na + 1 + nb <= MERGE_TILE + 1 of
    // s; each thread loads the weight prefixes of all its slots before it
    // computes any, so that their latencies overlap
    constexpr int SLOTS = (MERGE_TILE + 1 + MERGE_THREADS - 1) / MERGE_THREADS;
    const uint32_t nab = na + 1 + nb;
    uint64_t raw[SLOTS];
#pragma unroll
    for (int k = 0; k < SLOTS; ++k) {
        const uint32_t u = threadIdx.x + k * MERGE_THREADS;
        raw[k] = u <= na ? l.QL[x0 + u] : (u < nab ? l.QH[y0 + (u - na - 1)] : 0ull);
    }
#pragma unroll
    for (int k = 0; k < SLOTS; ++k) {
        const uint32_t u = threadIdx.x + k * MERGE_THREADS;
        if (u <= na) s[u] = (u128)(x0 + u) * l.W - (u128)l.N * raw[k];
        else if (u < nab) s[u] = (u128)l.N * raw[k] - (u128)(y0 + (u - na - 1) + 1) * l.W;
    }
    u128* Bs = s + na + 1;
    __syncthreads();
    const uint32_t dl = threadIdx.x * MERGE_ITEMS;
    if (dl < na + nb) {
        uint32_t xa = merge_path(s, na, Bs, nb, dl);
        uint32_t yb = dl - xa;
#pragma unroll
        for (int it = 0; it < MERGE_ITEMS; ++it) {
            if (xa + yb >= na + nb) break;
            if (xa < na && (yb >= nb || s[xa] < Bs[yb])) {
                rank[xa] = (uint16_t)yb;
                ++xa;
            } else {
                rank[na + yb] = (uint16_t)xa;
                ++yb;
            }
        }
    }
    __syncthreads();
    for (uint32_t t = threadIdx.x; t < na; t += MERGE_THREADS) {
        const uint32_t i = m.L[x0 + t];
        const uint64_t y = y0 + rank[t];
        const uint64_t a = l.W - (uint64_t)(s[t + 1] - s[t]);
        const uint32_t al = y < l.nH ? m.H[y] : i;  // y < nH whenever the totals are exact
        emit_entry(o, KIND, i, frac32(a, m.D), al);
    }
    for (uint32_t t = threadIdx.x; t < nb; t += MERGE_THREADS) {
        const uint64_t y = y0 + t;
        const uint32_t i = m.H[y];
        // own mass = S(y) + W - Dl(x); exact totals make the last heavy full,
        // the index guard only keeps a violated invariant from reading past H
        const uint64_t own = (uint64_t)(Bs[t] + (u128)l.W - s[rank[na + t]]);
        if (own >= l.W || y + 1 >= l.nH) emit_entry(o, KIND, i, 0xFFFFFFFFu, i);
        else emit_entry(o, KIND, i, frac32(own, m.D), m.H[y + 1]);
    }
}

struct Sum64 {
    const uint32_t* q;
    __device__ __forceinline__ uint64_t operator()(size_t i) const { return q[i]; }
};

// Alias table over N items with 32-bit weights q, written as `out` says.
// Returns false (nothing written) when the weights sum to zero.
// parts / nparts: when the weights' row sums are at hand (the edge table's
// r), their sum is the capacity W, a reduction over n values instead of N.
bool build_alias(drg_ctx* ctx, const uint32_t* q, uint64_t N, const AliasOut& out, const uint64_t* parts = nullptr,
                 uint64_t nparts = 0) {
    DRG_CHECK(N > 0 && N < (1ull << 32), DRG_EUNSUPPORTED, "alias table size must be in [1, 2^32)");
    DBuf<uint64_t> Wd(ctx, 1);
    if (parts) {
        DBuf<uint64_t> tmp(ctx, nparts);
        scan<uint64_t>(ctx, LoadArr<uint64_t>{parts}, nparts, tmp.p, false, Wd.p);
    } else {
        DBuf<uint64_t> sums(ctx, (N + ScanShape<uint64_t>::TILE - 1) / ScanShape<uint64_t>::TILE);
        const uint32_t nb = (uint32_t)sums.n;
        DRG_LAUNCH(ctx, (k_scan_reduce<uint64_t, Sum64>), nb, 256, 0, Sum64{q}, (size_t)N, sums.p);
        scan<uint64_t>(ctx, LoadArr<uint64_t>{sums.p}, nb, sums.p, false, Wd.p);
    }
    const uint64_t W = read1(ctx, Wd.p);
    if (W == 0) return false;
    // split scan: tile sums, their exclusive prefix, then the lists
    const uint64_t stiles = (N + SPLIT_TILE - 1) / SPLIT_TILE;
    DBuf<SplitAcc> tsum(ctx, stiles + 1);
    DRG_LAUNCH(ctx, k_split_reduce, (uint32_t)((stiles + SPLIT_REDUCE_TILES - 1) / SPLIT_REDUCE_TILES),
               SPLIT_THREADS, 0, q, N, W, stiles, tsum.p);
    scan<SplitAcc>(ctx, LoadArr<SplitAcc>{tsum.p}, stiles, tsum.p, false, tsum.p + stiles);
    SplitAcc tot(0);
    d2h(ctx, &tot, tsum.p + stiles, 1);
    sync(ctx);
    const uint64_t nL = tot.c, nH = N - nL;
    DBuf<uint64_t> QL(ctx, nL + 1), QH(ctx, nH);
    DBuf<uint32_t> L(ctx, nL), H(ctx, nH);
    DRG_CUDA(cudaFuncSetAttribute(k_split_down, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SPLIT_DOWN_SMEM));
    DRG_LAUNCH(ctx, k_split_down, (uint32_t)stiles, SPLIT_THREADS, SPLIT_DOWN_SMEM, q, N, W, tsum.p, QL.p, L.p, QH.p,
               H.p);
    h2d(ctx, QL.p + nL, &tot.QL, 1);
    // merge-path splits, then the merge writing the table
    const SweepLists lists{QL.p, QH.p, nL, nH, N, W};
    const uint64_t tiles = (N + MERGE_TILE - 1) / MERGE_TILE;
    DBuf<uint64_t> part(ctx, tiles + 1);
    DRG_LAUNCH(ctx, k_merge_partition, grid_for(tiles + 1, 256, 65536), 256, 0, lists, tiles, part.p);
    const EmitArgs m{lists, L.p, H.p, make_invdiv(W), part.p};
    auto kern = out.kind == kOutNodes ? k_alias_emit<kOutNodes>
                                      : (out.kind == kOutEdges16 ? k_alias_emit<kOutEdges16> : k_alias_emit<kOutEdges32>);
    DRG_LAUNCH(ctx, kern, (uint32_t)tiles, MERGE_THREADS, 0, m, out);
    sync(ctx);  // `tot` is a host value read by an asynchronous copy above
    return true;
}

// Alias entry of buckets [e0, e1) of the edge table, recovered from the
// records (inspection only; the sampling path never needs it): the alias's
// endpoints (i1, j1) name the entry of row i1 whose column is j1, found by a
// binary search of that sorted row.
__global__ void k_edge_alias_ids(const void* __restrict__ etab, int packed, const uint64_t* __restrict__ rp,
                                 const uint32_t* __restrict__ col, uint64_t e0, uint64_t e1, uint32_t* __restrict__ out) {
    for (uint64_t b = e0 + blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; b < e1; b += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t i1, j1;
        if (packed) {
            const uint4 e = static_cast<const uint4*>(etab)[b];
            i1 = (e.z >> 16) | ((e.w & 0xFFu) << 16);
            j1 = e.w >> 8;
        } else {
            const EdgeRec& r = static_cast<const EdgeRec*>(etab)[b];
            i1 = r.i1;
            j1 = r.j1;
        }
        uint64_t lo = rp[i1], hi = rp[i1 + 1];
        while (lo < hi) {
            const uint64_t mid = (lo + hi) >> 1;
            if (col[mid] < j1) lo = mid + 1; else hi = mid;
        }
        out[b - e0] = (uint32_t)lo;
    }
}

void edge_alias_ids(drg_ctx* ctx, const drg_dmat* d, uint64_t e0, uint64_t e1, uint32_t* host_out) {
    if (e1 <= e0) return;
    DBuf<uint32_t> tmp(ctx, e1 - e0);
    DRG_LAUNCH(ctx, k_edge_alias_ids, grid_for(e1 - e0, 256, (uint32_t)ctx->num_sms * 16), 256, 0, d->etab,
               d->erec_bytes == 16 ? 1 : 0, d->rp, d->col, e0, e1, tmp.p);
    d2h(ctx, host_out, tmp.p, e1 - e0);
    sync(ctx);
}

void dmat_free(drg_dmat* d) {
    if (!d) return;
    drg_ctx* c = d->ctx;
    void* ps[] = {d->rp, d->col, d->dist, d->q, d->r, d->Z, d->etab, d->vtab, d->beta};
    for (void* p : ps)
        if (p) dfree(c, p);
    delete d;
}

// Replaces d's kept rows K by the union pattern K u K^T (rows, columns,
// distances) and returns each union entry's flags (1: own, 2: back).
static DBuf<uint8_t> cap_union(drg_ctx* ctx, drg_dmat* d) {
    const uint32_t n = d->n;
    const uint64_t nK = d->nnz;
    DRG_CHECK(2 * nK < (1ull << 32), DRG_EUNSUPPORTED, "the capped rows hold 2^31 entries or more");
    const uint32_t cb = (uint32_t)std::max(1, bitlen(n > 1 ? n - 1 : 1));
    const uint32_t gk = grid_for(nK, 256, 65536);
    DBuf<uint32_t> esrc(ctx, nK);
    DRG_LAUNCH(ctx, k_expand_rows, grid_for((size_t)n * 32, 256, (uint32_t)ctx->num_sms * 16), 256, 0, d->rp, n,
               esrc.p);
    // T = K^T sorted by row (stable: ascending column within a row)
    DBuf<uint64_t> tkey(ctx, nK), tkalt(ctx, nK);
    DBuf<uint32_t> tval(ctx, nK), tvalt(ctx, nK);
    DRG_LAUNCH(ctx, k_cap_transpose, gk, 256, 0, esrc.p, d->col, d->dist, nK, tkey.p, tval.p);
    uint64_t* kp = tkey.p;
    uint64_t* ap = tkalt.p;
    uint32_t* vp = tval.p;
    uint32_t* vq = tvalt.p;
    radix_sort(ctx, kp, ap, vp, vq, nK, 0, (int)cb);
    DBuf<uint32_t> rpT(ctx, (size_t)n + 1);
    DRG_LAUNCH(ctx, k_rows_of_sorted, gk, 256, 0, kp, nK, n, rpT.p);
    // pairs kept on both sides, and each own entry's count of smaller back entries
    DBuf<uint32_t> tlo(ctx, nK), dup(ctx, nK), dpre(ctx, nK + 1);
    DRG_LAUNCH(ctx, k_cap_dups, gk, 256, 0, d->rp, esrc.p, d->col, rpT.p, vp, nK, tlo.p, dup.p);
    scan<uint32_t>(ctx, LoadArr<uint32_t>{dup.p}, nK, dpre.p, false, dpre.p + nK);
    DBuf<uint64_t> cnt(ctx, n), rpU(ctx, (size_t)n + 1), tot(ctx, 1);
    DRG_LAUNCH(ctx, k_cap_rowsize, grid_for(n, 256, 65536), 256, 0, d->rp, rpT.p, dpre.p, n, cnt.p);
    scan<uint64_t>(ctx, LoadArr<uint64_t>{cnt.p}, n, rpU.p, false, tot.p);
    const uint64_t nu = read1(ctx, tot.p);
    uint32_t* ucol = static_cast<uint32_t*>(dalloc(ctx, sizeof(uint32_t) * (nu ? nu : 1)));
    uint8_t* udist = static_cast<uint8_t*>(dalloc(ctx, dist_bytes(nu)));
    DRG_CUDA(cudaMemsetAsync(udist, 0, dist_bytes(nu), ctx->stream));
    DBuf<uint8_t> flag(ctx, nu);
    DRG_LAUNCH(ctx, k_cap_write_own, gk, 256, 0, d->rp, esrc.p, d->col, d->dist, tlo.p, dup.p, dpre.p, rpU.p, nK,
               ucol, udist, flag.p);
    DRG_LAUNCH(ctx, k_cap_write_back, gk, 256, 0, d->rp, d->col, rpT.p, kp, vp, dpre.p, rpU.p, nK, ucol, udist,
               flag.p);
    d2d(ctx, d->rp, rpU.p, (size_t)n);
    d2d(ctx, d->rp + n, tot.p, 1);
    dfree(ctx, d->col);
    dfree(ctx, d->dist);
    d->col = ucol;
    d->dist = udist;
    d->nnz = nu;
    return flag;
}

drg_dmat* build_dmat(drg_ctx* ctx, const drg_graph* g, uint32_t k, float sigma, float perplexity, uint32_t row_cap) {
    DRG_CHECK(g, DRG_EINVAL, "null graph");
    DRG_CHECK(row_cap == 0 || perplexity == 0.f, DRG_EUNSUPPORTED,
              "a row cap together with perplexity-calibrated sigma is not supported");
    DRG_CHECK(k >= 1 && k <= 15, DRG_EINVAL, "k must be in [1, 15]");
    DRG_CHECK(sigma > 0.f, DRG_EINVAL, "sigma must be positive");
    DRG_CHECK(perplexity >= 0.f && perplexity < 4.2e9f, DRG_EINVAL, "perplexity must be in [0, 4.2e9)");
    drg_dmat* d = new drg_dmat();
    d->ctx = ctx;
    d->n = g->n;
    d->k = k;
    d->sigma = sigma;
    d->perplexity = perplexity;
    try {
        DRG_CHECK(g->nnz > 0, DRG_EEMPTY, "graph has no edges");
        ProfSpan span(ctx, DRG_PROF_DMAT, 0);
        build_korder(ctx, g, k, d, row_cap);
        DBuf<uint8_t> flag;  // row cap: own / back flag of every union entry
        if (row_cap) flag = cap_union(ctx, d);
        d->row_cap = row_cap;
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
        DBuf<float> W;
        if (perplexity > 0.f) {
            ExpPoly P;
            P.c[0] = 1.0;
            for (int x = 1; x < 14; ++x) P.c[x] = P.c[x - 1] / (double)x;
            DBuf<uint32_t> cnt(ctx, (size_t)n * k);
            W = DBuf<float>(ctx, (size_t)n * k);
            d->beta = static_cast<double*>(dalloc(ctx, sizeof(double) * n));
            DRG_LAUNCH(ctx, k_row_Z<true>, gw, 256, 0, d->rp, d->dist, n, k, gs, d->Z, cnt.p);
            DRG_LAUNCH(ctx, k_calibrate, grid_for(n, 128, (uint32_t)ctx->num_sms * 16), 128, 0, cnt.p, n, k,
                       (double)perplexity, P, d->beta, d->Z, W.p);
        } else if (row_cap) {
            DRG_LAUNCH(ctx, k_row_Z_own, gw, 256, 0, d->rp, d->dist, flag.p, n, k, gs, d->Z);
        } else {
            DRG_LAUNCH(ctx, k_row_Z<false>, gw, 256, 0, d->rp, d->dist, n, k, gs, d->Z, (uint32_t*)nullptr);
        }
        DBuf<uint32_t> esrc(ctx, nnz);
        DRG_LAUNCH(ctx, k_expand_rows, gw, 256, 0, d->rp, n, esrc.p);
        DRG_CUDA(cudaMemsetAsync(d->r, 0, sizeof(uint64_t) * n, ctx->stream));
        const uint32_t gq = grid_for((nnz + 3) / 4, 256, 65536);
        unsigned long long* rr = reinterpret_cast<unsigned long long*>(d->r);
        if (row_cap)
            DRG_LAUNCH(ctx, k_quantise_r<Q_CAPPED>, gq, 256, 0, esrc.p, d->col, d->dist, d->Z, gs, nnz, d->q, rr,
                       (const float*)nullptr, k, (const uint8_t*)flag.p);
        else if (perplexity > 0.f)
            DRG_LAUNCH(ctx, k_quantise_r<Q_PER_NODE>, gq, 256, 0, esrc.p, d->col, d->dist, d->Z, gs, nnz, d->q, rr,
                       (const float*)W.p, k, (const uint8_t*)nullptr);
        else
            DRG_LAUNCH(ctx, k_quantise_r<Q_GLOBAL_SIGMA>, gq, 256, 0, esrc.p, d->col, d->dist, d->Z, gs, nnz, d->q, rr,
                       (const float*)nullptr, k, (const uint8_t*)nullptr);
        W.reset();
        flag.reset();
        DBuf<unsigned long long> rmax(ctx, 1);
        DRG_CUDA(cudaMemsetAsync(rmax.p, 0, 8, ctx->stream));
        DRG_LAUNCH(ctx, k_rmax, grid_for(n, 256, (uint32_t)ctx->num_sms * 8), 256, 0, d->r, n, rmax.p);
        const uint64_t mx = read1(ctx, rmax.p);
        const int bits = bitlen(mx);
        d->shift = bits > 32 ? (uint32_t)(bits - 32) : 0u;
        ss.reopen(DRG_PROF_ALIAS, nnz + n);
        // edge table over the entries (positive samples)
        {
            const bool packed = n <= kPackedIdLimit;
            d->erec_bytes = packed ? 16u : (uint32_t)sizeof(EdgeRec);
            d->etab = dalloc(ctx, (size_t)d->erec_bytes * nnz);
            AliasOut out{packed ? kOutEdges16 : kOutEdges32, nullptr, d->etab, esrc.p, d->col};
            // W = sum of q = sum of the row sums r (exact integers)
            DRG_CHECK(build_alias(ctx, d->q, nnz, out, d->r, n), DRG_EEMPTY, "all edge weights are zero");
        }
        // node table (negative samples)
        {
            DBuf<uint32_t> r32(ctx, n);
            DRG_LAUNCH(ctx, k_shift_u32, grid_for(n, 256, 65536), 256, 0, d->r, n, d->shift, r32.p);
            d->vtab = static_cast<uint2*>(dalloc(ctx, sizeof(uint2) * n));
            AliasOut out{kOutNodes, d->vtab, nullptr, nullptr, nullptr};
            DRG_CHECK(build_alias(ctx, r32.p, n, out), DRG_EEMPTY, "all node weights are zero");
        }
        sync(ctx);
    } catch (...) {
        dmat_free(d);
        throw;
    }
    return d;
}

}  // namespace drg
