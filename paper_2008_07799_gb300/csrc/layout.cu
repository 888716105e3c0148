// The layout optimisation of DRGraph (Sec. 3.2.2, Eqs. 11-12) on one level
// of the hierarchy (Sec. 3.2.3), and the whole coarse-to-fine run.
//
// A sample draws its random words from Philox (counter = sample, epoch,
// stream tag, call), reads one edge-table record (positive pair) and M
// node-table records (negatives), maps the drawn level-0 nodes to the level
// through the ancestor map, gathers 2 + M positions, forms the attractive and
// repulsive pair forces and adds them, with vector atomics, to the gradient
// buffer (synchronous mode) or straight into the positions (Hogwild mode).
// Every access after the Philox step is a random 8- to 16-byte read or
// atomic: the kernels are bound by L2 (positions, node tables) and HBM (edge
// table) request rate and latency, not by arithmetic.
//
// Two kernel families run the samples: k_hogwild (FP32 Hogwild: one
// cooperative launch per level run, each thread walking its share of every
// epoch) and k_epoch (synchronous mode and half-precision copies: one thread
// per sample of a sub-step run, the runs of an epoch chained in a CUDA graph).
#include "prims.cuh"

#include <atomic>
#include <cmath>
#include <cstring>
#include <cuda.h>
#include <exception>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <tuple>
#include <type_traits>

namespace drg {

// Epoch counter of a level run, advanced on the device between epochs.
struct EpochState {
    uint32_t t, t_end;       // current epoch, end of the run
    float lr;                // lr0 (1 - t / epochs) of the current epoch
    uint32_t pad;
    const float* lr_tab;     // [epochs] learning rates, computed on the host
};

struct EpochArgs {
    const EpochState* st;               // current epoch and learning rate
    int late;                           // 1: the previous kernel may change st; wait before reading it
    const void* __restrict__ etab;      // edge records (packed 16-byte or EdgeRec)
    int packed;                         // 1: packed 16-byte edge records
    uint64_t nnz;
    const uint2* __restrict__ vtab;
    const uint4* __restrict__ vtab_l;  // level node table (Hogwild kernels on coarse levels)
    uint32_t n0;
    const uint32_t* __restrict__ anc;  // level-0 node -> level node; nullptr = identity
    float2* Y;                          // positions of the level
    float2* G;                          // gradient accumulator (synchronous mode)
    const void* Yh;                     // half-precision copy for negative gathers (or nullptr)
    uint32_t M;
    float gamma, b, twob, clip;
    int bint;                           // 1, 2, 3: integer b; 0: general
    uint2 key;
    uint32_t tag, t;                    // t: epoch of k_draws (k_epoch reads st->t)
    float lr;                           // Hogwild step size of the current epoch (set in k_epoch)
    uint64_t s_begin, s_end;
};

__device__ __forceinline__ uint32_t lane_word(const uint4& v, uint32_t l) {
    return l == 0 ? v.x : (l == 1 ? v.y : (l == 2 ? v.z : v.w));
}

// Random word `w` of sample s: Philox call w/4, lane w%4.  Calls are made
// lazily and in increasing order, each once.
struct Words {
    uint4 cur;
    uint32_t idx;
    uint4 ctr;
    uint2 key;
    __device__ __forceinline__ Words(uint32_t s, uint32_t t, uint32_t tag, uint2 k)
        : idx(0xFFFFFFFFu), ctr(make_uint4(s, t, tag, 0)), key(k) {}
    __device__ __forceinline__ uint32_t operator()(uint32_t w) {
        if ((w >> 2) != idx) {
            idx = w >> 2;
            ctr.w = idx;
            cur = philox(ctr, key);
        }
        return lane_word(cur, w & 3);
    }
};

// A 16-byte edge record, read with an L2 evict-first policy and a 64-byte
// L2 prefetch size: the table is far larger than L2 and each record is read
// once at a random place, so its lines should leave L2 before the positions
// and node tables do, and a miss should fetch 64 bytes rather than a
// 128-byte line.
__device__ __forceinline__ uint4 ld_record(const uint4* p) {
    uint64_t pol;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    uint4 v;
    asm("ld.global.nc.L2::cache_hint.L2::64B.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
        : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
        : "l"(p), "l"(pol));
    return v;
}

// Edge record of bucket bkt: the first 16 bytes, and j1 of the wide form.
__device__ __forceinline__ void load_edge(const EpochArgs& a, uint64_t bkt, uint4& e, uint32_t& j1) {
    if (a.packed) {
        e = ld_record(static_cast<const uint4*>(a.etab) + bkt);
        j1 = 0;
    } else {
        const EdgeRec* r = static_cast<const EdgeRec*>(a.etab) + bkt;
        e = ld_record(reinterpret_cast<const uint4*>(r));
        j1 = __ldg(&r->j1);
    }
}

// The drawn pair: the bucket's own entry when U < thresh, else its alias.
__device__ __forceinline__ void edge_pair(const EpochArgs& a, const uint4& e, uint32_t j1, uint32_t U, uint32_t& i,
                                          uint32_t& j) {
    const bool keep = U < e.x;
    if (a.packed) {
        i = keep ? (e.y & 0xFFFFFFu) : ((e.z >> 16) | ((e.w & 0xFFu) << 16));
        j = keep ? ((e.y >> 24) | ((e.z & 0xFFFFu) << 8)) : (e.w >> 8);
    } else {
        i = keep ? e.y : e.w;
        j = keep ? e.z : j1;
    }
}

__device__ __forceinline__ void draw_edge(const EpochArgs& a, Words& W, uint32_t& i, uint32_t& j) {
    const uint64_t R = (uint64_t)W(0) | ((uint64_t)W(1) << 32);
    const uint32_t U = W(2);
    uint4 e;
    uint32_t j1;
    load_edge(a, alias_bucket(R, a.nnz), e, j1);
    edge_pair(a, e, j1, U, i, j);
}

__device__ __forceinline__ uint32_t draw_negative(const EpochArgs& a, Words& W, uint32_t m) {
    const uint64_t R = (uint64_t)W(3 + 3 * m) | ((uint64_t)W(4 + 3 * m) << 32);
    const uint32_t U = W(5 + 3 * m);
    const uint64_t bkt = alias_bucket(R, a.n0);
    const uint2 v = __ldg(&a.vtab[bkt]);
    return U < v.x ? (uint32_t)bkt : v.y;
}

__device__ __forceinline__ void pow_terms(float d2, float b, int bint, float& d2bm1, float& d2b) {
    if (bint == 1) {
        d2bm1 = 1.f;
        d2b = d2;
    } else if (bint == 2) {
        d2bm1 = d2;
        d2b = d2 * d2;
    } else if (bint == 3) {
        d2bm1 = d2 * d2;
        d2b = d2bm1 * d2;
    } else {
        d2bm1 = powf(d2, b - 1.f);
        d2b = d2bm1 * d2;
    }
}

__device__ __forceinline__ float clipf(float x, float c) { return fminf(fmaxf(x, -c), c); }

// Attraction on y_a from y_c: -2b d^{2b-2} (y_a - y_c) / (1 + d^{2b}).
__device__ __forceinline__ float2 attract(const EpochArgs& a, float2 ya, float2 yc) {
    const float dx = ya.x - yc.x, dy = ya.y - yc.y;
    const float d2 = dx * dx + dy * dy;
    if (!(d2 > 0.f)) return make_float2(0.f, 0.f);
    float d2bm1, d2b;
    pow_terms(d2, a.b, a.bint, d2bm1, d2b);
    const float coef = -a.twob * d2bm1 / (1.f + d2b);
    return make_float2(clipf(coef * dx, a.clip), clipf(coef * dy, a.clip));
}

// Repulsion on y_a from y_m: gamma 2b (y_a - y_m) / (d^2 (1 + d^{2b})).
__device__ __forceinline__ float2 repel(const EpochArgs& a, float2 ya, float2 ym) {
    const float dx = ya.x - ym.x, dy = ya.y - ym.y;
    const float d2 = dx * dx + dy * dy;
    if (!(d2 > 0.f)) return make_float2(0.f, 0.f);
    float d2bm1, d2b;
    pow_terms(d2, a.b, a.bint, d2bm1, d2b);
    const float coef = a.gamma * a.twob / (d2 * (1.f + d2b));
    return make_float2(clipf(coef * dx, a.clip), clipf(coef * dy, a.clip));
}

template <int PREC>
__device__ __forceinline__ float2 load_neg(const EpochArgs& a, uint32_t v) {
    if constexpr (PREC == DRG_PREC_FP16) {
        return __half22float2(reinterpret_cast<const __half2*>(a.Yh)[v]);
    } else if constexpr (PREC == DRG_PREC_BF16) {
        return __bfloat1622float2(reinterpret_cast<const __nv_bfloat162*>(a.Yh)[v]);
    } else {
        return a.Y[v];
    }
}

template <bool SYNC>
__device__ __forceinline__ void push(const EpochArgs& a, uint32_t v, float fx, float fy) {
    if constexpr (SYNC) {
        atomicAdd(&a.G[v], make_float2(fx, fy));
    } else {
        atomicAdd(&a.Y[v], make_float2(a.lr * fx, a.lr * fy));
    }
}

// One sample per thread.  Prologue (independent of the positions): Philox
// words, the edge record, the node records and the ancestor lookups.  Then
// wait for the previous run of samples to finish (programmatic dependent
// launch), and gather, compute and push.
// MT > 0: compile-time number of negatives (their loads are all issued before
// any is used); MT == 0: runtime M, negatives handled one after another.
template <int MT, bool SYNC, int PREC>
__device__ __forceinline__ void epoch_sample(EpochArgs& a, const uint64_t s) {
    const bool active = s < a.s_end;
    {
        Words W((uint32_t)s, __ldcg(&a.st->t), a.tag, a.key);
        uint32_t i = 0, j = 0;
        if (active) draw_edge(a, W, i, j);
        if constexpr (MT > 0) {
            uint32_t jm[MT];
            uint32_t ia = i, ic = j;
            if (active) {
#pragma unroll
                for (int m = 0; m < MT; ++m) jm[m] = draw_negative(a, W, m);
                if (a.anc) {
                    ia = __ldg(&a.anc[i]);
                    ic = __ldg(&a.anc[j]);
#pragma unroll
                    for (int m = 0; m < MT; ++m) jm[m] = __ldg(&a.anc[jm[m]]);
                }
            }
            if (!a.late) grid_dependency_wait();
            if (!active) return;
            if constexpr (!SYNC) a.lr = __ldcg(&a.st->lr);
            const float2 ya = a.Y[ia], yc = a.Y[ic];
            float2 ym[MT];
#pragma unroll
            for (int m = 0; m < MT; ++m) ym[m] = load_neg<PREC>(a, jm[m]);
            const float2 fa = attract(a, ya, yc);
            float Fx = fa.x, Fy = fa.y;
#pragma unroll
            for (int m = 0; m < MT; ++m) {
                if (jm[m] == ia || jm[m] == ic) continue;
                const float2 fr = repel(a, ya, ym[m]);
                Fx += fr.x;
                Fy += fr.y;
                push<SYNC>(a, jm[m], -fr.x, -fr.y);
            }
            push<SYNC>(a, ia, Fx, Fy);
            push<SYNC>(a, ic, -fa.x, -fa.y);
        } else {
            uint32_t ia = i, ic = j;
            if (active && a.anc) {
                ia = __ldg(&a.anc[i]);
                ic = __ldg(&a.anc[j]);
            }
            if (!a.late) grid_dependency_wait();
            if (!active) return;
            if constexpr (!SYNC) a.lr = __ldcg(&a.st->lr);
            const float2 ya = a.Y[ia], yc = a.Y[ic];
            const float2 fa = attract(a, ya, yc);
            float Fx = fa.x, Fy = fa.y;
            for (uint32_t m = 0; m < a.M; ++m) {
                uint32_t cm = draw_negative(a, W, m);
                if (a.anc) cm = __ldg(&a.anc[cm]);
                if (cm == ia || cm == ic) continue;
                const float2 fr = repel(a, ya, load_neg<PREC>(a, cm));
                Fx += fr.x;
                Fy += fr.y;
                push<SYNC>(a, cm, -fr.x, -fr.y);
            }
            push<SYNC>(a, ia, Fx, Fy);
            push<SYNC>(a, ic, -fa.x, -fa.y);
        }
    }
}

template <int MT, bool SYNC, int PREC>
__global__ void __launch_bounds__(256) k_epoch(EpochArgs a) {
    grid_dependency_trigger();
    if (a.late) grid_dependency_wait();
    epoch_sample<MT, SYNC, PREC>(a, a.s_begin + blockIdx.x * (uint64_t)blockDim.x + threadIdx.x);
}

// Index of the last entry of prefix[0 .. njobs) that is <= blk (prefix is
// non-decreasing, prefix[0] = 0): the job that owns block or thread blk.
__device__ __forceinline__ uint32_t find_job(const uint32_t* prefix, uint32_t njobs, uint32_t blk) {
    uint32_t lo = 0, hi = njobs;  // last job whose prefix is <= blk
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (prefix[mid] <= blk) lo = mid; else hi = mid;
    }
    return lo;
}

// ------------------------------------------------------------------ Hogwild level run in one launch
// Asynchronous mode (Sec. 4.3) as one persistent grid of T threads.  In every
// epoch thread g takes the samples g, g + T, g + 2T, ... < n_l one at a time,
// so at most T <= ceil(n_l / substeps) samples are in flight (between their
// position gathers and their atomic adds) at any moment -- the bound the
// sub-step runs give -- and no thread waits for another inside an epoch.
// Epochs stay in step: a warp starts epoch e only when every warp of the
// grid has finished epoch e - kEpochLag (the grid is launched cooperatively,
// so all its warps are resident).  Without this fast threads finish the
// low-learning-rate epochs while slow ones are epochs behind, which costs
// local quality (1M-node DC-SBM: NP .024 instead of .039); with a lag of two
// epochs and no block-wide wait only warps running ahead ever pause.
// Each thread keeps two samples ahead of the one it updates: the next
// sample's table records are resolved (and mapped through the ancestors) and
// the one after has its Philox words drawn and its records requested while
// the current sample's gathers are in flight; this position-independent work
// runs on across the epoch gates.  Positions are read through L2 only
// (ld.global.cg), since other SMs change them for the whole launch.
struct HogwildArgs {
    EpochArgs a;
    const float* lr_tab;  // [epochs] learning rate of each epoch
    uint32_t t_begin;     // first epoch
    uint32_t epochs;      // epochs of this launch
    uint32_t T;           // threads of the run
    uint32_t nl;          // samples per epoch (and nodes of the level)
    uint32_t refresh;     // half-precision copies: threads g < refresh rewrite nodes g, g + refresh, ...
};

// Epoch gates of one launch: done[e] counts the warps that finished epoch e
// (zero before the launch; nullptr: no gates); an error flag set when a wait
// runs out (then every warp leaves the kernel).  All lanes of a warp pass the
// gates together (they contain warp-wide shuffles).
struct GridSync {
    unsigned int* done;   // [epochs]
    int* err;
    uint32_t nwarps;      // warps that complete an epoch
    uint32_t lag;         // epoch e waits for epoch e - lag
    uint64_t timeout_ns;  // longest wait at one gate
};

constexpr uint32_t kEpochLag = 2;
constexpr uint64_t kGateTimeoutNs = 2000000000ull;  // 2 s, far above any epoch

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Before epoch e (e >= lag): wait until every warp finished epoch e - lag.
// False (on every lane) when the wait ran out or another warp gave up.
__device__ __forceinline__ bool epoch_gate(const GridSync& gs, uint32_t e) {
    __syncwarp();
    int ok = 1;
    if ((threadIdx.x & 31) == 0) {
        volatile unsigned int* d = gs.done + (e - gs.lag);
        volatile int* err = gs.err;
        if (*d < gs.nwarps) {
            const uint64_t t0 = global_ns();
            uint32_t nap = 64;
            while (*d < gs.nwarps) {
                if (*err || global_ns() - t0 > gs.timeout_ns) {
                    atomicExch(gs.err, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(nap);
                nap = nap < 1024 ? 2 * nap : nap;
            }
        }
        ok = ok && !*err;
    }
    return __shfl_sync(0xFFFFFFFFu, ok, 0) != 0;
}

// After epoch e: the warp reports it done.  No fence: the gates bound how far
// warps drift apart; the positions themselves are shared without ordering, as
// asynchronous SGD allows.
__device__ __forceinline__ void epoch_done(const GridSync& gs, uint32_t e) {
    __syncwarp();
    if ((threadIdx.x & 31) == 0) atomicAdd(gs.done + e, 1u);
}

// A sample's table records, requested (stage 1).  On level 0 a negative's
// record is the node table's {thresh, alias} and the bucket is the own item;
// on coarser levels it is the level's node table {thresh, anc(own),
// anc(alias), 0}, so no ancestor lookup follows.
template <int MT, bool ANC>
struct Requested {
    uint4 e;             // first 16 bytes of the drawn edge record
    uint32_t j1, Ue;
    typename std::conditional<ANC, uint4, uint2>::type v[MT];
    uint32_t bkt[MT], Uv[MT];
};

// A sample's nodes on the level (stage 2).
template <int MT>
struct Resolved {
    uint32_t ia, ic, jm[MT];
};

// The sample's random words: call 0 first, so that the edge record (the one
// access that goes to HBM) is requested before anything else; the other
// calls are independent chains computed side by side.
template <int MT, bool ANC>
__device__ __forceinline__ void hw_request(const EpochArgs& a, uint32_t s, uint32_t t, Requested<MT, ANC>& r) {
    constexpr int kCalls = (3 + 3 * MT + 3) / 4;  // words 0 .. 2 + 3 MT
    uint4 w[kCalls];
    w[0] = philox(make_uint4(s, t, a.tag, 0u), a.key);
    const uint64_t R = (uint64_t)w[0].x | ((uint64_t)w[0].y << 32);
    r.Ue = w[0].z;
    load_edge(a, alias_bucket(R, a.nnz), r.e, r.j1);
#pragma unroll
    for (int c = 1; c < kCalls; ++c) w[c] = philox(make_uint4(s, t, a.tag, (uint32_t)c), a.key);
#pragma unroll
    for (int m = 0; m < MT; ++m) {
        const int w0 = 3 + 3 * m, w1 = 4 + 3 * m, w2 = 5 + 3 * m;
        const uint64_t Rm = (uint64_t)lane_word(w[w0 >> 2], w0 & 3) | ((uint64_t)lane_word(w[w1 >> 2], w1 & 3) << 32);
        r.Uv[m] = lane_word(w[w2 >> 2], w2 & 3);
        r.bkt[m] = (uint32_t)alias_bucket(Rm, a.n0);
        if constexpr (ANC) r.v[m] = __ldg(&a.vtab_l[r.bkt[m]]);
        else r.v[m] = __ldg(&a.vtab[r.bkt[m]]);
    }
}

template <int MT, bool ANC>
__device__ __forceinline__ void hw_resolve(const EpochArgs& a, const Requested<MT, ANC>& r, Resolved<MT>& o) {
    uint32_t i, j;
    edge_pair(a, r.e, r.j1, r.Ue, i, j);
    o.ia = ANC ? __ldg(&a.anc[i]) : i;
    o.ic = ANC ? __ldg(&a.anc[j]) : j;
#pragma unroll
    for (int m = 0; m < MT; ++m) {
        if constexpr (ANC) o.jm[m] = r.Uv[m] < r.v[m].x ? r.v[m].y : r.v[m].z;
        else o.jm[m] = r.Uv[m] < r.v[m].x ? r.bkt[m] : r.v[m].y;
    }
}

// Level node table: the node table with both items mapped to the level.
__global__ void k_level_nodes(const uint2* __restrict__ vtab, const uint32_t* __restrict__ anc, uint32_t n0,
                              uint4* __restrict__ out) {
    for (uint64_t b = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; b < n0; b += (uint64_t)gridDim.x * blockDim.x) {
        const uint2 v = vtab[b];
        out[b] = make_uint4(v.x, anc[b], anc[v.y], 0u);
    }
}

// A negative's position for the force: the FP32 master or the half-precision
// copy, read through L2 only (both change during the launch).
template <int PREC>
__device__ __forceinline__ float2 hw_gather_neg(const EpochArgs& a, uint32_t v) {
    if constexpr (PREC == DRG_PREC_FP32) {
        return __ldcg(&a.Y[v]);
    } else {
        const unsigned int u = __ldcg(reinterpret_cast<const unsigned int*>(a.Yh) + v);
        if constexpr (PREC == DRG_PREC_FP16) {
            __half2 h;
            memcpy(&h, &u, sizeof(h));
            return __half22float2(h);
        } else {
            __nv_bfloat162 h;
            memcpy(&h, &u, sizeof(h));
            return __bfloat1622float2(h);
        }
    }
}

// End of an epoch with half-precision copies: thread g rewrites the copies of
// nodes g, g + stride, ... from the FP32 masters (coalesced), so a copy lags
// its master by at most the epochs that warps drift apart.
template <int PREC>
__device__ __forceinline__ void hw_refresh(const HogwildArgs& h, uint32_t g) {
    if constexpr (PREC != DRG_PREC_FP32) {
        if (g >= h.refresh) return;
        for (uint32_t v = g; v < h.nl; v += h.refresh) {
            const float2 y = __ldcg(&h.a.Y[v]);
            if constexpr (PREC == DRG_PREC_FP16) reinterpret_cast<__half2*>(const_cast<void*>(h.a.Yh))[v] = __float22half2_rn(y);
            else reinterpret_cast<__nv_bfloat162*>(const_cast<void*>(h.a.Yh))[v] = __float22bfloat162_rn(y);
        }
    }
}

__device__ __forceinline__ void hw_push(float2* Y, uint32_t v, float lr, float fx, float fy) {
    atomicAdd(&Y[v], make_float2(lr * fx, lr * fy));
}

// a thread's next sample: s += T within the epoch, else sample g of the next epoch
__device__ __forceinline__ void hw_advance(uint32_t& t, uint32_t& s, uint32_t g, uint32_t T, uint32_t nl) {
    if (s >= nl - T) {
        s = g;
        ++t;
    } else {
        s += T;
    }
}

// A thread's software pipeline over its samples 0, 1, 2, ...: while sample k
// is gathered, computed and pushed, sample k + 2 is resolved (its records,
// requested two samples earlier, have arrived; its ancestor lookups are
// issued) and sample k + 4 is requested (Philox words, table loads).  Two
// slots of each kind, used by sample parity, keep everything in registers.
template <int MT, bool ANC>
struct HwPipe {
    Requested<MT, ANC> Q[2];
    Resolved<MT> V[2];
    uint32_t tQ[2], tV[2];  // epochs of the slots' samples
    uint32_t t1, s1, g;     // next sample to request; the thread's first sample
};

template <int MT, bool ANC, int PREC, int P>
__device__ __forceinline__ void hw_step(const HogwildArgs& h, HwPipe<MT, ANC>& p, uint64_t k, uint64_t cnt) {
    const EpochArgs& a = h.a;
    const Resolved<MT> I = p.V[P];
    const float2 ya = __ldcg(&a.Y[I.ia]), yc = __ldcg(&a.Y[I.ic]);
    float2 ym[MT];
#pragma unroll
    for (int m = 0; m < MT; ++m) ym[m] = hw_gather_neg<PREC>(a, I.jm[m]);
    const float lr = __ldg(&h.lr_tab[p.tV[P]]);
    if (k + 2 < cnt) {
        hw_resolve<MT, ANC>(a, p.Q[P], p.V[P]);
        p.tV[P] = p.tQ[P];
    }
    if (k + 4 < cnt) {
        hw_request<MT, ANC>(a, p.s1, p.t1, p.Q[P]);
        p.tQ[P] = p.t1;
        hw_advance(p.t1, p.s1, p.g, h.T, h.nl);
    }
    const float2 fa = attract(a, ya, yc);
    float Fx = fa.x, Fy = fa.y;
#pragma unroll
    for (int m = 0; m < MT; ++m) {
        if (I.jm[m] == I.ia || I.jm[m] == I.ic) continue;
        const float2 fr = repel(a, ya, ym[m]);
        Fx += fr.x;
        Fy += fr.y;
        hw_push(a.Y, I.jm[m], lr, -fr.x, -fr.y);
    }
    hw_push(a.Y, I.ia, lr, Fx, Fy);
    hw_push(a.Y, I.ic, lr, -fa.x, -fa.y);
}

template <int MT, bool ANC, int P>
__device__ __forceinline__ void hw_fill(const HogwildArgs& h, HwPipe<MT, ANC>& p) {
    hw_request<MT, ANC>(h.a, p.s1, p.t1, p.Q[P]);
    p.tQ[P] = p.t1;
    hw_advance(p.t1, p.s1, p.g, h.T, h.nl);
}

// Samples of thread g in each epoch (0 for threads past the run's T).
__device__ __forceinline__ uint32_t hw_share(const HogwildArgs& h, uint32_t g) {
    return g < h.T ? (h.nl - g + h.T - 1) / h.T : 0u;
}

// One thread's share of a run: in each epoch the samples g, g + T, ... < n_l;
// every thread of the grid takes part in every epoch barrier.
template <int MT, bool ANC, int PREC>
__device__ __forceinline__ bool hogwild_thread(const HogwildArgs& h, const GridSync& gs, uint32_t g,
                                               uint32_t t_begin, uint32_t epochs) {
    const uint32_t share = hw_share(h, g);
    const uint64_t cnt = (uint64_t)share * epochs;  // samples of this thread
    HwPipe<MT, ANC> p;
    p.t1 = t_begin;
    p.s1 = g;
    p.g = g;
    if (cnt > 0) hw_fill<MT, ANC, 0>(h, p);                // sample 0
    if (cnt > 1) hw_fill<MT, ANC, 1>(h, p);                // sample 1
    if (cnt > 0) {
        hw_resolve<MT, ANC>(h.a, p.Q[0], p.V[0]);
        p.tV[0] = p.tQ[0];
    }
    if (cnt > 2) hw_fill<MT, ANC, 0>(h, p);                // sample 2
    if (cnt > 1) {
        hw_resolve<MT, ANC>(h.a, p.Q[1], p.V[1]);
        p.tV[1] = p.tQ[1];
    }
    if (cnt > 3) hw_fill<MT, ANC, 1>(h, p);                // sample 3
    uint64_t k = 0;
    for (uint32_t e = 0; e < epochs; ++e) {
        if (gs.done && e >= gs.lag && !epoch_gate(gs, e)) return false;
        // samples [k, end) of this epoch, two at a time (slot parity = sample
        // parity; the pair body lets one sample's compute fill the other's waits)
        const uint64_t end = k + share;
        if (k < end && (k & 1)) hw_step<MT, ANC, PREC, 1>(h, p, k++, cnt);
        for (; k + 1 < end; k += 2) {
            hw_step<MT, ANC, PREC, 0>(h, p, k, cnt);
            hw_step<MT, ANC, PREC, 1>(h, p, k + 1, cnt);
        }
        if (k < end) hw_step<MT, ANC, PREC, 0>(h, p, k++, cnt);
        hw_refresh<PREC>(h, g);
        if (gs.done) epoch_done(gs, e);
    }
    return true;
}

// Runtime number of negatives: the same samples, one after another.
template <bool ANC, int PREC>
__device__ __forceinline__ bool hogwild_thread_rt(const HogwildArgs& h, const GridSync& gs, uint32_t g,
                                                  uint32_t t_begin, uint32_t epochs) {
    const EpochArgs& a = h.a;
    const uint32_t share = hw_share(h, g);
    for (uint32_t e = 0; e < epochs; ++e) {
        if (gs.done && e >= gs.lag && !epoch_gate(gs, e)) return false;
        const uint32_t t = t_begin + e;
        const float lr = __ldg(&h.lr_tab[t]);
        for (uint32_t i = 0, s = g; i < share; ++i, s += h.T) {
            Words W(s, t, a.tag, a.key);
            uint32_t ii, jj;
            draw_edge(a, W, ii, jj);
            const uint32_t ia = ANC ? __ldg(&a.anc[ii]) : ii, ic = ANC ? __ldg(&a.anc[jj]) : jj;
            const float2 ya = __ldcg(&a.Y[ia]), yc = __ldcg(&a.Y[ic]);
            const float2 fa = attract(a, ya, yc);
            float Fx = fa.x, Fy = fa.y;
            for (uint32_t m = 0; m < a.M; ++m) {
                uint32_t cm = draw_negative(a, W, m);
                if (ANC) cm = __ldg(&a.anc[cm]);
                if (cm == ia || cm == ic) continue;
                const float2 fr = repel(a, ya, hw_gather_neg<PREC>(a, cm));
                Fx += fr.x;
                Fy += fr.y;
                hw_push(a.Y, cm, lr, -fr.x, -fr.y);
            }
            hw_push(a.Y, ia, lr, Fx, Fy);
            hw_push(a.Y, ic, lr, -fa.x, -fa.y);
        }
        hw_refresh<PREC>(h, g);
        if (gs.done) epoch_done(gs, e);
    }
    return true;
}

template <int MT, bool ANC, int PREC>
__device__ __forceinline__ void hogwild_dispatch(const HogwildArgs& h, const GridSync& gs, uint32_t g,
                                                 uint32_t t_begin, uint32_t epochs) {
    if constexpr (MT > 0) hogwild_thread<MT, ANC, PREC>(h, gs, g, t_begin, epochs);
    else hogwild_thread_rt<ANC, PREC>(h, gs, g, t_begin, epochs);
}

// MT > 0: compile-time number of negatives; MT == 0: runtime M.  PREC: the
// negatives' positions from the FP32 masters or from a half-precision copy
// (refreshed at the end of every epoch).  Every thread of the grid (also
// those past T) runs, for the epoch barriers.
template <int MT, bool ANC, int PREC>
__global__ void __launch_bounds__(256, 2) k_hogwild(HogwildArgs h, GridSync gs) {
    hogwild_dispatch<MT, ANC, PREC>(h, gs, blockIdx.x * blockDim.x + threadIdx.x, h.t_begin, h.epochs);
}

// One level of each of many graphs in one launch: run x owns the threads
// [prefix[x], prefix[x + 1]); threads past the last run only pass the epoch
// gates (all runs have the same number of epochs).  Every run has an
// ancestor map (level-0 runs the identity), so all threads of a block take
// the same code path through the gates.
template <int MT, int PREC>
__global__ void __launch_bounds__(256, 2) k_hogwild_batch(const HogwildArgs* __restrict__ runs,
                                                       const uint32_t* __restrict__ prefix, uint32_t nruns,
                                                       GridSync gs, uint32_t t_begin, uint32_t epochs) {
    const uint32_t gt = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t x = find_job(prefix, nruns, gt);
    const HogwildArgs& h = runs[x];
    const uint32_t g = gt - prefix[x];
    hogwild_dispatch<MT, true, PREC>(h, gs, g, t_begin, epochs);
}

__global__ void k_iota(uint32_t* __restrict__ out, uint32_t n) {
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x)
        out[v] = (uint32_t)v;
}

// ------------------------------------------------------------------ batches of graphs
// Sub-step c of the current level of many graphs in one launch.  Blocks are
// assigned to jobs (graph, level) by a prefix sum of each job's block count;
// each job's run c covers its own samples [c chunk, min(n_l, (c+1) chunk)).
struct BatchJob {
    const void* etab;
    int packed;
    uint64_t nnz;
    const uint2* vtab;
    const uint32_t* anc;
    float2* Y;
    float2* G;
    void* Yh;
    uint32_t n0, nl, chunk, tag;
    float gamma, b, twob;
    int bint;
};

struct BatchArgs {
    EpochArgs common;             // st, late, M, clip, key
    const BatchJob* jobs;
    const uint32_t* block_prefix; // [njobs + 1] sample blocks per job, prefix-summed
    const uint32_t* node_prefix;  // [njobs + 1] node blocks per job, prefix-summed
    uint32_t njobs;
};

template <int MT, bool SYNC, int PREC>
__global__ void __launch_bounds__(256) k_epoch_batch(BatchArgs ba, uint32_t c) {
    grid_dependency_trigger();
    if (ba.common.late) grid_dependency_wait();
    const uint32_t jb = find_job(ba.block_prefix, ba.njobs, blockIdx.x);
    const BatchJob J = ba.jobs[jb];
    EpochArgs a = ba.common;
    a.etab = J.etab;
    a.packed = J.packed;
    a.nnz = J.nnz;
    a.vtab = J.vtab;
    a.n0 = J.n0;
    a.anc = J.anc;
    a.Y = J.Y;
    a.G = J.G;
    a.Yh = J.Yh;
    a.tag = J.tag;
    a.gamma = J.gamma;
    a.b = J.b;
    a.twob = J.twob;
    a.bint = J.bint;
    a.s_begin = (uint64_t)c * J.chunk;
    a.s_end = a.s_begin + J.chunk < J.nl ? a.s_begin + J.chunk : J.nl;
    const uint64_t s = a.s_begin + (uint64_t)(blockIdx.x - ba.block_prefix[jb]) * blockDim.x + threadIdx.x;
    epoch_sample<MT, SYNC, PREC>(a, s);
}

template <int PREC>
__global__ void k_apply_batch(BatchArgs ba) {
    grid_dependency_trigger();
    grid_dependency_wait();
    const uint32_t jb = find_job(ba.node_prefix, ba.njobs, blockIdx.x);
    const BatchJob J = ba.jobs[jb];
    const float lr = __ldcg(&ba.common.st->lr);
    const uint64_t v = (uint64_t)(blockIdx.x - ba.node_prefix[jb]) * blockDim.x + threadIdx.x;
    if (v >= J.nl) return;
    float2 y = J.Y[v];
    if (J.G) {
        const float2 g = J.G[v];
        y.x += lr * g.x;
        y.y += lr * g.y;
        J.Y[v] = y;
        J.G[v] = make_float2(0.f, 0.f);
    }
    if constexpr (PREC == DRG_PREC_FP16) reinterpret_cast<__half2*>(J.Yh)[v] = __float22half2_rn(y);
    if constexpr (PREC == DRG_PREC_BF16) reinterpret_cast<__nv_bfloat162*>(J.Yh)[v] = __float22bfloat162_rn(y);
}

// Synchronous sub-step end: Y += lr G, G = 0 (and the half copy refreshed).
template <int PREC>
__global__ void k_apply(float2* __restrict__ Y, float2* __restrict__ G, void* __restrict__ Yh, uint32_t n,
                        const EpochState* __restrict__ st) {
    grid_dependency_trigger();
    grid_dependency_wait();
    const float lr = __ldcg(&st->lr);
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x) {
        const float2 g = G[v];
        float2 y = Y[v];
        y.x += lr * g.x;
        y.y += lr * g.y;
        Y[v] = y;
        G[v] = make_float2(0.f, 0.f);
        if constexpr (PREC == DRG_PREC_FP16) reinterpret_cast<__half2*>(Yh)[v] = __float22half2_rn(y);
        if constexpr (PREC == DRG_PREC_BF16) reinterpret_cast<__nv_bfloat162*>(Yh)[v] = __float22bfloat162_rn(y);
    }
}

template <int PREC>
__global__ void k_refresh(const float2* __restrict__ Y, void* __restrict__ Yh, uint32_t n) {
    grid_dependency_trigger();
    grid_dependency_wait();
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x) {
        if constexpr (PREC == DRG_PREC_FP16) reinterpret_cast<__half2*>(Yh)[v] = __float22half2_rn(Y[v]);
        if constexpr (PREC == DRG_PREC_BF16) reinterpret_cast<__nv_bfloat162*>(Yh)[v] = __float22bfloat162_rn(Y[v]);
    }
}

// End of an epoch inside the level graph: next epoch and learning rate, and
// the condition of the graph's WHILE loop.
__global__ void k_advance(EpochState* st, cudaGraphConditionalHandle loop) {
    const uint32_t t = st->t + 1;
    st->t = t;
    const bool more = t < st->t_end;
    if (more) st->lr = st->lr_tab[t];
    cudaGraphSetConditional(loop, more ? 1u : 0u);
}

// Epoch state set from the host side of a level run.
__global__ void k_set_epoch(EpochState* st, uint32_t t, uint32_t t_end, float lr) {
    st->t = t;
    st->t_end = t_end;
    st->lr = lr;
    st->pad = 0;
    st->lr_tab = nullptr;
}

// Draws only (inspection): the same random streams as k_epoch.
__global__ void k_draws(EpochArgs a, uint32_t* __restrict__ oi, uint32_t* __restrict__ oj, uint32_t* __restrict__ oneg) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t s = a.s_begin + blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < a.s_end; s += stride) {
        Words W((uint32_t)s, a.t, a.tag, a.key);
        uint32_t i, j;
        draw_edge(a, W, i, j);
        const uint64_t o = s - a.s_begin;
        oi[o] = i;
        oj[o] = j;
        for (uint32_t m = 0; m < a.M; ++m) oneg[o * a.M + m] = draw_negative(a, W, m);
    }
}

// Sec. 3.2.3: random coarsest layout, uniform in [-scale, scale]^2.
__global__ void k_init(float2* __restrict__ Y, uint32_t n, uint2 key, uint32_t tag, float scale) {
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x) {
        const uint4 w = philox(make_uint4((uint32_t)v, 0, tag, 0), key);
        const float ux = __fmul_rn(__uint2float_rn(w.x >> 8), 5.9604644775390625e-08f);
        const float uy = __fmul_rn(__uint2float_rn(w.y >> 8), 5.9604644775390625e-08f);
        Y[v] = make_float2(__fmul_rn(__fsub_rn(__fmul_rn(2.f, ux), 1.f), scale),
                           __fmul_rn(__fsub_rn(__fmul_rn(2.f, uy), 1.f), scale));
    }
}

// Sec. 3.2.3 refinement: a fine node starts at its coarse node's position.
__global__ void k_interp(const float2* __restrict__ coarse, const uint32_t* __restrict__ parent,
                         float2* __restrict__ fine, uint32_t n) {
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x)
        fine[v] = coarse[parent[v]];
}

// ------------------------------------------------------------------ host side
void check_params(const drg_params& p) {
    DRG_CHECK(p.k >= 1 && p.k <= 15, DRG_EINVAL, "k must be in [1, 15]");
    DRG_CHECK(p.M <= 64, DRG_EINVAL, "M must be at most 64");
    DRG_CHECK(p.epochs >= 1, DRG_EINVAL, "epochs must be >= 1");
    DRG_CHECK(p.b > 0.f && p.clip > 0.f && p.sigma > 0.f, DRG_EINVAL, "b, clip and sigma must be positive");
    DRG_CHECK(p.gamma >= 0.f && p.gamma_coarsest >= 0.f, DRG_EINVAL, "gamma must be non-negative");
    DRG_CHECK(p.mode == DRG_MODE_SYNC || p.mode == DRG_MODE_HOGWILD, DRG_EINVAL, "mode must be 0 or 1");
    DRG_CHECK(p.precision >= 0 && p.precision <= 2, DRG_EINVAL, "precision must be 0, 1 or 2");
    DRG_CHECK(p.substeps >= 1, DRG_EINVAL, "substeps must be >= 1");
    DRG_CHECK(p.max_levels >= 1 && p.max_levels <= 64, DRG_EINVAL, "max_levels must be in [1, 64]");
    DRG_CHECK(p.rho > 0.f && p.rho <= 1.f, DRG_EINVAL, "rho must be in (0, 1]");
    DRG_CHECK(p.coarsen == DRG_COARSEN_HEM || p.coarsen == DRG_COARSEN_STAR, DRG_EINVAL,
              "coarsen must be DRG_COARSEN_HEM or DRG_COARSEN_STAR");
    DRG_CHECK(p.level_tables == 0 || p.level_tables == 1, DRG_EINVAL, "level_tables must be 0 or 1");
    DRG_CHECK(p.perplexity >= 0.f && p.perplexity < 4.2e9f, DRG_EINVAL, "perplexity must be in [0, 4.2e9)");
}

static int int_b(float b) {
    if (b == 1.f) return 1;
    if (b == 2.f) return 2;
    if (b == 3.f) return 3;
    return 0;
}

static EpochArgs epoch_args(const drg_dmat* d, const uint32_t* anc, float2* Y, const drg_params& p, float gamma,
                            uint32_t level) {
    EpochArgs a{};
    a.etab = d->etab;
    a.packed = d->erec_bytes == 16 ? 1 : 0;
    a.nnz = d->nnz;
    a.vtab = d->vtab;
    a.n0 = d->n;
    a.anc = anc;
    a.Y = Y;
    a.M = p.M;
    a.gamma = gamma;
    a.b = p.b;
    a.twob = 2.f * p.b;
    a.clip = p.clip;
    a.bint = int_b(p.b);
    a.key = seed_key(p.seed);
    a.tag = stream_tag(kPurposeSample, p.gid, level);
    return a;
}

typedef void (*EpochKernel)(EpochArgs);

static EpochKernel pick_epoch(uint32_t M, bool sync, int prec) {
    static const EpochKernel tab[2][2][3] = {
        {{k_epoch<0, false, 0>, k_epoch<0, false, 1>, k_epoch<0, false, 2>},
         {k_epoch<0, true, 0>, k_epoch<0, true, 1>, k_epoch<0, true, 2>}},
        {{k_epoch<5, false, 0>, k_epoch<5, false, 1>, k_epoch<5, false, 2>},
         {k_epoch<5, true, 0>, k_epoch<5, true, 1>, k_epoch<5, true, 2>}},
    };
    return tab[M == 5 ? 1 : 0][sync ? 1 : 0][prec];
}

// one thread per sample
static uint32_t epoch_grid(drg_ctx*, uint64_t count) { return (uint32_t)((count + 255) / 256); }

typedef void (*HogwildKernel)(HogwildArgs, GridSync);

static HogwildKernel pick_hogwild(uint32_t M, bool anc, int prec) {
    static const HogwildKernel tab[2][2][3] = {
        {{k_hogwild<0, false, 0>, k_hogwild<0, false, 1>, k_hogwild<0, false, 2>},
         {k_hogwild<0, true, 0>, k_hogwild<0, true, 1>, k_hogwild<0, true, 2>}},
        {{k_hogwild<5, false, 0>, k_hogwild<5, false, 1>, k_hogwild<5, false, 2>},
         {k_hogwild<5, true, 0>, k_hogwild<5, true, 1>, k_hogwild<5, true, 2>}},
    };
    return tab[M == 5 ? 1 : 0][anc ? 1 : 0][prec];
}

// Cooperative launch (all blocks resident together); false when the grid
// cannot be resident at once, with nothing launched.
template <typename... KArgs, typename... Args>
static bool launch_cooperative(drg_ctx* ctx, const char* name, void (*kernel)(KArgs...), uint32_t grid,
                               uint32_t block, Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = ctx->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
    if (e == cudaErrorCooperativeLaunchTooLarge) {
        (void)cudaGetLastError();
        return false;
    }
    DRG_CUDA(e);
    after_launch(ctx, name);
    return true;
}

// The epoch-gate state of a launch: one counter per epoch and the error
// flag, zeroed on the stream.
struct SyncBuf {
    DBuf<unsigned int> done;
    DBuf<int> err;
    SyncBuf(drg_ctx* ctx, uint32_t epochs) : done(ctx, epochs), err(ctx, 1) {
        DRG_CUDA(cudaMemsetAsync(done.p, 0, (size_t)(epochs ? epochs : 1) * sizeof(unsigned int), ctx->stream));
        DRG_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), ctx->stream));
    }
    GridSync sync(uint32_t nwarps, uint32_t lag, uint64_t timeout_ns) const {
        return GridSync{done.p, err.p, nwarps, lag, timeout_ns};
    }
    void check(drg_ctx* ctx) {
        DRG_CHECK(read1(ctx, err.p) == 0, DRG_ETIMEOUT, "an epoch gate of a Hogwild level run timed out");
    }
};

// ------------------------------------------------------------------ launch-shape autotuner
// The Hogwild level kernels run a fixed number of threads T <= the in-flight
// bound, so their launch shape is the one free choice: threads per block
// (64, 128 or 256: how the warps spread over the SMs) and the samples per
// thread (T = the bound, half or a quarter of it; a smaller T only tightens the
// bound).
// The first long run of each (device, kernel, M, precision, ancestor map,
// size bucket) times every candidate for a few epochs on a scratch copy of
// its positions and keeps the fastest for the process.
struct TuneKey {
    int dev, family, prec, anc;
    uint32_t M, bucket;
    bool operator<(const TuneKey& o) const {
        return std::tie(dev, family, prec, anc, M, bucket) < std::tie(o.dev, o.family, o.prec, o.anc, o.M, o.bucket);
    }
};

struct TuneChoice {
    uint32_t block, div;
    float ms;  // per epoch, of the choice, in the tuning run
};

static std::mutex g_tune_mu;
static std::map<TuneKey, TuneChoice> g_tune;
constexpr uint32_t kTuneBlocks[3] = {64, 128, 256};
constexpr uint32_t kTuneDivs[3] = {1, 2, 4};
constexpr uint32_t kTuneEpochs = 3;      // epochs timed per candidate
constexpr uint32_t kTuneMinEpochs = 50;  // runs shorter than this use the default shape
constexpr TuneChoice kTuneDefault{128, 1, 0.f};

static uint32_t bitlen32(uint64_t x) {
    uint32_t b = 0;
    while (x) {
        ++b;
        x >>= 1;
    }
    return b;
}

static bool tune_lookup(const TuneKey& key, TuneChoice& out) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    const auto it = g_tune.find(key);
    if (it == g_tune.end()) return false;
    out = it->second;
    return true;
}

static void tune_store(const TuneKey& key, const TuneChoice& c) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune[key] = c;
}

uint32_t autotune_read(uint32_t cap, uint32_t* keys, uint32_t* choice, float* ms) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    uint32_t i = 0;
    for (const auto& kv : g_tune) {
        if (i < cap) {
            if (keys) {
                uint32_t* k = keys + 6 * (size_t)i;
                k[0] = (uint32_t)kv.first.family;
                k[1] = kv.first.M;
                k[2] = (uint32_t)kv.first.prec;
                k[3] = (uint32_t)kv.first.anc;
                k[4] = kv.first.bucket;
                k[5] = (uint32_t)kv.first.dev;
            }
            if (choice) {
                choice[2 * (size_t)i] = kv.second.block;
                choice[2 * (size_t)i + 1] = kv.second.div;
            }
            if (ms) ms[i] = kv.second.ms;
        }
        ++i;
    }
    return i;
}

void autotune_clear() {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune.clear();
}

// Threads of a block size that can be resident at once.
template <typename K>
static uint64_t resident_threads(drg_ctx* ctx, K kernel, uint32_t block) {
    int per_sm = 0;
    DRG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, (int)block, 0));
    return (uint64_t)(per_sm > 0 ? per_sm : 1) * (uint64_t)ctx->num_sms * block;
}

// One Hogwild level run of h.T threads in blocks of `block`: one cooperative
// launch (all epochs, warps kept in step by the gates), or one launch per
// epoch when the grid cannot be resident at once.  Returns the launches made.
static uint64_t run_hogwild(drg_ctx* ctx, HogwildKernel k, HogwildArgs h, uint32_t block) {
    const uint32_t grid = (h.T + block - 1) / block;
    h.refresh = grid * block;
    SyncBuf sb(ctx, h.epochs);
    uint64_t launches = 1;
    if (!launch_cooperative(ctx, "k_hogwild", k, grid, block, h,
                            sb.sync(grid * (block / 32), kEpochLag, kGateTimeoutNs))) {
        launches = h.epochs;
        for (uint32_t e = 0; e < h.epochs; ++e) {
            HogwildArgs h1 = h;
            h1.t_begin = h.t_begin + e;
            h1.epochs = 1;
            DRG_LAUNCH(ctx, k, grid, block, 0, h1, GridSync{nullptr, nullptr, grid, 0, 0});
        }
    }
    sb.check(ctx);
    return launches;
}

static uint32_t hogwild_threads(drg_ctx* ctx, HogwildKernel k, uint64_t bound, const TuneChoice& c) {
    const uint64_t want = (bound + c.div - 1) / c.div;
    const uint64_t res = resident_threads(ctx, k, c.block);
    return (uint32_t)(want < res ? want : res);
}

static void refresh_half(drg_ctx* ctx, int prec, const float2* Y, void* Yh, uint32_t n) {
    const uint32_t gn = grid_for(n, 256, (uint32_t)ctx->num_sms * 8);
    if (prec == 1) DRG_LAUNCH(ctx, k_refresh<1>, gn, 256, 0, Y, Yh, n);
    else if (prec == 2) DRG_LAUNCH(ctx, k_refresh<2>, gn, 256, 0, Y, Yh, n);
}

// Times every candidate shape for kTuneEpochs epochs on scratch copies of
// the run's positions (and half copies) and returns the fastest.
static TuneChoice tune_hogwild(drg_ctx* ctx, HogwildKernel k, const HogwildArgs& h0, uint64_t bound, int prec) {
    DBuf<float2> Yt(ctx, h0.nl);
    DBuf<uint32_t> Yht;
    d2d(ctx, Yt.p, h0.a.Y, h0.nl);
    if (prec) {
        Yht = DBuf<uint32_t>(ctx, h0.nl);
        refresh_half(ctx, prec, Yt.p, Yht.p, h0.nl);
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    DRG_CUDA(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        fail(DRG_ECUDA, "cudaEventCreate failed");
    }
    TuneChoice best{kTuneDefault.block, kTuneDefault.div, 3.4e38f};
    try {
        for (uint32_t block : kTuneBlocks) {
            for (uint32_t div : kTuneDivs) {
                HogwildArgs h = h0;
                h.a.Y = Yt.p;
                h.a.Yh = prec ? Yht.p : nullptr;
                h.epochs = kTuneEpochs;
                const TuneChoice c{block, div, 0.f};
                h.T = hogwild_threads(ctx, k, bound, c);
                DRG_CUDA(cudaEventRecord(e0, ctx->stream));
                run_hogwild(ctx, k, h, block);
                DRG_CUDA(cudaEventRecord(e1, ctx->stream));
                DRG_CUDA(cudaEventSynchronize(e1));
                float t = 0.f;
                DRG_CUDA(cudaEventElapsedTime(&t, e0, e1));
                t /= (float)kTuneEpochs;
                if (t < best.ms) best = TuneChoice{block, div, t};
            }
        }
    } catch (...) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return best;
}

// Epochs [t_begin, t_end) of a Hogwild level run in one cooperative launch of
// T <= min(ceil(n_l / substeps), resident threads) threads, in the launch
// shape the autotuner chose (one launch per epoch when the grid cannot be
// resident at once).  With half-precision copies (a.Yh, filled before the
// call) the negatives read the copy, which every thread of the grid helps
// rewrite at the end of each epoch.
static void hogwild_level(drg_ctx* ctx, const EpochArgs& a, const drg_params& p, uint32_t nl, const float* lr_tab,
                          uint32_t t_begin, uint32_t t_end) {
    const HogwildKernel k = pick_hogwild(p.M, a.anc != nullptr, p.precision);
    const uint64_t bound = ((uint64_t)nl + p.substeps - 1) / p.substeps;
    HogwildArgs h{};
    h.a = a;
    h.lr_tab = lr_tab;
    h.t_begin = t_begin;
    h.epochs = t_end - t_begin;
    h.nl = nl;
    DBuf<uint4> vl;
    if (a.anc) {
        vl = DBuf<uint4>(ctx, a.n0);
        DRG_LAUNCH(ctx, k_level_nodes, grid_for(a.n0, 256, (uint32_t)ctx->num_sms * 8), 256, 0, a.vtab, a.anc, a.n0,
                   vl.p);
        h.a.vtab_l = vl.p;
    }
    TuneChoice c = kTuneDefault;
    const TuneKey key{ctx->device, 0, p.precision, a.anc ? 1 : 0, p.M == 5 ? 5u : 0u, bitlen32(nl)};
    if (ctx->autotune && bound > 1 && h.epochs >= kTuneMinEpochs && !tune_lookup(key, c)) {
        c = tune_hogwild(ctx, k, h, bound, p.precision);
        tune_store(key, c);
    }
    h.T = hogwild_threads(ctx, k, bound, c);
    ProfSpan span(ctx, DRG_PROF_EPOCH, (uint64_t)h.epochs * nl, 1);
    span.count = run_hogwild(ctx, k, h, c.block);
}

// Hogwild runs of many graphs (each with T = ceil(n_l / substeps) set) in one
// launch.  When their threads exceed what the GPU holds at once, every run's
// thread count is scaled down in proportion (at least one each), so that all
// threads are resident together and the bound only tightens.  The block size
// is tuned like the single-graph runs' (per total thread count).
typedef void (*BatchKernel)(const HogwildArgs*, const uint32_t*, uint32_t, GridSync, uint32_t, uint32_t);

static uint64_t run_hogwild_batch(drg_ctx* ctx, BatchKernel k, std::vector<HogwildArgs> runs, uint32_t block,
                                  uint32_t epochs) {
    const uint64_t resident = resident_threads(ctx, k, block);
    uint64_t want = 0;
    for (const auto& h : runs) want += h.T;
    const uint64_t nruns = runs.size();
    if (want > resident) {
        const uint64_t room = resident > nruns ? resident - nruns : 0;
        for (auto& h : runs) h.T = (uint32_t)(1 + (uint64_t)h.T * room / want);
    }
    std::vector<uint32_t> prefix(nruns + 1, 0);
    for (size_t x = 0; x < nruns; ++x) {
        prefix[x + 1] = prefix[x] + runs[x].T;
        runs[x].refresh = runs[x].T;  // a run's copies are rewritten by its own threads
    }
    DBuf<HogwildArgs> druns(ctx, nruns);
    DBuf<uint32_t> dprefix(ctx, nruns + 1);
    h2d(ctx, druns.p, runs.data(), nruns);
    h2d(ctx, dprefix.p, prefix.data(), nruns + 1);
    const uint32_t grid = (prefix[nruns] + block - 1) / block;
    SyncBuf sb(ctx, epochs);
    uint64_t launches = 1;
    if (!launch_cooperative(ctx, "k_hogwild_batch", k, grid, block, druns.p, dprefix.p, (uint32_t)nruns,
                            sb.sync(grid * (block / 32), kEpochLag, kGateTimeoutNs), 0u, epochs)) {
        launches = epochs;
        for (uint32_t t = 0; t < epochs; ++t)
            DRG_LAUNCH(ctx, k, grid, block, 0, druns.p, dprefix.p, (uint32_t)nruns,
                       GridSync{nullptr, nullptr, grid, 0, 0}, t, 1u);
    }
    sb.check(ctx);
    return launches;
}

static void hogwild_batch(drg_ctx* ctx, uint32_t M, int prec, std::vector<HogwildArgs>& runs, uint32_t epochs,
                          uint64_t samples) {
    if (runs.empty()) return;
    std::vector<DBuf<uint4>> tables;     // level node tables
    std::vector<DBuf<uint32_t>> idmaps;  // identity ancestor maps of level-0 runs
    for (auto& h : runs) {
        if (!h.a.anc) {
            idmaps.emplace_back(ctx, h.a.n0);
            DRG_LAUNCH(ctx, k_iota, grid_for(h.a.n0, 256, (uint32_t)ctx->num_sms * 8), 256, 0, idmaps.back().p,
                       h.a.n0);
            h.a.anc = idmaps.back().p;
        }
        tables.emplace_back(ctx, h.a.n0);
        DRG_LAUNCH(ctx, k_level_nodes, grid_for(h.a.n0, 256, (uint32_t)ctx->num_sms * 8), 256, 0, h.a.vtab, h.a.anc,
                   h.a.n0, tables.back().p);
        h.a.vtab_l = tables.back().p;
    }
    static const BatchKernel tab[2][3] = {{k_hogwild_batch<0, 0>, k_hogwild_batch<0, 1>, k_hogwild_batch<0, 2>},
                                          {k_hogwild_batch<5, 0>, k_hogwild_batch<5, 1>, k_hogwild_batch<5, 2>}};
    const BatchKernel k = tab[M == 5 ? 1 : 0][prec];
    uint64_t want = 0, nodes = 0;
    for (const auto& h : runs) {
        want += h.T;
        nodes += h.nl;
    }
    TuneChoice c = kTuneDefault;
    const TuneKey key{ctx->device, 1, prec, 1, M == 5 ? 5u : 0u, bitlen32(want)};
    if (ctx->autotune && epochs >= kTuneMinEpochs && !tune_lookup(key, c)) {
        // every candidate block size on scratch copies of all runs' positions
        DBuf<float2> Yt(ctx, nodes);
        DBuf<uint32_t> Yht;
        if (prec) Yht = DBuf<uint32_t>(ctx, nodes);
        std::vector<HogwildArgs> trial = runs;
        uint64_t off = 0;
        for (auto& h : trial) {
            d2d(ctx, Yt.p + off, h.a.Y, h.nl);
            h.a.Y = Yt.p + off;
            if (prec) {
                h.a.Yh = Yht.p + off;
                refresh_half(ctx, prec, h.a.Y, const_cast<void*>(h.a.Yh), h.nl);
            }
            h.epochs = kTuneEpochs;
            off += h.nl;
        }
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        DRG_CUDA(cudaEventCreate(&e0));
        if (cudaEventCreate(&e1) != cudaSuccess) {
            cudaEventDestroy(e0);
            fail(DRG_ECUDA, "cudaEventCreate failed");
        }
        TuneChoice best{kTuneDefault.block, 1, 3.4e38f};
        try {
            for (uint32_t block : kTuneBlocks) {
                DRG_CUDA(cudaEventRecord(e0, ctx->stream));
                run_hogwild_batch(ctx, k, trial, block, kTuneEpochs);
                DRG_CUDA(cudaEventRecord(e1, ctx->stream));
                DRG_CUDA(cudaEventSynchronize(e1));
                float t = 0.f;
                DRG_CUDA(cudaEventElapsedTime(&t, e0, e1));
                t /= (float)kTuneEpochs;
                if (t < best.ms) best = TuneChoice{block, 1, t};
            }
        } catch (...) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            throw;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        c = best;
        tune_store(key, c);
    }
    ProfSpan span(ctx, DRG_PROF_EPOCH, samples, 1);
    span.count = run_hogwild_batch(ctx, k, runs, c.block, epochs);
}

// Gate check: `blocks` one-warp blocks run `rounds` empty epochs through
// gates (lag one) that open when `arrivals` warps have finished the previous
// epoch.  With arrivals > blocks no gate opens and every wait runs out after
// timeout_ms: DRG_ETIMEOUT.
__global__ void k_gate_probe(GridSync gs, uint32_t rounds) {
    for (uint32_t e = 0; e < rounds; ++e) {
        if (e >= gs.lag && !epoch_gate(gs, e)) return;
        epoch_done(gs, e);
    }
}

void check_epoch_barrier(drg_ctx* ctx, uint32_t blocks, uint32_t arrivals, uint32_t rounds, uint32_t timeout_ms) {
    DRG_CHECK(blocks >= 1 && blocks <= (uint32_t)ctx->num_sms && arrivals >= 1 && rounds >= 1 && rounds <= 100000 &&
                  timeout_ms >= 1 && timeout_ms <= 10000,
              DRG_EINVAL, "blocks in [1, SMs], arrivals >= 1, rounds in [1, 100000], timeout in [1, 10000] ms");
    SyncBuf sb(ctx, rounds);
    DRG_CHECK(launch_cooperative(ctx, "k_gate_probe", k_gate_probe, blocks, 32,
                                 sb.sync(arrivals, 1, (uint64_t)timeout_ms * 1000000ull), rounds),
              DRG_EUNSUPPORTED, "the probe grid cannot be resident at once");
    sb.check(ctx);
}

// One CUDA graph for a level run: a WHILE node whose body is one epoch --
// `body` captures its launches (sub-step runs chained by programmatic
// dependent launch) -- closed by k_advance, which moves the epoch state on and
// sets the loop condition.  One graph launch then runs every epoch.
template <typename Body>
static void run_epoch_loop_graph(drg_ctx* ctx, EpochState* st, Body&& body, uint64_t launches_run,
                                 uint64_t prof_units, uint64_t prof_launches) {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    const uint64_t launches_before = ctx->launches;
    auto cleanup = [&]() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
    };
    try {
        DRG_CUDA(cudaGraphCreate(&graph, 0));
        cudaGraphConditionalHandle loop;
        DRG_CUDA(cudaGraphConditionalHandleCreate(&loop, graph, 1, cudaGraphCondAssignDefault));
        cudaGraphNodeParams np = {};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = loop;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        cudaGraphNode_t wnode;
        DRG_CUDA(cudaGraphAddNode(&wnode, graph, nullptr, nullptr, 0, &np));
        cudaGraph_t bodyg = np.conditional.phGraph_out[0];
        DRG_CUDA(cudaStreamBeginCaptureToGraph(ctx->stream, bodyg, nullptr, nullptr, 0,
                                               cudaStreamCaptureModeThreadLocal));
        try {
            body();
            DRG_LAUNCH(ctx, k_advance, 1, 1, 0, st, loop);
        } catch (...) {
            cudaGraph_t dummy = nullptr;
            cudaStreamEndCapture(ctx->stream, &dummy);
            (void)cudaGetLastError();
            throw;
        }
        DRG_CUDA(cudaStreamEndCapture(ctx->stream, &bodyg));
        DRG_CUDA(cudaGraphInstantiate(&exec, graph, 0));
        ctx->launches = launches_before + launches_run;  // count what runs, not what was captured
        {
            ProfSpan span(ctx, DRG_PROF_EPOCH, prof_units, prof_launches);
            DRG_CUDA(cudaGraphLaunch(exec, ctx->stream));
        }
        sync(ctx);
    } catch (...) {
        cleanup();
        throw;
    }
    cleanup();
}

void layout_level(drg_ctx* ctx, const drg_dmat* d, const drg_hier* h, uint32_t level, float* pos,
                  const drg_params& p, float gamma, uint32_t t_begin, uint32_t t_end) {
    check_params(p);
    DRG_CHECK(d && pos, DRG_EINVAL, "null distance matrix or positions");
    DRG_CHECK(level == 0 || (h && level < h->g.size()), DRG_EINVAL, "level out of range");
    DRG_CHECK(t_begin <= t_end && t_end <= p.epochs, DRG_EINVAL, "epoch range outside [0, epochs]");
    // d is G^0's matrix (samples mapped to the level through its ancestor
    // map) or, at a coarse level, the level graph's own (no mapping)
    const bool own = level > 0 && h && d->n != h->g[0]->n && d->n == h->g[level]->n;
    DRG_CHECK(!h || own || h->g[0]->n == d->n, DRG_EINVAL, "hierarchy and distance matrix describe different graphs");
    const uint32_t nl = level == 0 ? d->n : h->g[level]->n;
    const uint32_t* anc = (level == 0 || own) ? nullptr : h->anc[level];
    float2* Y = reinterpret_cast<float2*>(pos);
    const bool sync_mode = p.mode == DRG_MODE_SYNC;
    const int prec = p.precision;
    EpochArgs a = epoch_args(d, anc, Y, p, gamma, level);
    DBuf<float2> G;
    DBuf<uint32_t> Yh;
    if (sync_mode) {
        G = DBuf<float2>(ctx, nl);
        DRG_CUDA(cudaMemsetAsync(G.p, 0, sizeof(float2) * nl, ctx->stream));
        a.G = G.p;
    }
    const uint32_t gn = grid_for(nl, 256, (uint32_t)ctx->num_sms * 8);
    if (prec) {
        Yh = DBuf<uint32_t>(ctx, nl);
        a.Yh = Yh.p;
        if (prec == 1) DRG_LAUNCH(ctx, k_refresh<1>, gn, 256, 0, Y, (void*)Yh.p, nl);
        else DRG_LAUNCH(ctx, k_refresh<2>, gn, 256, 0, Y, (void*)Yh.p, nl);
    }
    if (t_begin == t_end) return;
    const EpochKernel ek = pick_epoch(p.M, sync_mode, prec);
    const uint32_t chunk = (uint32_t)(((uint64_t)nl + p.substeps - 1) / p.substeps);
    const uint32_t nchunks = (uint32_t)(((uint64_t)nl + chunk - 1) / chunk);

    // learning rates of every epoch (host, as lr0 (1 - t/T)) and the epoch state
    std::vector<float> lr_host(p.epochs);
    for (uint32_t t = 0; t < p.epochs; ++t)
        lr_host[t] = (float)((double)p.lr0 * (1.0 - (double)t / (double)p.epochs));
    DBuf<float> lr_tab(ctx, p.epochs);
    h2d(ctx, lr_tab.p, lr_host.data(), p.epochs);
    if (!sync_mode) {
        hogwild_level(ctx, a, p, nl, lr_tab.p, t_begin, t_end);
        return;
    }
    DBuf<EpochState> st(ctx, 1);
    const EpochState st0{t_begin, t_end, lr_host[t_begin], 0u, lr_tab.p};
    h2d(ctx, st.p, &st0, 1);
    a.st = st.p;

    // One graph per level run: a WHILE node whose body is one epoch -- its
    // sub-step runs (each a k_epoch launch, chained by programmatic dependent
    // launch; synchronous mode applies the gradient after each run) and
    // k_advance, which moves the epoch state on and sets the loop condition.
    auto epoch_body = [&]() {
        for (uint32_t c = 0; c < nchunks; ++c) {
            a.s_begin = (uint64_t)c * chunk;
            a.s_end = a.s_begin + chunk < nl ? a.s_begin + chunk : nl;
            a.late = c == 0 ? 1 : 0;  // the first run follows the epoch-state update
            launch_pdl(ctx, "k_epoch", ek, epoch_grid(ctx, a.s_end - a.s_begin), 256, 0, a);
            if (sync_mode) {
                if (prec == 0) launch_pdl(ctx, "k_apply", k_apply<0>, gn, 256, 0, Y, G.p, (void*)nullptr, nl, st.p);
                else if (prec == 1) launch_pdl(ctx, "k_apply", k_apply<1>, gn, 256, 0, Y, G.p, (void*)Yh.p, nl, st.p);
                else launch_pdl(ctx, "k_apply", k_apply<2>, gn, 256, 0, Y, G.p, (void*)Yh.p, nl, st.p);
            }
        }
        if (!sync_mode && prec == 1) launch_pdl(ctx, "k_refresh", k_refresh<1>, gn, 256, 0, Y, (void*)Yh.p, nl);
        if (!sync_mode && prec == 2) launch_pdl(ctx, "k_refresh", k_refresh<2>, gn, 256, 0, Y, (void*)Yh.p, nl);
    };
    const uint64_t epochs = t_end - t_begin;
    if (ctx->direct_launch) {
        // the same launches issued from the host, epoch by epoch (profilers
        // cannot look inside graphs with conditional nodes)
        {
            ProfSpan span(ctx, DRG_PROF_EPOCH, (uint64_t)nl * epochs, epochs * nchunks);
            for (uint32_t t = t_begin; t < t_end; ++t) {
                DRG_LAUNCH(ctx, k_set_epoch, 1, 1, 0, st.p, t, t_end, lr_host[t]);
                epoch_body();
            }
        }
        sync(ctx);
        return;
    }
    const uint64_t per_epoch = (uint64_t)nchunks * (sync_mode ? 2 : 1) + 1 + (!sync_mode && prec ? 1 : 0);
    run_epoch_loop_graph(ctx, st.p, epoch_body, epochs * per_epoch, (uint64_t)nl * epochs, epochs * nchunks);
}

void init_positions(drg_ctx* ctx, uint32_t n, uint32_t level, const drg_params& p, float* pos) {
    DRG_CHECK(pos || n == 0, DRG_EINVAL, "null positions");
    DRG_LAUNCH(ctx, k_init, grid_for(n, 256, (uint32_t)ctx->num_sms * 8), 256, 0, reinterpret_cast<float2*>(pos), n,
               seed_key(p.seed), stream_tag(kPurposeInit, p.gid, level), p.init_scale);
}

void interpolate(drg_ctx* ctx, const drg_hier* h, uint32_t coarse_level, const float* coarse_pos, float* fine_pos) {
    DRG_CHECK(h && coarse_pos && fine_pos, DRG_EINVAL, "null argument");
    DRG_CHECK(coarse_level >= 1 && coarse_level < h->g.size(), DRG_EINVAL, "coarse level out of range");
    const uint32_t nf = h->g[coarse_level - 1]->n;
    DRG_LAUNCH(ctx, k_interp, grid_for(nf, 256, (uint32_t)ctx->num_sms * 8), 256, 0,
               reinterpret_cast<const float2*>(coarse_pos), h->parent[coarse_level - 1],
               reinterpret_cast<float2*>(fine_pos), nf);
}

void sample_draws(drg_ctx* ctx, const drg_dmat* d, uint32_t level, uint32_t t, uint32_t s_begin, uint32_t s_end,
                  const drg_params& p, uint32_t* oi, uint32_t* oj, uint32_t* oneg) {
    check_params(p);
    DRG_CHECK(d && oi && oj && (oneg || p.M == 0), DRG_EINVAL, "null argument");
    DRG_CHECK(s_begin <= s_end, DRG_EINVAL, "empty sample range");
    EpochArgs a = epoch_args(d, nullptr, nullptr, p, p.gamma, level);
    a.t = t;
    a.s_begin = s_begin;
    a.s_end = s_end;
    DRG_LAUNCH(ctx, k_draws, grid_for(s_end - s_begin, 256, (uint32_t)ctx->num_sms * 8), 256, 0, a, oi, oj, oneg);
}

// ------------------------------------------------------------------ caller-given samples
// One synchronous step over S samples the caller fixes (for closed-form tests
// of Eq. 12): the forces of every sampled term are computed from the
// positions at the start, summed per node with the level kernels' arithmetic
// (attract, repel, the skip rule for negatives that hit the source or
// target), then applied, Y += lr G.
__global__ void k_explicit_check(const uint32_t* __restrict__ sa, const uint32_t* __restrict__ sc,
                                 const uint32_t* __restrict__ sneg, uint32_t S, uint32_t M, uint32_t n,
                                 uint32_t* __restrict__ bad) {
    for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < S; s += (uint64_t)gridDim.x * blockDim.x) {
        bool ok = sa[s] < n && sc[s] < n;
        for (uint32_t m = 0; m < M; ++m) ok = ok && sneg[s * M + m] < n;
        if (!ok) atomicOr(bad, 1u);
    }
}

__global__ void k_explicit_forces(EpochArgs a, const uint32_t* __restrict__ sa, const uint32_t* __restrict__ sc,
                                  const uint32_t* __restrict__ sneg, uint32_t S) {
    for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < S; s += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t ia = sa[s], ic = sc[s];
        const float2 ya = a.Y[ia], yc = a.Y[ic];
        const float2 fa = attract(a, ya, yc);
        float Fx = fa.x, Fy = fa.y;
        for (uint32_t m = 0; m < a.M; ++m) {
            const uint32_t cm = sneg[s * a.M + m];
            if (cm == ia || cm == ic) continue;
            const float2 fr = repel(a, ya, a.Y[cm]);
            Fx += fr.x;
            Fy += fr.y;
            push<true>(a, cm, -fr.x, -fr.y);
        }
        push<true>(a, ia, Fx, Fy);
        push<true>(a, ic, -fa.x, -fa.y);
    }
}

void layout_step_explicit(drg_ctx* ctx, uint32_t n, float* pos, uint32_t S, const uint32_t* sa, const uint32_t* sc,
                          const uint32_t* sneg, uint32_t M, float gamma, float b, float lr, float clip) {
    DRG_CHECK(pos && n >= 1, DRG_EINVAL, "null positions or no node");
    DRG_CHECK(S == 0 || (sa && sc && (sneg || M == 0)), DRG_EINVAL, "null sample array");
    DRG_CHECK(M <= 64 && b > 0.f && clip > 0.f && gamma >= 0.f, DRG_EINVAL,
              "M must be at most 64, b and clip positive, gamma non-negative");
    if (S == 0) return;
    DBuf<uint32_t> bad(ctx, 1);
    DRG_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(uint32_t), ctx->stream));
    const uint32_t gs = grid_for(S, 256, (uint32_t)ctx->num_sms * 8);
    DRG_LAUNCH(ctx, k_explicit_check, gs, 256, 0, sa, sc, sneg, S, M, n, bad.p);
    DRG_CHECK(read1(ctx, bad.p) == 0, DRG_EINVAL, "a sample names a node id >= n");
    DBuf<float2> G(ctx, n);
    DRG_CUDA(cudaMemsetAsync(G.p, 0, sizeof(float2) * n, ctx->stream));
    EpochArgs a{};
    a.Y = reinterpret_cast<float2*>(pos);
    a.G = G.p;
    a.M = M;
    a.gamma = gamma;
    a.b = b;
    a.twob = 2.f * b;
    a.clip = clip;
    a.bint = int_b(b);
    DRG_LAUNCH(ctx, k_explicit_forces, gs, 256, 0, a, sa, sc, sneg, S);
    DBuf<EpochState> st(ctx, 1);
    DRG_LAUNCH(ctx, k_set_epoch, 1, 1, 0, st.p, 0u, 1u, lr);
    DRG_LAUNCH(ctx, k_apply<0>, grid_for(n, 256, (uint32_t)ctx->num_sms * 8), 256, 0, a.Y, G.p, (void*)nullptr, n,
               (const EpochState*)st.p);
    sync(ctx);
}

// A context for a host worker thread: the parent's device and settings, its
// own stream, no profiling events.
struct WorkerCtx {
    drg_ctx c;
    explicit WorkerCtx(const drg_ctx* parent) {
        c.device = parent->device;
        c.num_sms = parent->num_sms;
        c.max_smem_optin = parent->max_smem_optin;
        c.direct_launch = parent->direct_launch;
        c.autotune = parent->autotune;
        c.bfs_stage_limit = parent->bfs_stage_limit;
        DRG_CUDA(cudaSetDevice(c.device));
        DRG_CUDA(cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking));
        c.own_stream = true;
    }
    ~WorkerCtx() {
        if (c.stream) cudaStreamDestroy(c.stream);  // released once its queued work is done
    }
    WorkerCtx(const WorkerCtx&) = delete;
    WorkerCtx& operator=(const WorkerCtx&) = delete;
};

// The whole path of Fig. 1: distance matrix and sampling tables on G^0,
// hierarchy, random coarsest layout, then coarse to fine: all epochs of a
// level, refinement to the next finer level.
void layout_full(drg_ctx* ctx, const drg_graph* g, const drg_params& p, float* pos) {
    check_params(p);
    DRG_CHECK(g && pos, DRG_EINVAL, "null argument");
    drg_dmat* d = nullptr;
    drg_hier* h = nullptr;
    std::unique_ptr<WorkerCtx> hw;  // owns h when built concurrently; freed after h
    try {
        if (ctx->prof) {
            d = build_dmat(ctx, g, p.k, p.sigma, p.perplexity, p.row_cap);
            h = build_hierarchy(ctx, g, p);
        } else {
            // the hierarchy does not need the distance matrix: a worker thread
            // builds it on its own stream meanwhile
            hw.reset(new WorkerCtx(ctx));
            std::exception_ptr herr;
            std::thread th([&]() {
                try {
                    DRG_CUDA(cudaSetDevice(ctx->device));
                    h = build_hierarchy(&hw->c, g, p);
                    sync(&hw->c);
                } catch (...) {
                    herr = std::current_exception();
                }
            });
            try {
                d = build_dmat(ctx, g, p.k, p.sigma, p.perplexity, p.row_cap);
            } catch (...) {
                th.join();
                throw;
            }
            th.join();
            ctx->launches += hw->c.launches;
            if (herr) std::rethrow_exception(herr);
        }
        const uint32_t L = (uint32_t)h->g.size() - 1;
        DBuf<float2> cur, nxt;
        float* cur_pos = pos;
        if (L > 0) {
            cur = DBuf<float2>(ctx, h->g[L]->n);
            cur_pos = reinterpret_cast<float*>(cur.p);
        }
        init_positions(ctx, h->g[L]->n, L, p, cur_pos);
        for (int l = (int)L; l >= 0; --l) {
            const float gamma = (l == (int)L && L > 0) ? p.gamma_coarsest : p.gamma;
            if (p.level_tables && l > 0) {
                // the conventional scheme: this level's own matrix and tables
                drg_dmat* dl = build_dmat(ctx, h->g[l], p.k, p.sigma, p.perplexity, p.row_cap);
                try {
                    layout_level(ctx, dl, h, (uint32_t)l, cur_pos, p, gamma, 0, p.epochs);
                    sync(ctx);
                } catch (...) {
                    cudaStreamSynchronize(ctx->stream);
                    dmat_free(dl);
                    throw;
                }
                dmat_free(dl);
            } else {
                layout_level(ctx, d, h, (uint32_t)l, cur_pos, p, gamma, 0, p.epochs);
            }
            if (l > 0) {
                float* fine_pos = pos;
                if (l - 1 > 0) {
                    nxt = DBuf<float2>(ctx, h->g[l - 1]->n);
                    fine_pos = reinterpret_cast<float*>(nxt.p);
                }
                interpolate(ctx, h, (uint32_t)l, cur_pos, fine_pos);
                cur = std::move(nxt);
                cur_pos = fine_pos;
            }
        }
        sync(ctx);
    } catch (...) {
        cudaStreamSynchronize(ctx->stream);
        (void)cudaGetLastError();
        hier_free(h);
        dmat_free(d);
        throw;
    }
    hier_free(h);
    dmat_free(d);
}

typedef void (*EpochBatchKernel)(BatchArgs, uint32_t);

static EpochBatchKernel pick_epoch_batch(uint32_t M, bool sync, int prec) {
    static const EpochBatchKernel tab[2][2][3] = {
        {{k_epoch_batch<0, false, 0>, k_epoch_batch<0, false, 1>, k_epoch_batch<0, false, 2>},
         {k_epoch_batch<0, true, 0>, k_epoch_batch<0, true, 1>, k_epoch_batch<0, true, 2>}},
        {{k_epoch_batch<5, false, 0>, k_epoch_batch<5, false, 1>, k_epoch_batch<5, false, 2>},
         {k_epoch_batch<5, true, 0>, k_epoch_batch<5, true, 1>, k_epoch_batch<5, true, 2>}},
    };
    return tab[M == 5 ? 1 : 0][sync ? 1 : 0][prec];
}

static void launch_apply_batch(drg_ctx* ctx, int prec, uint32_t grid, const BatchArgs& ba) {
    if (prec == 0) launch_pdl(ctx, "k_apply_batch", k_apply_batch<0>, grid, 256, 0, ba);
    else if (prec == 1) launch_pdl(ctx, "k_apply_batch", k_apply_batch<1>, grid, 256, 0, ba);
    else launch_pdl(ctx, "k_apply_batch", k_apply_batch<2>, grid, 256, 0, ba);
}

// Many independent graphs as one job.  Every graph gets its own distance
// matrix, tables and hierarchy (graph id g in all random streams).  Levels
// run in rounds aligned at each graph's coarsest level: in round r graph g
// lays out its level L_g - r.  A round is one CUDA graph: a WHILE loop over
// the epochs whose body launches, for each sub-step run c, one batched
// k_epoch over all active graphs (and the batched apply in synchronous mode).
constexpr uint32_t kBatchPrepThreads = 8;

void layout_batch(drg_ctx* ctx, uint32_t count, const drg_graph* const* graphs, const drg_params& p,
                  const float* b_per_graph, float* const* pos) {
    check_params(p);
    DRG_CHECK(p.level_tables == 0, DRG_EUNSUPPORTED, "per-level tables are for whole runs of one graph");
    DRG_CHECK(count == 0 || (graphs && pos), DRG_EINVAL, "null argument");
    for (uint32_t g = 0; g < count; ++g) {
        DRG_CHECK(graphs[g] && pos[g], DRG_EINVAL, "null graph or position buffer");
        DRG_CHECK(!b_per_graph || b_per_graph[g] > 0.f, DRG_EINVAL, "b must be positive");
    }
    if (count == 0) return;
    std::vector<std::unique_ptr<WorkerCtx>> workers;  // outlive the tables they own (freed in free_all)
    struct GS {
        drg_dmat* d = nullptr;
        drg_hier* h = nullptr;
        uint32_t L = 0;
        DBuf<float2> buf;
        float2* cur = nullptr;
        DBuf<float2> G;
        DBuf<uint32_t> Yh;
    };
    std::vector<GS> gs(count);
    auto free_all = [&]() {
        for (auto& s : gs) {
            hier_free(s.h);
            dmat_free(s.d);
            s.h = nullptr;
            s.d = nullptr;
        }
    };
    try {
        const bool sync_mode = p.mode == DRG_MODE_SYNC;
        const int prec = p.precision;
        uint32_t Lmax = 0;
        // Distance matrices, tables and hierarchies of the graphs are
        // independent: host worker threads build them concurrently, each on
        // its own stream (sequentially when profiling, so that the phase
        // timers stay meaningful).
        const uint32_t nthreads = ctx->prof ? 1u : (count < kBatchPrepThreads ? count : kBatchPrepThreads);
        if (nthreads <= 1) {
            for (uint32_t g = 0; g < count; ++g) {
                drg_params q = p;
                q.gid = g;
                gs[g].d = build_dmat(ctx, graphs[g], p.k, p.sigma, p.perplexity, p.row_cap);
                gs[g].h = build_hierarchy(ctx, graphs[g], q);
            }
        } else {
            for (uint32_t w = 0; w < nthreads; ++w) workers.emplace_back(new WorkerCtx(ctx));
            std::atomic<uint32_t> next{0};
            std::atomic<bool> failed{false};
            std::vector<std::exception_ptr> errs(nthreads);
            std::vector<std::thread> th;
            for (uint32_t w = 0; w < nthreads; ++w) {
                th.emplace_back([&, w]() {
                    try {
                        DRG_CUDA(cudaSetDevice(ctx->device));
                        drg_ctx* wc = &workers[w]->c;
                        for (;;) {
                            const uint32_t g = next.fetch_add(1);
                            if (g >= count || failed.load()) break;
                            drg_params q = p;
                            q.gid = g;
                            gs[g].d = build_dmat(wc, graphs[g], p.k, p.sigma, p.perplexity, p.row_cap);
                            gs[g].h = build_hierarchy(wc, graphs[g], q);
                        }
                        sync(wc);
                    } catch (...) {
                        errs[w] = std::current_exception();
                        failed.store(true);
                    }
                });
            }
            for (auto& t : th) t.join();
            for (auto& w : workers) ctx->launches += w->c.launches;
            for (auto& e : errs)
                if (e) std::rethrow_exception(e);
        }
        for (uint32_t g = 0; g < count; ++g) {
            drg_params q = p;
            q.gid = g;
            gs[g].L = (uint32_t)gs[g].h->g.size() - 1;
            const uint32_t nL = gs[g].h->g[gs[g].L]->n;
            if (gs[g].L > 0) {
                gs[g].buf = DBuf<float2>(ctx, nL);
                gs[g].cur = gs[g].buf.p;
            } else {
                gs[g].cur = reinterpret_cast<float2*>(pos[g]);
            }
            init_positions(ctx, nL, gs[g].L, q, reinterpret_cast<float*>(gs[g].cur));
            Lmax = gs[g].L > Lmax ? gs[g].L : Lmax;
        }
        std::vector<float> lr_host(p.epochs);
        for (uint32_t t = 0; t < p.epochs; ++t)
            lr_host[t] = (float)((double)p.lr0 * (1.0 - (double)t / (double)p.epochs));
        DBuf<float> lr_tab(ctx, p.epochs);
        h2d(ctx, lr_tab.p, lr_host.data(), p.epochs);
        DBuf<EpochState> st(ctx, 1);
        const EpochState st_host{0u, p.epochs, lr_host[0], 0u, lr_tab.p};
        const EpochBatchKernel ek = pick_epoch_batch(p.M, sync_mode, prec);
        const EpochArgs proto = epoch_args(gs[0].d, nullptr, nullptr, p, p.gamma, 0);
        const bool one_launch = !sync_mode;  // Hogwild: one launch per round
        for (uint32_t r = 0; r <= Lmax; ++r) {
            std::vector<BatchJob> jobs;
            std::vector<HogwildArgs> runs;
            std::vector<uint32_t> bpre(1, 0), npre(1, 0), owner;
            uint64_t samples = 0;
            uint32_t max_chunks = 0;
            for (uint32_t g = 0; g < count; ++g) {
                GS& s = gs[g];
                if (s.L < r) continue;
                const uint32_t level = s.L - r;
                const uint32_t nl = s.h->g[level]->n;
                const float b = b_per_graph ? b_per_graph[g] : p.b;
                BatchJob J{};
                J.etab = s.d->etab;
                J.packed = s.d->erec_bytes == 16 ? 1 : 0;
                J.nnz = s.d->nnz;
                J.vtab = s.d->vtab;
                J.anc = level == 0 ? nullptr : s.h->anc[level];
                J.Y = s.cur;
                if (sync_mode) {
                    s.G = DBuf<float2>(ctx, nl);
                    DRG_CUDA(cudaMemsetAsync(s.G.p, 0, sizeof(float2) * nl, ctx->stream));
                    J.G = s.G.p;
                }
                if (prec) {
                    s.Yh = DBuf<uint32_t>(ctx, nl);
                    J.Yh = s.Yh.p;
                }
                J.n0 = s.d->n;
                J.nl = nl;
                J.chunk = (uint32_t)(((uint64_t)nl + p.substeps - 1) / p.substeps);
                J.tag = stream_tag(kPurposeSample, g, level);
                J.gamma = (level == s.L && s.L > 0) ? p.gamma_coarsest : p.gamma;
                J.b = b;
                J.twob = 2.f * b;
                J.bint = int_b(b);
                const uint32_t chunks = (uint32_t)(((uint64_t)nl + J.chunk - 1) / J.chunk);
                max_chunks = chunks > max_chunks ? chunks : max_chunks;
                jobs.push_back(J);
                owner.push_back(g);
                bpre.push_back(bpre.back() + (J.chunk + 255) / 256);
                npre.push_back(npre.back() + (nl + 255) / 256);
                samples += nl;
                if (one_launch) {
                    HogwildArgs h{};
                    h.a = proto;
                    h.a.etab = J.etab;
                    h.a.packed = J.packed;
                    h.a.nnz = J.nnz;
                    h.a.vtab = J.vtab;
                    h.a.n0 = J.n0;
                    h.a.anc = J.anc;
                    h.a.Y = J.Y;
                    h.a.Yh = J.Yh;
                    h.a.tag = J.tag;
                    h.a.gamma = J.gamma;
                    h.a.b = J.b;
                    h.a.twob = J.twob;
                    h.a.bint = J.bint;
                    h.lr_tab = lr_tab.p;
                    h.t_begin = 0;
                    h.epochs = p.epochs;
                    h.T = J.chunk;
                    h.nl = nl;
                    runs.push_back(h);
                }
            }
            const uint32_t njobs = (uint32_t)jobs.size();
            if (one_launch) {
                if (prec) {  // first half copies of every run
                    for (const auto& h : runs) {
                        const uint32_t gn = grid_for(h.nl, 256, (uint32_t)ctx->num_sms * 8);
                        if (prec == 1) DRG_LAUNCH(ctx, k_refresh<1>, gn, 256, 0, h.a.Y, const_cast<void*>(h.a.Yh), h.nl);
                        else DRG_LAUNCH(ctx, k_refresh<2>, gn, 256, 0, h.a.Y, const_cast<void*>(h.a.Yh), h.nl);
                    }
                }
                hogwild_batch(ctx, p.M, prec, runs, p.epochs, samples * p.epochs);
            } else {
                DBuf<BatchJob> djobs(ctx, njobs);
                DBuf<uint32_t> dbpre(ctx, njobs + 1), dnpre(ctx, njobs + 1);
                h2d(ctx, djobs.p, jobs.data(), njobs);
                h2d(ctx, dbpre.p, bpre.data(), njobs + 1);
                h2d(ctx, dnpre.p, npre.data(), njobs + 1);
                BatchArgs ba{};
                ba.common = proto;
                ba.common.st = st.p;
                ba.jobs = djobs.p;
                ba.block_prefix = dbpre.p;
                ba.node_prefix = dnpre.p;
                ba.njobs = njobs;
                h2d(ctx, st.p, &st_host, 1);
                if (prec) launch_apply_batch(ctx, prec, npre.back(), ba);  // first half copies (G is zero)
                auto epoch_body = [&]() {
                    for (uint32_t c = 0; c < max_chunks; ++c) {
                        BatchArgs bc = ba;
                        bc.common.late = c == 0 ? 1 : 0;
                        launch_pdl(ctx, "k_epoch_batch", ek, bpre.back(), 256, 0, bc, c);
                        if (sync_mode) launch_apply_batch(ctx, prec, npre.back(), ba);
                    }
                    if (!sync_mode && prec) launch_apply_batch(ctx, prec, npre.back(), ba);
                };
                const uint64_t per_epoch = (uint64_t)max_chunks * (sync_mode ? 2 : 1) + 1 + (!sync_mode && prec ? 1 : 0);
                if (ctx->direct_launch) {
                    ProfSpan span(ctx, DRG_PROF_EPOCH, samples * p.epochs, (uint64_t)p.epochs * max_chunks);
                    for (uint32_t t = 0; t < p.epochs; ++t) {
                        DRG_LAUNCH(ctx, k_set_epoch, 1, 1, 0, st.p, t, p.epochs, lr_host[t]);
                        epoch_body();
                    }
                } else {
                    run_epoch_loop_graph(ctx, st.p, epoch_body, (uint64_t)p.epochs * per_epoch, samples * p.epochs,
                                         (uint64_t)p.epochs * max_chunks);
                }
            }
            sync(ctx);
            // refinement of every graph whose level was not its finest
            for (uint32_t x = 0; x < njobs; ++x) {
                GS& s = gs[owner[x]];
                const uint32_t level = s.L - r;
                s.G.reset();
                s.Yh.reset();
                if (level == 0) continue;
                const uint32_t nf = s.h->g[level - 1]->n;
                DBuf<float2> nb;
                float2* fine = reinterpret_cast<float2*>(pos[owner[x]]);
                if (level - 1 > 0) {
                    nb = DBuf<float2>(ctx, nf);
                    fine = nb.p;
                }
                DRG_LAUNCH(ctx, k_interp, grid_for(nf, 256, (uint32_t)ctx->num_sms * 8), 256, 0, s.cur,
                           s.h->parent[level - 1], fine, nf);
                s.buf = std::move(nb);
                s.cur = fine;
            }
        }
        sync(ctx);
    } catch (...) {
        // tables owned by worker contexts are freed on their streams: let the
        // main stream finish with them first
        cudaStreamSynchronize(ctx->stream);
        (void)cudaGetLastError();
        free_all();
        throw;
    }
    free_all();
}

// ------------------------------------------------------------------ allocation-free level run
// A variant of the synchronous FP32 level run for callers that must not
// allocate device memory.  Its scratch -- the epoch state (first 256 bytes)
// and the gradient accumulator, one float2 per node -- is a file-scope
// device array that every GPU loading this library holds until the process
// exits.  Host code cannot use the array's name as a device address, so the
// first call on each device looks the address up with cudaGetSymbolAddress
// (that device current) and keeps it together with the id of the CUDA context
// it was read in; a call in another context (the primary context reset and
// created again, which reloads the module) looks it up again.
constexpr uint32_t kNoAllocMaxNodes = 1u << 20;
constexpr uint32_t kNoAllocStateSlots = 32;  // 256 bytes reserved for the EpochState
static __device__ __align__(256) float2 g_noalloc_scratch[kNoAllocStateSlots + kNoAllocMaxNodes];

static_assert(sizeof(EpochState) <= kNoAllocStateSlots * sizeof(float2), "epoch state does not fit its slot");


// Unique id of the calling thread's current CUDA context (driver entry points
// reached through the runtime, so the library needs no link to libcuda); 0
// when the driver cannot say.
static unsigned long long current_context_id() {
    typedef CUresult (*GetCurrent)(CUcontext*);
    typedef CUresult (*GetId)(CUcontext, unsigned long long*);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, []() {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrent>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(f);
        (void)cudaGetLastError();
    });
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS) return 0;
    return id;
}

static float2* noalloc_scratch(drg_ctx* ctx) {
    static std::mutex mu;
    static void* addr[256] = {};
    static unsigned long long ctx_id[256] = {};
    DRG_CHECK(ctx->device >= 0 && ctx->device < 256, DRG_EUNSUPPORTED, "device index beyond 255");
    std::lock_guard<std::mutex> lock(mu);
    int prev = 0;
    DRG_CUDA(cudaGetDevice(&prev));
    DRG_CUDA(cudaSetDevice(ctx->device));
    const unsigned long long id = current_context_id();
    // 0: the context cannot be identified, so the address is looked up on every call
    if (!addr[ctx->device] || id == 0 || id != ctx_id[ctx->device]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) {
            cudaSetDevice(prev);
            fail(DRG_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        }
        addr[ctx->device] = p;
        ctx_id[ctx->device] = id;
    }
    DRG_CUDA(cudaSetDevice(prev));
    return static_cast<float2*>(addr[ctx->device]);
}

void layout_level_noalloc(drg_ctx* ctx, const drg_dmat* d, const drg_hier* h, uint32_t level, float* pos,
                          const drg_params& p, float gamma, uint32_t t_begin, uint32_t t_end) {
    check_params(p);
    DRG_CHECK(d && pos, DRG_EINVAL, "null distance matrix or positions");
    DRG_CHECK(level == 0 || (h && level < h->g.size()), DRG_EINVAL, "level out of range");
    DRG_CHECK(t_begin <= t_end && t_end <= p.epochs, DRG_EINVAL, "epoch range outside [0, epochs]");
    // as in layout_level: d is G^0's matrix (samples mapped to the level) or,
    // at a coarse level, the level graph's own (no mapping)
    const bool own = level > 0 && h && d->n != h->g[0]->n && d->n == h->g[level]->n;
    DRG_CHECK(!h || own || h->g[0]->n == d->n, DRG_EINVAL, "hierarchy and distance matrix describe different graphs");
    DRG_CHECK(p.mode == DRG_MODE_SYNC && p.precision == DRG_PREC_FP32, DRG_EUNSUPPORTED,
              "the allocation-free run supports synchronous FP32 mode only");
    const uint32_t nl = level == 0 ? d->n : h->g[level]->n;
    DRG_CHECK(nl <= kNoAllocMaxNodes, DRG_EUNSUPPORTED,
              "the allocation-free run is limited to 1048576 nodes per level (its static scratch)");
    float2* scratch = noalloc_scratch(ctx);
    EpochState* st = reinterpret_cast<EpochState*>(scratch);
    float2* G = scratch + kNoAllocStateSlots;
    float2* Y = reinterpret_cast<float2*>(pos);
    // the array keeps the previous call's contents: the gradient must start at zero
    DRG_CUDA(cudaMemsetAsync(G, 0, sizeof(float2) * (size_t)nl, ctx->stream));
    EpochArgs a = epoch_args(d, (level == 0 || own) ? nullptr : h->anc[level], Y, p, gamma, level);
    a.G = G;
    a.st = st;
    const EpochKernel ek = pick_epoch(p.M, true, DRG_PREC_FP32);
    const uint32_t chunk = (uint32_t)(((uint64_t)nl + p.substeps - 1) / p.substeps);
    const uint32_t gn = grid_for(nl, 256, (uint32_t)ctx->num_sms * 8);
    for (uint32_t t = t_begin; t < t_end; ++t) {
        const float lr = (float)((double)p.lr0 * (1.0 - (double)t / (double)p.epochs));
        DRG_LAUNCH(ctx, k_set_epoch, 1, 1, 0, st, t, t_end, lr);
        for (uint64_t s0 = 0; s0 < nl; s0 += chunk) {
            a.s_begin = s0;
            a.s_end = s0 + chunk < nl ? s0 + chunk : nl;
            a.late = s0 == 0 ? 1 : 0;
            launch_pdl(ctx, "k_epoch", ek, epoch_grid(ctx, a.s_end - a.s_begin), 256, 0, a);
            launch_pdl(ctx, "k_apply", k_apply<0>, gn, 256, 0, Y, G, (void*)nullptr, nl, (const EpochState*)st);
        }
    }
}

}  // namespace drg
