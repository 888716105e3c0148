// Internal declarations shared by the CUDA translation units of libdrgraph.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>

#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/drgraph.h"

namespace drg {

typedef unsigned __int128 u128;

constexpr uint32_t kNone = 0xFFFFFFFFu;
constexpr uint32_t kPurposeSample = 0, kPurposeInit = 1, kPurposeMatch = 2, kPurposeStar = 3;

// ------------------------------------------------------------------ errors
struct Error {
    drg_status status;
    std::string msg;
};

[[noreturn]] inline void fail(drg_status s, const std::string& msg) { throw Error{s, msg}; }

#define DRG_CUDA(call)                                                                         \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            ::drg::fail(e_ == cudaErrorMemoryAllocation ? DRG_ENOMEM : DRG_ECUDA,              \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                   \
    } while (0)

#define DRG_CHECK(cond, status, msg)          \
    do {                                              \
        if (!(cond)) ::drg::fail((status), (msg));  \
    } while (0)

}  // namespace drg

// ------------------------------------------------------------------ handles
struct drg_prof_span {
    cudaEvent_t start, stop;
    int which;
    uint64_t units, count;
};

struct drg_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int num_sms = 0;
    int max_smem_optin = 0;
    std::string err;
    uint64_t launches = 0;
    bool direct_launch = false;             // DRG_DIRECT_LAUNCH=1: no level graphs (for profilers)
    bool autotune = true;                   // tune the Hogwild kernels' launch shape (drg_autotune_enable)
    int64_t bfs_stage_limit = -1;           // DRG_BFS_STAGE_LIMIT=<entries>: cap the k-order staging
                                            // area (rows past it take the direct traversal); -1: none
    // profiling (drg_profile_*)
    bool prof = false;
    std::vector<drg_prof_span> spans;       // recorded, not yet read
    std::vector<cudaEvent_t> free_events;
    double prof_ms[DRG_PROF_COUNT] = {};
    uint64_t prof_launches[DRG_PROF_COUNT] = {};
    uint64_t prof_units[DRG_PROF_COUNT] = {};
};

struct drg_graph {
    drg_ctx* ctx = nullptr;
    uint32_t n = 0;
    uint64_t nnz = 0;
    uint64_t* rp = nullptr;  // [n + 1]
    uint32_t* col = nullptr; // [nnz]
    uint32_t* w = nullptr;   // [nnz], nullptr = all ones
};

// One bucket of the edge alias table: the acceptance threshold and the
// endpoints of the bucket's own entry and of its alias entry.  Graphs with
// fewer than 2^24 nodes use the packed 16-byte form (one 16-byte load per
// draw): {thresh, i0 | j0 << 24, j0 >> 8 | i1 << 16, i1 >> 16 | j1 << 8}.
// Larger graphs use this 32-byte form, aligned so that a draw reads one
// 32-byte sector.
struct __align__(32) EdgeRec {
    uint32_t thresh, i0, j0, i1, j1, pad0, pad1, pad2;
};

constexpr uint32_t kPackedIdLimit = 1u << 24;  // node ids of packed edge records

__host__ __device__ __forceinline__ uint4 pack_edge16(uint32_t thresh, uint32_t i0, uint32_t j0, uint32_t i1,
                                                      uint32_t j1) {
    return make_uint4(thresh, i0 | (j0 << 24), (j0 >> 8) | (i1 << 16), (i1 >> 16) | (j1 << 8));
}

struct drg_dmat {
    drg_ctx* ctx = nullptr;
    uint32_t n = 0, k = 0;
    uint64_t nnz = 0;
    float sigma = 1.f;
    float perplexity = 0.f;      // > 0: sigma_i calibrated per node (beta below)
    uint32_t row_cap = 0;        // > 0: rows capped to their row_cap nearest nodes, pattern K u K^T
    uint32_t shift = 0;
    uint64_t* rp = nullptr;      // [n + 1]
    uint32_t* col = nullptr;     // [nnz]
    uint8_t* dist = nullptr;     // [nnz]
    uint32_t* q = nullptr;       // [nnz]
    uint64_t* r = nullptr;       // [n]
    float* Z = nullptr;          // [n]
    void* etab = nullptr;        // [nnz] edge records: packed 16-byte (erec_bytes 16) or EdgeRec (32)
    uint32_t erec_bytes = 32;
    uint2* vtab = nullptr;       // [n] {thresh, alias}
    double* beta = nullptr;      // [n] 1/(2 sigma_i^2) when calibrated
};

struct drg_hier {
    drg_ctx* ctx = nullptr;
    std::vector<const drg_graph*> g;   // g[0] borrowed, others owned
    std::vector<drg_graph*> owned;
    std::vector<uint32_t*> parent;     // [L-1], level l -> l+1
    std::vector<uint32_t*> anc;        // [L], anc[0] = nullptr (identity)
};

namespace drg {

// ------------------------------------------------------------------ device memory
void* dalloc(drg_ctx* ctx, size_t bytes);
void dfree(drg_ctx* ctx, void* p);

template <typename T>
struct DBuf {
    drg_ctx* ctx = nullptr;
    T* p = nullptr;
    size_t n = 0;
    DBuf() = default;
    DBuf(drg_ctx* c, size_t count) : ctx(c), n(count) { p = static_cast<T*>(dalloc(c, (count ? count : 1) * sizeof(T))); }
    DBuf(const DBuf&) = delete;
    DBuf& operator=(const DBuf&) = delete;
    DBuf(DBuf&& o) noexcept : ctx(o.ctx), p(o.p), n(o.n) { o.p = nullptr; }
    DBuf& operator=(DBuf&& o) noexcept {
        reset();
        ctx = o.ctx; p = o.p; n = o.n; o.p = nullptr;
        return *this;
    }
    ~DBuf() { reset(); }
    void reset() {
        if (p) dfree(ctx, p);
        p = nullptr;
    }
    T* release() { T* q = p; p = nullptr; return q; }
    T* get() const { return p; }
};

// Launch accounting: every kernel launch of the library goes through here.
void after_launch(drg_ctx* ctx, const char* name);

// Profiling spans: an NVTX range always (free unless a tool listens), CUDA
// events on the context stream when profiling is enabled on the context.
struct ProfSpan {
    drg_ctx* ctx;
    int which;
    uint64_t units, count;
    cudaEvent_t start = nullptr;
    bool nvtx_open = false;
    ProfSpan(drg_ctx* c, int w, uint64_t u, uint64_t launches = 1);
    ~ProfSpan() { close(); }
    void close();                          // end the span now (idempotent)
    void reopen(int w, uint64_t u);        // end it and start a new one
    ProfSpan(const ProfSpan&) = delete;
    ProfSpan& operator=(const ProfSpan&) = delete;
};
void prof_collect(drg_ctx* ctx);

template <typename... KArgs, typename... Args>
inline void launch_k(drg_ctx* ctx, const char* name, void (*kernel)(KArgs...), uint32_t grid, uint32_t block,
                     size_t smem, Args&&... args) {
    if (grid == 0) return;
    kernel<<<grid, block, smem, ctx->stream>>>(static_cast<KArgs>(args)...);
    after_launch(ctx, name);
}

#define DRG_LAUNCH(ctx, kernel, grid, block, smem, ...) \
    ::drg::launch_k((ctx), #kernel, kernel, (uint32_t)(grid), (uint32_t)(block), (size_t)(smem), __VA_ARGS__)

// Programmatic dependent launch: the kernel may start while the previous
// kernel of the stream is still running; it must call grid_dependency_wait()
// before touching anything that kernel writes.
template <typename... KArgs, typename... Args>
inline void launch_pdl(drg_ctx* ctx, const char* name, void (*kernel)(KArgs...), uint32_t grid, uint32_t block,
                       size_t smem, Args&&... args) {
    if (grid == 0) return;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = ctx->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
    if (e != cudaSuccess) fail(DRG_ECUDA, std::string("launch of ") + name + ": " + cudaGetErrorString(e));
    after_launch(ctx, name);
}

// Let the next kernel of the stream start its prologue now.
__device__ __forceinline__ void grid_dependency_trigger() { asm volatile("griddepcontrol.launch_dependents;"); }
// Wait until the previous kernel of the stream has finished and its writes are visible.
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename T>
inline void h2d(drg_ctx* ctx, T* dst, const T* src, size_t n) {
    if (n) DRG_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(T), cudaMemcpyHostToDevice, ctx->stream));
}
template <typename T>
inline void d2h(drg_ctx* ctx, T* dst, const T* src, size_t n) {
    if (n) DRG_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(T), cudaMemcpyDeviceToHost, ctx->stream));
}
template <typename T>
inline void d2d(drg_ctx* ctx, T* dst, const T* src, size_t n) {
    if (n) DRG_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(T), cudaMemcpyDeviceToDevice, ctx->stream));
}
template <typename T>
inline T read1(drg_ctx* ctx, const T* src) {
    T v;
    DRG_CUDA(cudaMemcpyAsync(&v, src, sizeof(T), cudaMemcpyDeviceToHost, ctx->stream));
    DRG_CUDA(cudaStreamSynchronize(ctx->stream));
    return v;
}
inline void sync(drg_ctx* ctx) { DRG_CUDA(cudaStreamSynchronize(ctx->stream)); }

inline uint32_t grid_for(size_t n, uint32_t threads, uint32_t cap = 1u << 20) {
    size_t g = (n + threads - 1) / threads;
    return (uint32_t)(g < cap ? g : cap);
}

// ------------------------------------------------------------------ Philox4x32-10
// Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3"
// (SC'11): ten rounds; each round multiplies counter words 0 and 2 by the
// Philox constants, mixes the high halves with words 1 and 3 and the key;
// the key is bumped by the golden-ratio Weyl constants between rounds.
__host__ __device__ __forceinline__ uint4 philox(uint4 c, uint2 k) {
#ifdef __CUDA_ARCH__
#pragma unroll
#endif
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
#ifdef __CUDA_ARCH__
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
#else
        const uint64_t p0 = (uint64_t)0xD2511F53u * c.x, p1 = (uint64_t)0xCD9E8D57u * c.z;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
#endif
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// Third counter word: purpose | graph id | level.
__host__ __device__ __forceinline__ uint32_t stream_tag(uint32_t purpose, uint32_t gid, uint32_t level) {
    return (purpose << 28) | ((gid & 0xFFFFFu) << 8) | (level & 0xFFu);
}

__host__ __device__ __forceinline__ uint2 seed_key(uint64_t seed) {
    return make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
}

// Alias draw: bucket = floor(R * N / 2^64); keep the bucket when U < thresh.
__device__ __forceinline__ uint64_t alias_bucket(uint64_t R, uint64_t N) { return __umul64hi(R, N); }

// ------------------------------------------------------------------ internal entry points
void build_csr_from_keys(drg_ctx* ctx, uint32_t n, uint64_t* keys, uint32_t* vals, size_t count,
                         drg_graph* out);
drg_graph* graph_from_edges(drg_ctx* ctx, uint32_t n, uint64_t m, const uint32_t* src, const uint32_t* dst,
                            bool on_device);
void graph_free(drg_graph* g);
drg_dmat* build_dmat(drg_ctx* ctx, const drg_graph* g, uint32_t k, float sigma, float perplexity = 0.f,
                     uint32_t row_cap = 0);
void crossings(drg_ctx* ctx, const drg_graph* g, const float* pos, uint64_t* c, double* crosslessness);
double min_angle(drg_ctx* ctx, const drg_graph* g, const float* pos);
void dmat_free(drg_dmat* d);
void edge_alias_ids(drg_ctx* ctx, const drg_dmat* d, uint64_t e0, uint64_t e1, uint32_t* host_out);
drg_graph* coarsen(drg_ctx* ctx, const drg_graph* fine, uint32_t level, const drg_params& p, uint32_t* parent);
drg_hier* build_hierarchy(drg_ctx* ctx, const drg_graph* g0, const drg_params& p);
void hier_free(drg_hier* h);
void check_params(const drg_params& p);
void init_positions(drg_ctx* ctx, uint32_t n, uint32_t level, const drg_params& p, float* pos);
void layout_level(drg_ctx* ctx, const drg_dmat* d, const drg_hier* h, uint32_t level, float* pos,
                  const drg_params& p, float gamma, uint32_t t_begin, uint32_t t_end);
void check_epoch_barrier(drg_ctx* ctx, uint32_t blocks, uint32_t arrivals, uint32_t rounds, uint32_t timeout_ms);
void layout_level_noalloc(drg_ctx* ctx, const drg_dmat* d, const drg_hier* h, uint32_t level, float* pos,
                          const drg_params& p, float gamma, uint32_t t_begin, uint32_t t_end);
void interpolate(drg_ctx* ctx, const drg_hier* h, uint32_t coarse_level, const float* coarse_pos, float* fine_pos);
void layout_full(drg_ctx* ctx, const drg_graph* g, const drg_params& p, float* pos);
void layout_batch(drg_ctx* ctx, uint32_t count, const drg_graph* const* graphs, const drg_params& p,
                  const float* b_per_graph, float* const* pos);
void sample_draws(drg_ctx* ctx, const drg_dmat* d, uint32_t level, uint32_t t, uint32_t s_begin, uint32_t s_end,
                  const drg_params& p, uint32_t* oi, uint32_t* oj, uint32_t* oneg);
uint32_t autotune_read(uint32_t cap, uint32_t* keys, uint32_t* choice, float* ms);
void autotune_clear();
void layout_step_explicit(drg_ctx* ctx, uint32_t n, float* pos, uint32_t S, const uint32_t* sa, const uint32_t* sc,
                          const uint32_t* sneg, uint32_t M, float gamma, float b, float lr, float clip);
void probe_memory(drg_ctx* ctx, int kind, uint64_t bytes, uint64_t accesses, uint32_t blocks_per_sm, double* ms,
                  uint64_t* done);

}  // namespace drg
