// extern "C" entry points of libdrgraph (declared in include/drgraph.h).
// Each one validates its arguments, runs the internal implementation and
// turns any failure into a status code plus the context's error message.
#include "prims.cuh"

#include <nvtx3/nvToolsExt.h>

#include <chrono>
#include <cstdlib>
#include <new>

namespace drg {

void* dalloc(drg_ctx* ctx, size_t bytes) {
    void* p = nullptr;
    const auto t0 = std::chrono::steady_clock::now();
    cudaError_t e = cudaMallocAsync(&p, bytes ? bytes : 1, ctx->stream);
    if (ctx->prof) {
        ctx->prof_ms[DRG_PROF_ALLOC] +=
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        ctx->prof_launches[DRG_PROF_ALLOC] += 1;
        ctx->prof_units[DRG_PROF_ALLOC] += bytes;
    }
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        fail(e == cudaErrorMemoryAllocation ? DRG_ENOMEM : DRG_ECUDA,
             std::string("device allocation of ") + std::to_string(bytes) + " bytes: " + cudaGetErrorString(e));
    }
    return p;
}

void dfree(drg_ctx* ctx, void* p) {
    if (p) (void)cudaFreeAsync(p, ctx->stream);
}

static cudaEvent_t take_event(drg_ctx* ctx) {
    if (!ctx->free_events.empty()) {
        cudaEvent_t e = ctx->free_events.back();
        ctx->free_events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    DRG_CUDA(cudaEventCreate(&e));
    return e;
}

static const char* const kSpanNames[DRG_PROF_COUNT] = {
    "drg level runs", "drg sync apply", "drg distance matrix", "drg hierarchy", "drg graph",
    "drg k-order traversal", "drg similarity", "drg alias tables", "drg host allocations"};

static void nvtx_push(int which) {
    nvtxRangePushA(which >= 0 && which < DRG_PROF_COUNT ? kSpanNames[which] : "drg");
}

ProfSpan::ProfSpan(drg_ctx* c, int w, uint64_t u, uint64_t launches) : ctx(c), which(w), units(u), count(launches) {
    nvtx_push(which);
    nvtx_open = true;
    if (!ctx->prof) return;
    start = take_event(ctx);
    DRG_CUDA(cudaEventRecord(start, ctx->stream));
}

void ProfSpan::close() {
    if (nvtx_open) {
        nvtxRangePop();
        nvtx_open = false;
    }
    if (!start) return;
    cudaEvent_t stop = nullptr;
    if (!ctx->free_events.empty()) {
        stop = ctx->free_events.back();
        ctx->free_events.pop_back();
    } else if (cudaEventCreate(&stop) != cudaSuccess) {
        ctx->free_events.push_back(start);
        start = nullptr;
        return;
    }
    cudaEventRecord(stop, ctx->stream);
    ctx->spans.push_back(drg_prof_span{start, stop, which, units, count});
    start = nullptr;
}

void ProfSpan::reopen(int w, uint64_t u) {
    close();
    which = w;
    units = u;
    count = 1;
    nvtx_push(which);
    nvtx_open = true;
    if (!ctx->prof) return;
    start = take_event(ctx);
    DRG_CUDA(cudaEventRecord(start, ctx->stream));
}

void prof_collect(drg_ctx* ctx) {
    for (auto& sp : ctx->spans) {
        float ms = 0.f;
        DRG_CUDA(cudaEventSynchronize(sp.stop));
        DRG_CUDA(cudaEventElapsedTime(&ms, sp.start, sp.stop));
        ctx->prof_ms[sp.which] += ms;
        ctx->prof_launches[sp.which] += sp.count;
        ctx->prof_units[sp.which] += sp.units;
        ctx->free_events.push_back(sp.start);
        ctx->free_events.push_back(sp.stop);
    }
    ctx->spans.clear();
}

void after_launch(drg_ctx* ctx, const char* name) {
    ++ctx->launches;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) fail(DRG_ECUDA, std::string("launch of ") + name + ": " + cudaGetErrorString(e));
}

}  // namespace drg

using drg::Error;

#define API_TRY try {
#define API_CATCH(ctxp)                                                   \
    }                                                                     \
    catch (const Error& e) {                                              \
        if (ctxp) (ctxp)->err = e.msg;                                    \
        return e.status;                                                  \
    }                                                                     \
    catch (const std::bad_alloc&) {                                       \
        if (ctxp) (ctxp)->err = "host allocation failed";                 \
        return DRG_ENOMEM;                                                \
    }                                                                     \
    catch (...) {                                                         \
        if (ctxp) (ctxp)->err = "unexpected internal error";              \
        return DRG_ECUDA;                                                 \
    }                                                                     \
    if (ctxp) (ctxp)->err.clear();                                        \
    return DRG_OK;

extern "C" {

void drg_params_default(drg_params* p) {
    if (!p) return;
    p->k = 1;
    p->M = 5;
    p->epochs = 400;
    p->gamma = 0.1f;
    p->gamma_coarsest = 0.01f;
    p->b = 1.0f;
    p->lr0 = 1.0f;
    p->sigma = 1.0f;
    p->clip = 5.0f;
    p->init_scale = 1e-4f;
    p->rho = 0.8f;
    p->seed = 0;
    p->gid = 0;
    p->mode = DRG_MODE_SYNC;
    p->precision = DRG_PREC_FP32;
    p->substeps = 16;
    p->stop_nodes = 1000;
    p->match_rounds = 8;
    p->max_levels = 32;
    p->multilevel = 1;
    p->coarsen = DRG_COARSEN_HEM;
    p->level_tables = 0;
    p->perplexity = 0.f;
    p->row_cap = 0;
}

const char* drg_status_string(drg_status s) {
    switch (s) {
        case DRG_OK: return "ok";
        case DRG_EINVAL: return "invalid argument";
        case DRG_ENOMEM: return "out of memory";
        case DRG_ECUDA: return "CUDA error";
        case DRG_ETIMEOUT: return "device wait timed out";
        case DRG_EUNSUPPORTED: return "unsupported size";
        case DRG_EEMPTY: return "graph has no edges";
    }
    return "unknown status";
}

drg_status drg_create(drg_ctx** out, int device, void* stream) {
    if (!out) return DRG_EINVAL;
    *out = nullptr;
    drg_ctx* c = nullptr;
    API_TRY
    c = new drg_ctx();
    c->device = device;
    {
        const char* env = std::getenv("DRG_DIRECT_LAUNCH");
        c->direct_launch = env && env[0] == '1';
        const char* lim = std::getenv("DRG_BFS_STAGE_LIMIT");
        if (lim && lim[0]) c->bfs_stage_limit = std::strtoll(lim, nullptr, 10);
    }
    DRG_CUDA(cudaSetDevice(device));
    DRG_CUDA(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device));
    DRG_CUDA(cudaDeviceGetAttribute(&c->max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
    if (stream) {
        c->stream = static_cast<cudaStream_t>(stream);
    } else {
        DRG_CUDA(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
        c->own_stream = true;
    }
    // keep freed stream-ordered memory cached in the pool between calls
    cudaMemPool_t pool;
    DRG_CUDA(cudaDeviceGetDefaultMemPool(&pool, device));
    uint64_t thresh = ~0ull;
    DRG_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thresh));
    *out = c;
    }
    catch (const Error& e) {
        delete c;
        return e.status;
    }
    catch (...) {
        delete c;
        return DRG_ECUDA;
    }
    return DRG_OK;
}

drg_status drg_destroy(drg_ctx* ctx) {
    if (!ctx) return DRG_EINVAL;
    cudaStreamSynchronize(ctx->stream);
    for (auto& sp : ctx->spans) {
        cudaEventDestroy(sp.start);
        cudaEventDestroy(sp.stop);
    }
    for (auto e : ctx->free_events) cudaEventDestroy(e);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return DRG_OK;
}

drg_status drg_synchronize(drg_ctx* ctx) {
    if (!ctx) return DRG_EINVAL;
    API_TRY
    drg::sync(ctx);
    API_CATCH(ctx)
}

const char* drg_last_error(const drg_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

uint64_t drg_kernel_launches(const drg_ctx* ctx) { return ctx ? ctx->launches : 0; }

drg_status drg_profile_enable(drg_ctx* ctx, int on) {
    if (!ctx) return DRG_EINVAL;
    ctx->prof = on != 0;
    return DRG_OK;
}

drg_status drg_profile_reset(drg_ctx* ctx) {
    if (!ctx) return DRG_EINVAL;
    API_TRY
    drg::prof_collect(ctx);
    for (int w = 0; w < DRG_PROF_COUNT; ++w) {
        ctx->prof_ms[w] = 0;
        ctx->prof_launches[w] = 0;
        ctx->prof_units[w] = 0;
    }
    API_CATCH(ctx)
}

drg_status drg_profile_read(drg_ctx* ctx, int which, double* ms, uint64_t* launches, uint64_t* units) {
    if (!ctx || which < 0 || which >= DRG_PROF_COUNT) return DRG_EINVAL;
    API_TRY
    drg::prof_collect(ctx);
    if (ms) *ms = ctx->prof_ms[which];
    if (launches) *launches = ctx->prof_launches[which];
    if (units) *units = ctx->prof_units[which];
    API_CATCH(ctx)
}

// ---------------------------------------------------------------- graphs
drg_status drg_graph_from_edges(drg_ctx* ctx, uint32_t n, uint64_t m, const uint32_t* src, const uint32_t* dst,
                                int on_device, drg_graph** out) {
    if (!ctx || !out) return DRG_EINVAL;
    *out = nullptr;
    API_TRY
    *out = drg::graph_from_edges(ctx, n, m, src, dst, on_device != 0);
    API_CATCH(ctx)
}

drg_status drg_graph_info(const drg_graph* g, uint32_t* n, uint64_t* nnz) {
    if (!g) return DRG_EINVAL;
    if (n) *n = g->n;
    if (nnz) *nnz = g->nnz;
    return DRG_OK;
}

drg_status drg_graph_download(drg_ctx* ctx, const drg_graph* g, uint64_t* rp, uint32_t* col, uint32_t* w) {
    if (!ctx || !g) return DRG_EINVAL;
    API_TRY
    if (rp) drg::d2h(ctx, rp, g->rp, (size_t)g->n + 1);
    if (col) drg::d2h(ctx, col, g->col, g->nnz);
    if (w) {
        if (g->w) {
            drg::d2h(ctx, w, g->w, g->nnz);
        } else {
            for (uint64_t e = 0; e < g->nnz; ++e) w[e] = 1;
        }
    }
    drg::sync(ctx);
    API_CATCH(ctx)
}

drg_status drg_graph_destroy(drg_graph* g) {
    if (!g) return DRG_EINVAL;
    drg::graph_free(g);
    return DRG_OK;
}

// ---------------------------------------------------------------- distance matrix
drg_status drg_build_distance_matrix(drg_ctx* ctx, const drg_graph* g, uint32_t k, float sigma, drg_dmat** out) {
    if (!ctx || !g || !out) return DRG_EINVAL;
    *out = nullptr;
    API_TRY
    *out = drg::build_dmat(ctx, g, k, sigma);
    API_CATCH(ctx)
}

drg_status drg_build_distance_matrix_ex(drg_ctx* ctx, const drg_graph* g, uint32_t k, float sigma, float perplexity,
                                        drg_dmat** out) {
    if (!ctx || !g || !out) return DRG_EINVAL;
    *out = nullptr;
    API_TRY
    *out = drg::build_dmat(ctx, g, k, sigma, perplexity);
    API_CATCH(ctx)
}

drg_status drg_build_distance_matrix_capped(drg_ctx* ctx, const drg_graph* g, uint32_t k, float sigma,
                                            uint32_t row_cap, drg_dmat** out) {
    if (!ctx || !g || !out || row_cap == 0) return DRG_EINVAL;
    *out = nullptr;
    API_TRY
    *out = drg::build_dmat(ctx, g, k, sigma, 0.f, row_cap);
    API_CATCH(ctx)
}

drg_status drg_crossings(drg_ctx* ctx, const drg_graph* g, const float* pos, uint64_t* crossings,
                         double* crosslessness) {
    if (!ctx || !g || !pos || !crossings || !crosslessness) return DRG_EINVAL;
    API_TRY
    drg::crossings(ctx, g, pos, crossings, crosslessness);
    API_CATCH(ctx)
}

drg_status drg_min_angle(drg_ctx* ctx, const drg_graph* g, const float* pos, double* min_angle) {
    if (!ctx || !g || !pos || !min_angle) return DRG_EINVAL;
    API_TRY
    *min_angle = drg::min_angle(ctx, g, pos);
    API_CATCH(ctx)
}

drg_status drg_dmat_calibration(drg_ctx* ctx, const drg_dmat* d, double* beta) {
    if (!ctx || !d || !beta) return DRG_EINVAL;
    API_TRY
    DRG_CHECK(d->beta, DRG_EINVAL, "the matrix was built with a global sigma");
    DRG_CUDA(cudaMemcpyAsync(beta, d->beta, sizeof(double) * d->n, cudaMemcpyDeviceToHost, ctx->stream));
    drg::sync(ctx);
    API_CATCH(ctx)
}

drg_status drg_dmat_info(const drg_dmat* d, uint32_t* n, uint64_t* nnz, uint32_t* node_shift) {
    if (!d) return DRG_EINVAL;
    if (n) *n = d->n;
    if (nnz) *nnz = d->nnz;
    if (node_shift) *node_shift = d->shift;
    return DRG_OK;
}

drg_status drg_dmat_download(drg_ctx* ctx, const drg_dmat* d, uint64_t* rp, uint32_t* col, uint8_t* dist,
                             uint32_t* q, uint64_t* r, float* Z, uint32_t* e_thresh, uint32_t* e_alias,
                             uint32_t* v_thresh, uint32_t* v_alias) {
    if (!ctx || !d) return DRG_EINVAL;
    API_TRY
    if (rp) drg::d2h(ctx, rp, d->rp, (size_t)d->n + 1);
    if (col) drg::d2h(ctx, col, d->col, d->nnz);
    if (dist) drg::d2h(ctx, dist, d->dist, d->nnz);
    if (q) drg::d2h(ctx, q, d->q, d->nnz);
    if (r) drg::d2h(ctx, r, d->r, d->n);
    if (Z) drg::d2h(ctx, Z, d->Z, d->n);
    if (e_alias) drg::edge_alias_ids(ctx, d, 0, d->nnz, e_alias);
    if (e_thresh) {
        DRG_CUDA(cudaMemcpy2DAsync(e_thresh, sizeof(uint32_t), d->etab, d->erec_bytes, sizeof(uint32_t), d->nnz,
                                   cudaMemcpyDeviceToHost, ctx->stream));
    }
    if (v_thresh)
        DRG_CUDA(cudaMemcpy2DAsync(v_thresh, sizeof(uint32_t), d->vtab, sizeof(uint2), sizeof(uint32_t), d->n,
                                   cudaMemcpyDeviceToHost, ctx->stream));
    if (v_alias)
        DRG_CUDA(cudaMemcpy2DAsync(v_alias, sizeof(uint32_t), reinterpret_cast<const char*>(d->vtab) + 4, sizeof(uint2),
                                   sizeof(uint32_t), d->n, cudaMemcpyDeviceToHost, ctx->stream));
    drg::sync(ctx);
    API_CATCH(ctx)
}

drg_status drg_dmat_download_range(drg_ctx* ctx, const drg_dmat* d, uint64_t e_begin, uint64_t e_end, uint32_t* col,
                                   uint8_t* dist, uint32_t* q, uint32_t* e_thresh, uint32_t* e_alias) {
    if (!ctx || !d || e_begin > e_end || e_end > d->nnz) return DRG_EINVAL;
    API_TRY
    const uint64_t m = e_end - e_begin;
    if (col) drg::d2h(ctx, col, d->col + e_begin, m);
    if (dist) drg::d2h(ctx, dist, d->dist + e_begin, m);
    if (q) drg::d2h(ctx, q, d->q + e_begin, m);
    if (e_alias) drg::edge_alias_ids(ctx, d, e_begin, e_end, e_alias);
    if (e_thresh && m)
        DRG_CUDA(cudaMemcpy2DAsync(e_thresh, sizeof(uint32_t), static_cast<const char*>(d->etab) + e_begin * d->erec_bytes,
                                   d->erec_bytes, sizeof(uint32_t), m,
                                   cudaMemcpyDeviceToHost, ctx->stream));
    drg::sync(ctx);
    API_CATCH(ctx)
}

drg_status drg_dmat_destroy(drg_dmat* d) {
    if (!d) return DRG_EINVAL;
    drg::dmat_free(d);
    return DRG_OK;
}

// ---------------------------------------------------------------- hierarchy
drg_status drg_coarsen(drg_ctx* ctx, const drg_graph* fine, uint32_t level, const drg_params* p, drg_graph** coarse,
                       uint32_t* parent) {
    if (!ctx || !fine || !p || !coarse || !parent) return DRG_EINVAL;
    *coarse = nullptr;
    API_TRY
    DRG_CHECK(p->coarsen == DRG_COARSEN_HEM || p->coarsen == DRG_COARSEN_STAR, DRG_EINVAL,
              "coarsen must be DRG_COARSEN_HEM or DRG_COARSEN_STAR");
    *coarse = drg::coarsen(ctx, fine, level, *p, parent);
    API_CATCH(ctx)
}

drg_status drg_build_hierarchy(drg_ctx* ctx, const drg_graph* g0, const drg_params* p, drg_hier** out) {
    if (!ctx || !g0 || !p || !out) return DRG_EINVAL;
    *out = nullptr;
    API_TRY
    drg::check_params(*p);
    *out = drg::build_hierarchy(ctx, g0, *p);
    API_CATCH(ctx)
}

drg_status drg_hier_info(const drg_hier* h, uint32_t* levels, uint32_t* sizes) {
    if (!h) return DRG_EINVAL;
    if (levels) *levels = (uint32_t)h->g.size();
    if (sizes)
        for (size_t l = 0; l < h->g.size(); ++l) sizes[l] = h->g[l]->n;
    return DRG_OK;
}

drg_status drg_hier_download(drg_ctx* ctx, const drg_hier* h, uint32_t level, uint32_t* parent, uint32_t* anc) {
    if (!ctx || !h || level >= h->g.size()) return DRG_EINVAL;
    API_TRY
    if (parent) {
        DRG_CHECK(level + 1 < h->g.size(), DRG_EINVAL, "the coarsest level has no parent map");
        drg::d2h(ctx, parent, h->parent[level], h->g[level]->n);
    }
    if (anc) {
        DRG_CHECK(level >= 1, DRG_EINVAL, "level 0 has no ancestor map");
        drg::d2h(ctx, anc, h->anc[level], h->g[0]->n);
    }
    drg::sync(ctx);
    API_CATCH(ctx)
}

drg_status drg_hier_graph(const drg_hier* h, uint32_t level, const drg_graph** g) {
    if (!h || !g || level >= h->g.size()) return DRG_EINVAL;
    *g = h->g[level];
    return DRG_OK;
}

drg_status drg_hier_destroy(drg_hier* h) {
    if (!h) return DRG_EINVAL;
    drg::hier_free(h);
    return DRG_OK;
}

// ---------------------------------------------------------------- layout
drg_status drg_init_positions(drg_ctx* ctx, uint32_t n, uint32_t level, const drg_params* p, float* pos) {
    if (!ctx || !p) return DRG_EINVAL;
    API_TRY
    drg::init_positions(ctx, n, level, *p, pos);
    API_CATCH(ctx)
}

drg_status drg_layout_level(drg_ctx* ctx, const drg_dmat* d, const drg_hier* h, uint32_t level, float* pos,
                            const drg_params* p, float gamma, uint32_t t_begin, uint32_t t_end) {
    if (!ctx || !d || !p || !pos) return DRG_EINVAL;
    API_TRY
    drg::layout_level(ctx, d, h, level, pos, *p, gamma, t_begin, t_end);
    API_CATCH(ctx)
}

drg_status drg_layout_level_noalloc(drg_ctx* ctx, const drg_dmat* d, const drg_hier* h, uint32_t level,
                                    float* pos, const drg_params* p, float gamma, uint32_t t_begin, uint32_t t_end) {
    if (!ctx || !d || !p || !pos) return DRG_EINVAL;
    API_TRY
    drg::layout_level_noalloc(ctx, d, h, level, pos, *p, gamma, t_begin, t_end);
    API_CATCH(ctx)
}

drg_status drg_layout_step_explicit(drg_ctx* ctx, uint32_t n, float* pos, uint32_t S, const uint32_t* src,
                                    const uint32_t* dst, const uint32_t* neg, uint32_t M, float gamma, float b,
                                    float lr, float clip) {
    if (!ctx) return DRG_EINVAL;
    API_TRY
    drg::layout_step_explicit(ctx, n, pos, S, src, dst, neg, M, gamma, b, lr, clip);
    API_CATCH(ctx)
}

drg_status drg_autotune_enable(drg_ctx* ctx, int on) {
    if (!ctx) return DRG_EINVAL;
    ctx->autotune = on != 0;
    return DRG_OK;
}

drg_status drg_autotune_read(uint32_t cap, uint32_t* keys, uint32_t* choice, float* ms_per_epoch, uint32_t* count) {
    if (!count) return DRG_EINVAL;
    *count = drg::autotune_read(cap, keys, choice, ms_per_epoch);
    return DRG_OK;
}

drg_status drg_autotune_clear(void) {
    drg::autotune_clear();
    return DRG_OK;
}

drg_status drg_probe_memory(drg_ctx* ctx, int kind, uint64_t buffer_bytes, uint64_t accesses, uint32_t blocks_per_sm,
                            double* ms, uint64_t* done) {
    if (!ctx || !ms || !done) return DRG_EINVAL;
    API_TRY
    drg::probe_memory(ctx, kind, buffer_bytes, accesses, blocks_per_sm, ms, done);
    API_CATCH(ctx)
}

drg_status drg_check_epoch_barrier(drg_ctx* ctx, uint32_t blocks, uint32_t arrivals, uint32_t rounds,
                                   uint32_t timeout_ms) {
    if (!ctx) return DRG_EINVAL;
    API_TRY
    drg::check_epoch_barrier(ctx, blocks, arrivals, rounds, timeout_ms);
    API_CATCH(ctx)
}

drg_status drg_interpolate(drg_ctx* ctx, const drg_hier* h, uint32_t coarse_level, const float* coarse_pos,
                           float* fine_pos) {
    if (!ctx) return DRG_EINVAL;
    API_TRY
    drg::interpolate(ctx, h, coarse_level, coarse_pos, fine_pos);
    API_CATCH(ctx)
}

drg_status drg_layout(drg_ctx* ctx, const drg_graph* g, const drg_params* p, float* pos) {
    if (!ctx || !g || !p || !pos) return DRG_EINVAL;
    API_TRY
    drg::layout_full(ctx, g, *p, pos);
    API_CATCH(ctx)
}

drg_status drg_layout_edges(drg_ctx* ctx, uint32_t n, uint64_t m, const uint32_t* src, const uint32_t* dst,
                            int edges_on_device, const drg_params* p, float* pos, int pos_on_device) {
    if (!ctx || !p || !pos) return DRG_EINVAL;
    API_TRY
    drg::check_params(*p);
    drg_graph* g = drg::graph_from_edges(ctx, n, m, src, dst, edges_on_device != 0);
    try {
        if (pos_on_device) {
            drg::layout_full(ctx, g, *p, pos);
        } else {
            drg::DBuf<float> dpos(ctx, (size_t)2 * n);
            drg::layout_full(ctx, g, *p, dpos.p);
            drg::d2h(ctx, pos, dpos.p, (size_t)2 * n);
            drg::sync(ctx);
        }
    } catch (...) {
        drg::graph_free(g);
        throw;
    }
    drg::graph_free(g);
    API_CATCH(ctx)
}

drg_status drg_layout_batch(drg_ctx* ctx, uint32_t count, const drg_graph* const* graphs, const drg_params* p,
                            const float* b, float* const* pos) {
    if (!ctx || !p) return DRG_EINVAL;
    API_TRY
    drg::layout_batch(ctx, count, graphs, *p, b, pos);
    API_CATCH(ctx)
}

drg_status drg_sample_draws(drg_ctx* ctx, const drg_dmat* d, uint32_t level, uint32_t t, uint32_t s_begin,
                            uint32_t s_end, const drg_params* p, uint32_t* out_i, uint32_t* out_j, uint32_t* out_neg) {
    if (!ctx || !d || !p) return DRG_EINVAL;
    API_TRY
    drg::sample_draws(ctx, d, level, t, s_begin, s_end, *p, out_i, out_j, out_neg);
    API_CATCH(ctx)
}

}  // extern "C"
