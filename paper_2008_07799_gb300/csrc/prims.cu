// Stable LSD radix sort of 64-bit keys with optional 32-bit values, 8 bits
// per pass: per-tile digit histograms, one exclusive scan over
// (digit, tile), then a stable scatter.
#include "prims.cuh"

namespace drg {

constexpr int RS_THREADS = 256, RS_ITEMS = 16, RS_WARPS = RS_THREADS / 32;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;

__global__ void __launch_bounds__(RS_THREADS) k_rs_hist(const uint64_t* __restrict__ keys, size_t n, int shift,
                                                        uint32_t* __restrict__ counts, uint32_t nb) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const size_t base = (size_t)blockIdx.x * RS_TILE;
#pragma unroll 4
    for (int j = 0; j < RS_ITEMS; ++j) {
        size_t i = base + (size_t)j * RS_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&h[(uint32_t)(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    counts[(size_t)threadIdx.x * nb + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter of one tile: warp w owns RS_ITEMS rounds of 32 consecutive
// keys; ranks inside a round come from __match_any_sync, across rounds and
// warps from per-warp digit counters, across tiles from the scanned counts.
__global__ void __launch_bounds__(RS_THREADS) k_rs_scatter(const uint64_t* __restrict__ kin,
                                                           const uint32_t* __restrict__ vin,
                                                           uint64_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                                           size_t n, int shift, const uint32_t* __restrict__ offs,
                                                           uint32_t nb) {
    __shared__ uint32_t wc[RS_WARPS][256];
    __shared__ uint32_t goff[256];
    for (int x = threadIdx.x; x < RS_WARPS * 256; x += RS_THREADS) (&wc[0][0])[x] = 0;
    goff[threadIdx.x] = offs[(size_t)threadIdx.x * nb + blockIdx.x];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const size_t wbase = (size_t)blockIdx.x * RS_TILE + (size_t)warp * (32 * RS_ITEMS);
    const uint32_t lt = lanemask_lt();
    uint64_t k[RS_ITEMS];
    uint32_t v[RS_ITEMS], rk[RS_ITEMS], dg[RS_ITEMS];
#pragma unroll
    for (int r = 0; r < RS_ITEMS; ++r) {
        const size_t i = wbase + (size_t)r * 32 + lane;
        const bool valid = i < n;
        const uint64_t key = valid ? kin[i] : 0ull;
        const uint32_t d = valid ? ((uint32_t)(key >> shift) & 255u) : 256u;
        const uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
        const uint32_t prev = d < 256u ? wc[warp][d] : 0u;
        __syncwarp();
        if (d < 256u && lane == __ffs(peers) - 1) wc[warp][d] = prev + __popc(peers);
        __syncwarp();
        rk[r] = prev + __popc(peers & lt);
        k[r] = key;
        dg[r] = d;
        v[r] = (vin && valid) ? vin[i] : 0u;
    }
    __syncthreads();
    {
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < RS_WARPS; ++w) {
            uint32_t c = wc[w][threadIdx.x];
            wc[w][threadIdx.x] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RS_ITEMS; ++r) {
        if (dg[r] < 256u) {
            const uint32_t pos = goff[dg[r]] + wc[warp][dg[r]] + rk[r];
            kout[pos] = k[r];
            if (vout) vout[pos] = v[r];
        }
    }
}

void radix_sort(drg_ctx* ctx, uint64_t*& keys, uint64_t*& keys_alt, uint32_t*& vals, uint32_t*& vals_alt,
                       size_t n, int begin_bit, int end_bit) {
    if (n <= 1 || end_bit <= begin_bit) return;
    DRG_CHECK(n < (1ull << 32), DRG_EUNSUPPORTED, "radix sort limited to 2^32 keys");
    const uint32_t nb = (uint32_t)((n + RS_TILE - 1) / RS_TILE);
    DBuf<uint32_t> counts(ctx, (size_t)256 * nb);
    for (int shift = begin_bit; shift < end_bit; shift += 8) {
        DRG_LAUNCH(ctx, k_rs_hist, nb, RS_THREADS, 0, keys, n, shift, counts.p, nb);
        scan<uint32_t>(ctx, LoadArr<uint32_t>{counts.p}, (size_t)256 * nb, counts.p, false, nullptr);
        DRG_LAUNCH(ctx, k_rs_scatter, nb, RS_THREADS, 0, keys, vals, keys_alt, vals ? vals_alt : nullptr, n, shift,
                   counts.p, nb);
        std::swap(keys, keys_alt);
        if (vals) std::swap(vals, vals_alt);
    }
}

}  // namespace drg
