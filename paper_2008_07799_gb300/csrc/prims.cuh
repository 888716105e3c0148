// Device-wide primitives used by the graph, distance-matrix and alias-table
// builders: block/grid prefix sums over any unsigned type (up to 128 bits)
// and a stable LSD radix sort of 64-bit keys with optional 32-bit values.
#pragma once

#include "common.cuh"

namespace drg {

// ------------------------------------------------------------------ warp shuffles
__device__ __forceinline__ uint32_t shfl_up(uint32_t v, int d) { return __shfl_up_sync(0xFFFFFFFFu, v, d); }
__device__ __forceinline__ uint64_t shfl_up(uint64_t v, int d) { return __shfl_up_sync(0xFFFFFFFFu, v, d); }
__device__ __forceinline__ u128 shfl_up(u128 v, int d) {
    uint64_t lo = (uint64_t)v, hi = (uint64_t)(v >> 64);
    lo = __shfl_up_sync(0xFFFFFFFFu, lo, d);
    hi = __shfl_up_sync(0xFFFFFFFFu, hi, d);
    return ((u128)hi << 64) | lo;
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Exclusive prefix sum of one value per thread across the block; every thread
// also receives the block total.  warp_tot: shared array of THREADS/32.
template <typename T, int THREADS>
__device__ __forceinline__ T block_exclusive_scan(T v, T* warp_tot, T& total) {
    constexpr int NW = THREADS / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        T y = shfl_up(x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        T w = lane < NW ? warp_tot[lane] : T(0);
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            T y = shfl_up(w, d);
            if (lane >= d) w += y;
        }
        if (lane < NW) warp_tot[lane] = w;
    }
    __syncthreads();
    T prefix = warp ? warp_tot[warp - 1] : T(0);
    total = warp_tot[NW - 1];
    __syncthreads();
    return prefix + x - v;
}

// ------------------------------------------------------------------ input functors
template <typename T>
struct LoadArr {
    const T* p;
    __device__ __forceinline__ T operator()(size_t i) const { return p[i]; }
};
template <typename Tin, typename Tout>
struct LoadConv {
    const Tin* p;
    __device__ __forceinline__ Tout operator()(size_t i) const { return (Tout)p[i]; }
};

// ------------------------------------------------------------------ grid scan
template <typename T>
struct ScanShape {
    static constexpr int THREADS = 256;
    static constexpr int ITEMS = sizeof(T) > 16 ? 2 : (sizeof(T) == 16 ? 4 : 8);  // tile <= 32 KB of shared memory
    static constexpr int TILE = THREADS * ITEMS;
};

template <typename T, typename F>
__global__ void __launch_bounds__(256) k_scan_reduce(F in, size_t n, T* sums) {
    constexpr int TH = ScanShape<T>::THREADS, IT = ScanShape<T>::ITEMS;
    __shared__ T wt[TH / 32];
    const size_t base = (size_t)blockIdx.x * ScanShape<T>::TILE;
    T acc = 0;
#pragma unroll
    for (int j = 0; j < IT; ++j) {
        size_t i = base + (size_t)j * TH + threadIdx.x;
        if (i < n) acc += in(i);
    }
    T tot;
    block_exclusive_scan<T, TH>(acc, wt, tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

template <typename T, typename F>
__global__ void __launch_bounds__(256) k_scan_down(F in, size_t n, const T* offsets, T* out, int inclusive, T* total) {
    constexpr int TH = ScanShape<T>::THREADS, IT = ScanShape<T>::ITEMS;
    __shared__ T tile[TH * IT];
    __shared__ T wt[TH / 32];
    const size_t base = (size_t)blockIdx.x * ScanShape<T>::TILE;
#pragma unroll
    for (int j = 0; j < IT; ++j) {
        size_t i = base + (size_t)j * TH + threadIdx.x;
        tile[j * TH + threadIdx.x] = i < n ? in(i) : T(0);
    }
    __syncthreads();
    T loc[IT];
    T s = 0;
#pragma unroll
    for (int j = 0; j < IT; ++j) {
        loc[j] = tile[threadIdx.x * IT + j];
        s += loc[j];
    }
    T bt;
    T pre = block_exclusive_scan<T, TH>(s, wt, bt);
    const T off = offsets ? offsets[blockIdx.x] : T(0);
    T run = off + pre;
#pragma unroll
    for (int j = 0; j < IT; ++j) {
        if (inclusive) {
            run += loc[j];
            tile[threadIdx.x * IT + j] = run;
        } else {
            tile[threadIdx.x * IT + j] = run;
            run += loc[j];
        }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < IT; ++j) {
        size_t i = base + (size_t)j * TH + threadIdx.x;
        if (i < n) out[i] = tile[j * TH + threadIdx.x];
    }
    if (total && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *total = off + bt;
}

// out[i] = sum of in(0..i-1) (exclusive) or in(0..i) (inclusive); *total_dev
// (device, optional) receives the sum of all n values.  `out` may alias the
// array `in` reads from.
template <typename T, typename F>
void scan(drg_ctx* ctx, F in, size_t n, T* out, bool inclusive, T* total_dev) {
    if (n == 0) {
        if (total_dev) DRG_CUDA(cudaMemsetAsync(total_dev, 0, sizeof(T), ctx->stream));
        return;
    }
    const size_t tile = ScanShape<T>::TILE;
    const size_t nb = (n + tile - 1) / tile;
    if (nb == 1) {
        DRG_LAUNCH(ctx, (k_scan_down<T, F>), 1, 256, 0, in, n, (const T*)nullptr, out, (int)inclusive, total_dev);
        return;
    }
    DBuf<T> sums(ctx, nb);
    DRG_LAUNCH(ctx, (k_scan_reduce<T, F>), (uint32_t)nb, 256, 0, in, n, sums.p);
    scan<T>(ctx, LoadArr<T>{sums.p}, nb, sums.p, false, total_dev);
    DRG_LAUNCH(ctx, (k_scan_down<T, F>), (uint32_t)nb, 256, 0, in, n, (const T*)sums.p, out, (int)inclusive,
               (T*)nullptr);
}

// ------------------------------------------------------------------ radix sort
// Sorts keys (and vals, when non-null) stably by bits [begin_bit, end_bit).
// `keys`/`vals` and the equally sized `alt` buffers are swapped as passes
// go; on return `keys`/`vals` point at the sorted data.  n < 2^32.
void radix_sort(drg_ctx* ctx, uint64_t*& keys, uint64_t*& keys_alt, uint32_t*& vals, uint32_t*& vals_alt,
                size_t n, int begin_bit, int end_bit);

inline int bitlen(uint64_t x) {
    int b = 0;
    while (b < 64 && (x >> b) != 0) ++b;
    return b;
}

}  // namespace drg
