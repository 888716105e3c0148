// Layout quality metrics of Sec. 4.1 on the device: crosslessness (Eq. 17)
// and minimum angle (Eq. 19), for large layouts whose CPU evaluation would
// take hours.
#include <algorithm>
#include <cmath>

#include "prims.cuh"

namespace drg {

// ------------------------------------------------------------------ crossings
// Positions are snapped per axis to the grid 0..2^30-1 over the layout's
// bounding box, q = floor((x - min) / (max - min) * (2^30 - 1) + 0.5) in FP64
// (0 when max = min); an affine map changes no crossing, and on the grid the
// orientation (bx-ax)(cy-ay) - (by-ay)(cx-ax) is exact in 64-bit integers.
// Two edges without a common endpoint cross when each strictly separates the
// other's endpoints; touching and collinear pairs do not count.

constexpr uint32_t kBoxBlocks = 256;

// Per-block minimum and maximum of x and y: box[b] = {min x, max x, min y,
// max y}; `bad` is set when a coordinate is not finite.
__global__ void k_bbox(const float2* __restrict__ Y, uint32_t n, float4* __restrict__ box, uint32_t* __restrict__ bad) {
    float lx = INFINITY, hx = -INFINITY, ly = INFINITY, hy = -INFINITY;
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x) {
        const float2 p = Y[v];
        if (!isfinite(p.x) || !isfinite(p.y)) *bad = 1u;
        lx = fminf(lx, p.x);
        hx = fmaxf(hx, p.x);
        ly = fminf(ly, p.y);
        hy = fmaxf(hy, p.y);
    }
#pragma unroll
    for (int off = 16; off; off >>= 1) {
        lx = fminf(lx, __shfl_xor_sync(0xFFFFFFFFu, lx, off));
        hx = fmaxf(hx, __shfl_xor_sync(0xFFFFFFFFu, hx, off));
        ly = fminf(ly, __shfl_xor_sync(0xFFFFFFFFu, ly, off));
        hy = fmaxf(hy, __shfl_xor_sync(0xFFFFFFFFu, hy, off));
    }
    __shared__ float4 w[8];
    const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) w[wid] = make_float4(lx, hx, ly, hy);
    __syncthreads();
    if (threadIdx.x == 0) {
        float4 b = w[0];
        for (uint32_t x = 1; x < blockDim.x / 32; ++x) {
            b.x = fminf(b.x, w[x].x);
            b.y = fmaxf(b.y, w[x].y);
            b.z = fminf(b.z, w[x].z);
            b.w = fmaxf(b.w, w[x].w);
        }
        box[blockIdx.x] = b;
    }
}

__device__ __forceinline__ int32_t snap(float x, double lo, double span) {
    if (!(span > 0.0)) return 0;
    const double t = __dadd_rn(__dmul_rn(__ddiv_rn(__dsub_rn((double)x, lo), span), 1073741823.0), 0.5);
    return (int32_t)floor(t);
}

// Each undirected edge once: the entries of row u with column > u, which are
// the tail of the (column-sorted) row.
__global__ void k_upper_count(const uint64_t* __restrict__ rp, const uint32_t* __restrict__ col, uint32_t n,
                              uint32_t* __restrict__ cnt) {
    for (uint64_t u = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; u < n; u += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t lo = rp[u], hi = rp[u + 1];
        const uint64_t end = hi;
        while (lo < hi) {  // first entry with column > u
            const uint64_t mid = (lo + hi) >> 1;
            if (col[mid] > (uint32_t)u) hi = mid;
            else lo = mid + 1;
        }
        cnt[u] = (uint32_t)(end - lo);
    }
}

// Edge e: snapped endpoint coordinates and ids.
struct SegQ {
    int32_t ax, ay, bx, by;
};

__global__ void k_edge_list(const uint64_t* __restrict__ rp, const uint32_t* __restrict__ col, uint32_t n,
                            const uint32_t* __restrict__ off, const uint32_t* __restrict__ cnt,
                            const float2* __restrict__ Y, double lox, double spanx, double loy, double spany,
                            SegQ* __restrict__ seg, uint2* __restrict__ ends) {
    for (uint64_t u = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; u < n; u += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t c = cnt[u];
        if (c == 0) continue;
        const float2 pu = Y[u];
        const int32_t ux = snap(pu.x, lox, spanx), uy = snap(pu.y, loy, spany);
        const uint64_t first = rp[u + 1] - c;
        for (uint32_t x = 0; x < c; ++x) {
            const uint32_t v = col[first + x];
            const float2 pv = Y[v];
            const uint32_t e = off[u] + x;
            seg[e] = SegQ{ux, uy, snap(pv.x, lox, spanx), snap(pv.y, loy, spany)};
            ends[e] = make_uint2((uint32_t)u, v);
        }
    }
}

__device__ __forceinline__ int orient_sign(int32_t ax, int32_t ay, int32_t bx, int32_t by, int32_t cx, int32_t cy) {
    const long long o = (long long)(bx - ax) * (long long)(cy - ay) - (long long)(by - ay) * (long long)(cx - ax);
    return (o > 0) - (o < 0);
}

__device__ __forceinline__ bool crosses(const SegQ& s, uint2 se, const SegQ& t, uint2 te) {
    // disjoint bounding boxes cannot hold a proper crossing
    if (max(s.ax, s.bx) < min(t.ax, t.bx) || max(t.ax, t.bx) < min(s.ax, s.bx) ||
        max(s.ay, s.by) < min(t.ay, t.by) || max(t.ay, t.by) < min(s.ay, s.by))
        return false;
    if (se.x == te.x || se.x == te.y || se.y == te.x || se.y == te.y) return false;
    const int o1 = orient_sign(s.ax, s.ay, s.bx, s.by, t.ax, t.ay);
    const int o2 = orient_sign(s.ax, s.ay, s.bx, s.by, t.bx, t.by);
    if (o1 * o2 >= 0) return false;
    const int o3 = orient_sign(t.ax, t.ay, t.bx, t.by, s.ax, s.ay);
    const int o4 = orient_sign(t.ax, t.ay, t.bx, t.by, s.bx, s.by);
    return o3 * o4 < 0;
}

constexpr uint32_t kCrossTile = 256;
constexpr uint64_t kCrossPairsPerLaunch = 1ull << 21;  // tile pairs per launch (2^37 pair tests)
constexpr uint32_t kCrossMaxEdges = 1u << 23;

// Tile pairs [p0, p1) of all pairs of edges, taken from a persistent grid:
// tile pair p is (I, J) with J(J+1)/2 <= p < (J+1)(J+2)/2, I = p - J(J+1)/2.
// Thread x of a block owns edge I*256 + x and tests it against every edge of
// tile J (staged in shared memory) with a larger index.
__global__ void __launch_bounds__(kCrossTile) k_crossings(const SegQ* __restrict__ seg, const uint2* __restrict__ ends,
                                                           uint32_t m, uint64_t p0, uint64_t p1,
                                                           unsigned long long* __restrict__ total) {
    __shared__ SegQ ts[kCrossTile];
    __shared__ uint2 te[kCrossTile];
    __shared__ unsigned long long wsum[kCrossTile / 32];
    unsigned long long acc = 0;
    for (uint64_t p = p0 + blockIdx.x; p < p1; p += gridDim.x) {
        uint64_t J = (uint64_t)((sqrt(8.0 * (double)p + 1.0) - 1.0) * 0.5);
        while (J * (J + 1) / 2 > p) --J;
        while ((J + 1) * (J + 2) / 2 <= p) ++J;
        const uint64_t I = p - J * (J + 1) / 2;
        const uint64_t i = I * kCrossTile + threadIdx.x;
        const uint64_t j0 = J * kCrossTile;
        __syncthreads();  // the previous tile is no longer read
        if (j0 + threadIdx.x < m) {
            ts[threadIdx.x] = seg[j0 + threadIdx.x];
            te[threadIdx.x] = ends[j0 + threadIdx.x];
        }
        __syncthreads();
        if (i < m) {
            const SegQ s = seg[i];
            const uint2 se = ends[i];
            const uint32_t cnt = (uint32_t)min((uint64_t)kCrossTile, m - j0);
            const uint32_t start = (I == J) ? threadIdx.x + 1 : 0u;
            uint32_t c = 0;
            for (uint32_t x = start; x < cnt; ++x) c += crosses(s, se, ts[x], te[x]) ? 1u : 0u;
            acc += c;
        }
    }
#pragma unroll
    for (int off = 16; off; off >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, off);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long s = 0;
        for (uint32_t w = 0; w < kCrossTile / 32; ++w) s += wsum[w];
        atomicAdd(total, s);
    }
}

// sum over nodes of deg(v)(deg(v) - 1)/2: the pairs of edges that share a node
__global__ void k_adjacent_pairs(const uint64_t* __restrict__ rp, uint32_t n, unsigned long long* __restrict__ total) {
    unsigned long long acc = 0;
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x) {
        const unsigned long long d = rp[v + 1] - rp[v];
        acc += d * (d ? d - 1 : 0) / 2;
    }
#pragma unroll
    for (int off = 16; off; off >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, off);
    if ((threadIdx.x & 31) == 0) atomicAdd(total, acc);
}

static void layout_box(drg_ctx* ctx, const float2* Y, uint32_t n, double* lo, double* span) {
    DBuf<float4> box(ctx, kBoxBlocks);
    DBuf<uint32_t> bad(ctx, 1);
    DRG_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(uint32_t), ctx->stream));
    DRG_LAUNCH(ctx, k_bbox, kBoxBlocks, 256, 0, Y, n, box.p, bad.p);
    std::vector<float4> h(kBoxBlocks);
    DRG_CUDA(cudaMemcpyAsync(h.data(), box.p, sizeof(float4) * kBoxBlocks, cudaMemcpyDeviceToHost, ctx->stream));
    DRG_CHECK(read1(ctx, bad.p) == 0, DRG_EINVAL, "positions must be finite");
    float4 b = h[0];
    for (uint32_t x = 1; x < kBoxBlocks; ++x) {
        b.x = std::fmin(b.x, h[x].x);
        b.y = std::fmax(b.y, h[x].y);
        b.z = std::fmin(b.z, h[x].z);
        b.w = std::fmax(b.w, h[x].w);
    }
    lo[0] = (double)b.x;
    span[0] = (double)b.y - (double)b.x;
    lo[1] = (double)b.z;
    span[1] = (double)b.w - (double)b.z;
}

void crossings(drg_ctx* ctx, const drg_graph* g, const float* pos, uint64_t* c_out, double* crosslessness) {
    DRG_CHECK(g && pos && c_out && crosslessness, DRG_EINVAL, "null argument");
    const uint32_t n = g->n;
    const float2* Y = reinterpret_cast<const float2*>(pos);
    double lo[2], span[2];
    layout_box(ctx, Y, n, lo, span);
    DBuf<uint32_t> cnt(ctx, n), off(ctx, n), m_dev(ctx, 1);
    const uint32_t gt = grid_for(n, 256, (uint32_t)ctx->num_sms * 16);
    DRG_LAUNCH(ctx, k_upper_count, gt, 256, 0, g->rp, g->col, n, cnt.p);
    scan<uint32_t>(ctx, LoadArr<uint32_t>{cnt.p}, n, off.p, false, m_dev.p);
    const uint32_t m = read1(ctx, m_dev.p);
    DRG_CHECK(m <= kCrossMaxEdges, DRG_EUNSUPPORTED,
              "crossing count limited to 8388608 edges (all-pairs test, about 80 s at that size)");
    DBuf<unsigned long long> acc(ctx, 2);
    DRG_CUDA(cudaMemsetAsync(acc.p, 0, 2 * sizeof(unsigned long long), ctx->stream));
    DRG_LAUNCH(ctx, k_adjacent_pairs, gt, 256, 0, g->rp, n, acc.p + 1);
    if (m > 1) {
        DBuf<SegQ> seg(ctx, m);
        DBuf<uint2> ends(ctx, m);
        DRG_LAUNCH(ctx, k_edge_list, gt, 256, 0, g->rp, g->col, n, off.p, cnt.p, Y, lo[0], span[0], lo[1], span[1],
                   seg.p, ends.p);
        // bounded launches: at most kCrossPairsPerLaunch tile pairs (2^37
        // pair tests, about a third of a second) each
        const uint64_t tiles = (m + kCrossTile - 1) / kCrossTile;
        const uint64_t pairs = tiles * (tiles + 1) / 2;
        for (uint64_t p0 = 0; p0 < pairs; p0 += kCrossPairsPerLaunch) {
            const uint64_t p1 = std::min<uint64_t>(pairs, p0 + kCrossPairsPerLaunch);
            const uint32_t grid = (uint32_t)std::min<uint64_t>(p1 - p0, (uint64_t)ctx->num_sms * 8);
            DRG_LAUNCH(ctx, k_crossings, grid, kCrossTile, 0, seg.p, ends.p, m, p0, p1, acc.p);
        }
    }
    unsigned long long h[2];
    DRG_CUDA(cudaMemcpyAsync(h, acc.p, sizeof h, cudaMemcpyDeviceToHost, ctx->stream));
    sync(ctx);
    const uint64_t all = (uint64_t)m * (m ? m - 1 : 0) / 2;
    const uint64_t cmax = all - h[1];
    *c_out = h[0];
    *crosslessness = cmax > 0 ? 1.0 - std::sqrt((double)h[0] / (double)cmax) : 1.0;
}

// ------------------------------------------------------------------ minimum angle
// theta_min(v): the smallest angle between edges that are consecutive
// around v.  Every entry (v, u) gets its direction atan2(y_u - y_v, x_u - x_v)
// (FP64); one radix sort by (row, direction mapped monotonically to 32 bits)
// orders each row by angle; one warp per row then takes the smallest gap
// between consecutive directions, the wrap-around gap 2 pi - (last - first)
// included.  Directions closer than 2 pi / 2^32 may come out of order; their
// gap then counts as 0 (an error below 1.5e-9 rad).
__global__ void k_directions(const uint64_t* __restrict__ rp, const uint32_t* __restrict__ col, uint32_t n,
                             const float2* __restrict__ Y, double* __restrict__ phi,
                             uint64_t* __restrict__ keys, uint32_t* __restrict__ idx) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warp0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t v = warp0; v < n; v += nwarps) {
        const float2 pv = Y[v];
        for (uint64_t e = rp[v] + lane; e < rp[v + 1]; e += 32) {
            const float2 pu = Y[col[e]];
            const double a = atan2((double)pu.y - (double)pv.y, (double)pu.x - (double)pv.x);
            phi[e] = a;
            // [-pi, pi] -> [0, 2^32 - 1], monotone
            double t = (a + 3.141592653589793) * (4294967296.0 / 6.283185307179586);
            t = t < 0.0 ? 0.0 : (t > 4294967295.0 ? 4294967295.0 : t);
            keys[e] = (v << 32) | (uint64_t)(uint32_t)t;
            idx[e] = (uint32_t)e;
        }
    }
}

__global__ void k_min_angle_rows(const uint64_t* __restrict__ rp, uint32_t n, const double* __restrict__ phi,
                                 const uint32_t* __restrict__ idx, double* __restrict__ dev_sum,
                                 unsigned long long* __restrict__ counted) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warp0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const double two_pi = 6.283185307179586;
    double dsum = 0.0;
    unsigned long long cnt = 0;
    for (uint64_t v = warp0; v < n; v += nwarps) {
        const uint64_t b = rp[v], e = rp[v + 1], d = e - b;
        if (d == 0) continue;
        ++cnt;  // lane-uniform; only lane 0's count is kept
        if (d == 1) continue;
        double mn = INFINITY;
        for (uint64_t x = b + lane; x + 1 < e; x += 32) {
            const double gap = phi[idx[x + 1]] - phi[idx[x]];
            mn = fmin(mn, gap > 0.0 ? gap : 0.0);
        }
#pragma unroll
        for (int off = 16; off; off >>= 1) mn = fmin(mn, __shfl_xor_sync(0xFFFFFFFFu, mn, off));
        if (lane == 0) {
            const double wrap = two_pi - (phi[idx[e - 1]] - phi[idx[b]]);
            mn = fmin(mn, wrap);
            const double theta = two_pi / (double)d;
            dsum += fabs(theta - mn) / theta;
        }
    }
    if (lane == 0) {
        atomicAdd(dev_sum, dsum);
        atomicAdd(counted, cnt);
    }
}

double min_angle(drg_ctx* ctx, const drg_graph* g, const float* pos) {
    DRG_CHECK(g && pos, DRG_EINVAL, "null argument");
    const uint32_t n = g->n;
    const uint64_t nnz = g->nnz;
    const float2* Y = reinterpret_cast<const float2*>(pos);
    if (nnz == 0) return 1.0;
    DRG_CHECK(nnz < (1ull << 32), DRG_EUNSUPPORTED, "minimum angle limited to 2^32 entries");
    DBuf<double> phi(ctx, nnz), dsum(ctx, 1);
    DBuf<uint64_t> keys(ctx, nnz), kalt(ctx, nnz);
    DBuf<uint32_t> idx(ctx, nnz), ialt(ctx, nnz);
    DBuf<unsigned long long> counted(ctx, 1);
    const int rb = bitlen(n > 1 ? n - 1 : 1);
    const uint32_t gw = grid_for((size_t)n * 32, 256, (uint32_t)ctx->num_sms * 16);
    DRG_LAUNCH(ctx, k_directions, gw, 256, 0, g->rp, g->col, n, Y, phi.p, keys.p, idx.p);
    uint64_t* kp = keys.p;
    uint64_t* ap = kalt.p;
    uint32_t* vp = idx.p;
    uint32_t* vq = ialt.p;
    radix_sort(ctx, kp, ap, vp, vq, nnz, 0, 32 + rb);
    DRG_CUDA(cudaMemsetAsync(dsum.p, 0, sizeof(double), ctx->stream));
    DRG_CUDA(cudaMemsetAsync(counted.p, 0, sizeof(unsigned long long), ctx->stream));
    DRG_LAUNCH(ctx, k_min_angle_rows, gw, 256, 0, g->rp, n, phi.p, vp, dsum.p, counted.p);
    double s;
    unsigned long long c;
    DRG_CUDA(cudaMemcpyAsync(&s, dsum.p, sizeof s, cudaMemcpyDeviceToHost, ctx->stream));
    DRG_CUDA(cudaMemcpyAsync(&c, counted.p, sizeof c, cudaMemcpyDeviceToHost, ctx->stream));
    sync(ctx);
    return c ? 1.0 - s / (double)c : 1.0;
}

}  // namespace drg
