/*
 * drg_oracle.c -- plain, slow, obviously-correct CPU oracle of the DRGraph
 * layout path (Zhu et al., "DRGraph: An Efficient Graph Layout Algorithm for
 * Large-scale Graphs by Dimensionality Reduction", arXiv 2008.07799).
 *
 * TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and the timed
 * CPU-baseline leg of the benchmark may load this library.  It shares no code
 * with the CUDA library: every definition below is written out again from the
 * paper (and from the readings of it recorded in the design notes), not taken
 * from the GPU sources, and nothing here is blocked, fused or reordered
 * beyond what the definition states.
 *
 * Precision: layout arithmetic in FP64.  Graph and index work is exact
 * integer arithmetic.  The quantised sampling weights are defined by FP32
 * correctly-rounded operations in a fixed order (they decide integers, so
 * both implementations take that decision in the same precision); compile
 * with -ffp-contract=off so no multiply-add is fused.
 *
 * Randomness: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11), implemented here from that paper.
 *
 * Parity status per function: see the header comment of each.  Whole-run
 * layout quality against the paper's published numbers is "parity
 * unpinned" (the paper gives neither its RNG, sigma nor learning rate); it is
 * pinned only against this oracle's own definitions.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

#define ORC_NONE 0xFFFFFFFFu

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al. SC'11, Sec. 5): 10 rounds of two 32x32->64
 * multiplications with the Philox constants, key bumped by the Weyl
 * constants between rounds.  Pinned by the published known-answer vectors.  */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Stream tag of the Philox counter's third word: purpose (0 = layout
 * samples, 1 = initial positions, 2 = matching tie-break, 3 = order of the
 * star grouping), graph id, level. */
uint32_t orc_tag(uint32_t purpose, uint32_t gid, uint32_t level)
{
    return (purpose << 28) | ((gid & 0xFFFFFu) << 8) | (level & 0xFFu);
}

/* Word `w` of the random stream of (a, b, tag) under `seed`: Philox call
 * number w/4, lane w%4, counter (a, b, tag, w/4). */
static uint32_t orc_word(uint64_t seed, uint32_t a, uint32_t b, uint32_t tag, uint32_t w)
{
    uint32_t ctr[4] = {a, b, tag, w / 4u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return out[w % 4u];
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.2.1, Eq. 8: NNG(v_i,k) = { v : SPD(v_i,v) <= k, v != v_i }.
 * A breadth-first search from every source, stopped at depth k.  Pass 1
 * counts each row; pass 2 writes row i's neighbours sorted by node id with
 * their hop distance (the sparse distance matrix GD of Sec. 3.2.1).
 * Pinned by closed forms on paths, cycles and grids and by all-pairs
 * shortest paths on small random graphs.                                     */
static int orc_cmp_u32(const void* a, const void* b)
{
    uint32_t x = *(const uint32_t*)a, y = *(const uint32_t*)b;
    return (x > y) - (x < y);
}

static uint32_t orc_bfs(uint32_t n, const uint64_t* rp, const uint32_t* col, uint32_t k,
                        uint32_t src, int32_t* dist, uint32_t* queue)
{
    uint32_t head = 0, tail = 0;
    dist[src] = 0;
    queue[tail++] = src;
    while (head < tail) {
        uint32_t u = queue[head++];
        if ((uint32_t)dist[u] == k) continue;
        for (uint64_t e = rp[u]; e < rp[u + 1]; ++e) {
            uint32_t v = col[e];
            if (dist[v] < 0) {
                dist[v] = dist[u] + 1;
                queue[tail++] = v;
            }
        }
    }
    (void)n;
    return tail; /* queue[0..tail) = visited nodes incl. src */
}

int orc_korder_counts(uint32_t n, const uint64_t* rp, const uint32_t* col, uint32_t k, uint64_t* counts)
{
    int32_t* dist = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
    uint32_t* queue = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n ? n : 1));
    if (!dist || !queue) { free(dist); free(queue); return -1; }
    for (uint32_t v = 0; v < n; ++v) dist[v] = -1;
    for (uint32_t i = 0; i < n; ++i) {
        uint32_t cnt = orc_bfs(n, rp, col, k, i, dist, queue);
        counts[i] = cnt - 1;
        for (uint32_t q = 0; q < cnt; ++q) dist[queue[q]] = -1;
    }
    free(dist); free(queue);
    return 0;
}

int orc_korder_fill(uint32_t n, const uint64_t* rp, const uint32_t* col, uint32_t k,
                    const uint64_t* gd_rp, uint32_t* gd_col, uint8_t* gd_dist)
{
    int32_t* dist = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
    uint32_t* queue = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n ? n : 1));
    if (!dist || !queue) { free(dist); free(queue); return -1; }
    for (uint32_t v = 0; v < n; ++v) dist[v] = -1;
    for (uint32_t i = 0; i < n; ++i) {
        uint32_t cnt = orc_bfs(n, rp, col, k, i, dist, queue);
        uint32_t* row = gd_col + gd_rp[i];
        uint32_t w = 0;
        for (uint32_t q = 0; q < cnt; ++q)
            if (queue[q] != i) row[w++] = queue[q];
        qsort(row, w, sizeof(uint32_t), orc_cmp_u32);
        for (uint32_t q = 0; q < w; ++q) gd_dist[gd_rp[i] + q] = (uint8_t)dist[row[q]];
        for (uint32_t q = 0; q < cnt; ++q) dist[queue[q]] = -1;
    }
    free(dist); free(queue);
    return 0;
}

/* Row `src` of GD alone (the same BFS as above, for spot checks of large
 * graphs): writes the row sorted by node id with hop distances and returns
 * its length.  dist (n entries, all -1) and queue (n entries) are scratch the
 * caller provides; dist is restored to all -1 on return.                     */
uint32_t orc_korder_row(uint32_t n, const uint64_t* rp, const uint32_t* col, uint32_t k, uint32_t src,
                        int32_t* dist, uint32_t* queue, uint32_t* out_col, uint8_t* out_dist)
{
    uint32_t cnt = orc_bfs(n, rp, col, k, src, dist, queue);
    uint32_t w = 0;
    for (uint32_t q = 0; q < cnt; ++q)
        if (queue[q] != src) out_col[w++] = queue[q];
    qsort(out_col, w, sizeof(uint32_t), orc_cmp_u32);
    for (uint32_t q = 0; q < w; ++q) out_dist[q] = (uint8_t)dist[out_col[q]];
    for (uint32_t q = 0; q < cnt; ++q) dist[queue[q]] = -1;
    return w;
}

/* For each listed source, the number of nodes at hop distance d = 1..k
 * (counts[x * k + d - 1]): the class sizes that define Z_i in Eq. 9.        */
int orc_class_counts(uint32_t n, const uint64_t* rp, const uint32_t* col, uint32_t k,
                     uint32_t nsel, const uint32_t* sel, uint64_t* counts)
{
    int32_t* dist = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
    uint32_t* queue = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n ? n : 1));
    if (!dist || !queue) { free(dist); free(queue); return -1; }
    for (uint32_t v = 0; v < n; ++v) dist[v] = -1;
    for (uint32_t x = 0; x < nsel; ++x) {
        uint32_t cnt = orc_bfs(n, rp, col, k, sel[x], dist, queue);
        for (uint32_t d = 0; d < k; ++d) counts[(size_t)x * k + d] = 0;
        for (uint32_t q = 1; q < cnt; ++q) counts[(size_t)x * k + dist[queue[q]] - 1] += 1;
        for (uint32_t q = 0; q < cnt; ++q) dist[queue[q]] = -1;
    }
    free(dist); free(queue);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.2.1 Eq. 9 (sparse conditional similarity NS_{j|i} = g(GD_ij)/Z_i
 * over NNG(v_i,k), g(d) = exp(-d^2 / 2 sigma^2), the k values precomputed)
 * and Sec. 3.1 Eq. 4 (NS_ij = (NS_{i|j} + NS_{j|i}) / 2|V|).
 *
 * Outputs:
 *   g[d-1]  FP32 Gaussian for d = 1..k (computed in FP64 from the FP32
 *           parameter sigma, rounded once)
 *   Z[i]    FP32 normaliser, summed over d = 1..k in that order
 *   q[e]    quantised edge weight: floor((fl(g/Z_i) + fl(g/Z_j)) * 2^30)
 *           (FP32, correctly rounded, no fused multiply-add); proportional
 *           to NS_ij up to the quantisation
 *   r[i]    node weight sum_e q[e] over row i (exact, u64) -- the negative
 *           sampling weight sum_l NS_il of Sec. 3.2.2 up to a constant
 *   ns[e]   exact FP64 NS_ij (reference value, not used for sampling)
 * Pinned by: rows of NS_{j|i} summing to 1, k = 1 giving 1/deg, symmetry,
 * sum NS_ij = 1 and the quantisation error bound.                           */
/* Z_i in FP32: sum over d = 1..k, in that order, of fl(count_i(d) g(d)). */
float orc_normaliser(uint32_t k, const uint64_t* count, const float* g)
{
    float z = 0.0f;
    for (uint32_t d = 1; d <= k; ++d) {
        float term = (float)count[d - 1] * g[d - 1];
        z = z + term;
    }
    return z;
}

/* q_e = floor((fl(g / Z_i) + fl(g / Z_j)) * 2^30) in FP32. */
uint32_t orc_entry_weight(float gd, float zi, float zj)
{
    float p_ji = gd / zi;
    float p_ij = gd / zj;
    float s = p_ji + p_ij;
    float scaled = s * 1073741824.0f; /* 2^30, exact */
    return (uint32_t)scaled;
}

int orc_similarity(uint32_t n, const uint64_t* rp, const uint32_t* col, const uint8_t* dist,
                   uint32_t k, float sigma, float* g, float* Z, uint32_t* q, uint64_t* r, double* ns)
{
    double* g64 = (double*)malloc(sizeof(double) * (k + 1));
    double* Z64 = (double*)malloc(sizeof(double) * (size_t)(n ? n : 1));
    uint64_t* cnt = (uint64_t*)malloc(sizeof(uint64_t) * (k + 1));
    if (!g64 || !Z64 || !cnt) { free(g64); free(Z64); free(cnt); return -1; }
    for (uint32_t d = 1; d <= k; ++d) {
        g64[d] = exp(-(double)(d * d) / (2.0 * (double)sigma * (double)sigma));
        g[d - 1] = (float)g64[d];
    }
    for (uint32_t i = 0; i < n; ++i) {
        for (uint32_t d = 0; d <= k; ++d) cnt[d] = 0;
        for (uint64_t e = rp[i]; e < rp[i + 1]; ++e) cnt[dist[e]] += 1;
        double z64 = 0.0;
        for (uint32_t d = 1; d <= k; ++d) z64 += (double)cnt[d] * g64[d];
        Z[i] = orc_normaliser(k, cnt + 1, g);
        Z64[i] = z64;
    }
    for (uint32_t i = 0; i < n; ++i) {
        uint64_t acc = 0;
        for (uint64_t e = rp[i]; e < rp[i + 1]; ++e) {
            uint32_t j = col[e];
            uint32_t d = dist[e];
            q[e] = orc_entry_weight(g[d - 1], Z[i], Z[j]);
            acc += q[e];
            if (ns) ns[e] = (g64[d] / Z64[i] + g64[d] / Z64[j]) / (2.0 * (double)n);
        }
        r[i] = acc;
    }
    free(g64); free(Z64); free(cnt);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Per-node sigma_i of Eq. 9 set by perplexity, the t-SNE rule the paper's
 * sigma_i comes from: the conditional distribution NS_{.|i} over row i has
 * perplexity exp(H_i) = P.  Row i holds c_d nodes at hop distance d, so with
 * beta = 1/(2 sigma_i^2) and weights w_d = e^{-beta (d^2 - 1)} (the common
 * factor e^{-beta} cancels in NS_{j|i}):
 *   Z'(beta) = sum_d c_d w_d,   S'(beta) = sum_d c_d (d^2 - 1) w_d,
 *   exp(H) = Z' exp(beta S'/Z'),
 * which falls from the row size (beta = 0) to c_1 (beta -> inf).  beta_i is
 * found by 60 bisection steps on [0, 512]: mid = (lo + hi)/2, lo = mid when
 * exp(H(mid)) > P, else hi = mid; beta_i = (lo + hi)/2.  Every quantity is
 * FP64 with separately rounded +, -, *, / (this file is compiled without
 * contraction) and the exponential orc_exp below, so the result is a fixed
 * function of (c, P) that the GPU reproduces bit for bit.  Then
 *   g_i(d) = fl32(orc_exp(-(beta_i (d^2 - 1)))),  Z_i = FP32 sum of
 *   fl32(c_d) g_i(d) over d = 1..k,  NS_{j|i} ~ fl32(g_i(d) / Z_i),
 *   q_e = floor((fl32(g_i(d)/Z_i) + fl32(g_j(d)/Z_j)) 2^30).
 * Pinned by orc_exp against the C library's exp, by the perplexity of the
 * calibrated rows evaluated with numpy, and by scipy's root finder.          */

/* e^x in FP64: Cody & Waite's reduction x = m ln2 + r, |r| <= ln2/2 (ln 2
 * split into a 32-significant-bit head, so m ln2_hi is exact, and a tail),
 * the Taylor polynomial of e^r to degree 13 by Horner's rule (remainder below
 * 1e-17 relative), times 2^m built from its bits.  0 below -700.            */
static void orc_exp_coeffs(double c[14])
{
    c[0] = 1.0;
    for (int i = 1; i < 14; ++i) c[i] = c[i - 1] / (double)i;
}

double orc_exp(double x)
{
    const double inv_ln2 = 1.4426950408889634;
    const double ln2_hi = 0.6931471803691238;
    const double ln2_lo = 1.9082149292705877e-10;
    double c[14];
    if (x < -700.0) return 0.0;
    orc_exp_coeffs(c);
    double m = floor(x * inv_ln2 + 0.5);
    double r = (x - m * ln2_hi) - m * ln2_lo;
    double p = c[13];
    for (int i = 12; i >= 0; --i) p = p * r + c[i];
    uint64_t bits = (uint64_t)((int64_t)m + 1023) << 52;
    double scale;
    memcpy(&scale, &bits, sizeof scale);
    return p * scale;
}

/* exp(H_i(beta)) of a row with class counts cnt[0..k-1] (d = 1..k). */
double orc_row_perplexity(uint32_t k, const uint64_t* cnt, double beta)
{
    double z = 0.0, s = 0.0;
    for (uint32_t d = 1; d <= k; ++d) {
        double dd = (double)(d * d - 1);
        double w = orc_exp(-(beta * dd));
        z = z + (double)cnt[d - 1] * w;
        s = s + ((double)cnt[d - 1] * dd) * w;
    }
    return z * orc_exp(beta * (s / z));
}

/* beta_i of a non-empty row (cnt[0] >= 1). */
double orc_calibrate_row(uint32_t k, const uint64_t* cnt, double perplexity)
{
    double lo = 0.0, hi = 512.0;
    for (int it = 0; it < 60; ++it) {
        double mid = (lo + hi) * 0.5;
        if (orc_row_perplexity(k, cnt, mid) > perplexity) lo = mid;
        else hi = mid;
    }
    return (lo + hi) * 0.5;
}

/* The similarity of orc_similarity with sigma_i calibrated per node; beta
 * (n) receives beta_i (0 for an empty row).                                 */
int orc_similarity_perplexity(uint32_t n, const uint64_t* rp, const uint32_t* col, const uint8_t* dist,
                              uint32_t k, float perplexity, double* beta, float* Z, uint32_t* q, uint64_t* r,
                              double* ns)
{
    float* g = (float*)malloc(sizeof(float) * (size_t)(n ? n : 1) * k);
    double* g64 = (double*)malloc(sizeof(double) * (size_t)(n ? n : 1) * k);
    double* Z64 = (double*)malloc(sizeof(double) * (size_t)(n ? n : 1));
    uint64_t* cnt = (uint64_t*)malloc(sizeof(uint64_t) * (k + 1));
    if (!g || !g64 || !Z64 || !cnt) { free(g); free(g64); free(Z64); free(cnt); return -1; }
    for (uint32_t i = 0; i < n; ++i) {
        for (uint32_t d = 0; d <= k; ++d) cnt[d] = 0;
        for (uint64_t e = rp[i]; e < rp[i + 1]; ++e) cnt[dist[e]] += 1;
        if (rp[i + 1] == rp[i]) {
            beta[i] = 0.0;
            Z[i] = 0.0f;
            Z64[i] = 0.0;
            for (uint32_t d = 0; d < k; ++d) { g[(size_t)i * k + d] = 0.0f; g64[(size_t)i * k + d] = 0.0; }
            continue;
        }
        double b = orc_calibrate_row(k, cnt + 1, (double)perplexity);
        beta[i] = b;
        double z64 = 0.0;
        for (uint32_t d = 1; d <= k; ++d) {
            double w = orc_exp(-(b * (double)(d * d - 1)));
            g64[(size_t)i * k + d - 1] = w;
            g[(size_t)i * k + d - 1] = (float)w;
            z64 += (double)cnt[d] * w;
        }
        Z[i] = orc_normaliser(k, cnt + 1, g + (size_t)i * k);
        Z64[i] = z64;
    }
    for (uint32_t i = 0; i < n; ++i) {
        uint64_t acc = 0;
        for (uint64_t e = rp[i]; e < rp[i + 1]; ++e) {
            uint32_t j = col[e];
            uint32_t d = dist[e];
            float p_ji = g[(size_t)i * k + d - 1] / Z[i];
            float p_ij = g[(size_t)j * k + d - 1] / Z[j];
            float s = p_ji + p_ij;
            q[e] = (uint32_t)(s * 1073741824.0f);
            acc += q[e];
            if (ns) ns[e] = (g64[(size_t)i * k + d - 1] / Z64[i] + g64[(size_t)j * k + d - 1] / Z64[j])
                            / (2.0 * (double)n);
        }
        r[i] = acc;
    }
    free(g); free(g64); free(Z64); free(cnt);
    return 0;
}

/* Node weights for the negative-sample alias table: r_i shifted right by
 * s = max(0, bitlength(max r) - 32) so they fit 32 bits.  Returns s.        */
uint32_t orc_node_weights_u32(uint32_t n, const uint64_t* r, uint32_t* r32)
{
    uint64_t mx = 0;
    for (uint32_t i = 0; i < n; ++i) if (r[i] > mx) mx = r[i];
    uint32_t bits = 0;
    while (bits < 64 && (mx >> bits) != 0) ++bits;
    uint32_t s = bits > 32 ? bits - 32 : 0;
    for (uint32_t i = 0; i < n; ++i) r32[i] = (uint32_t)(r[i] >> s);
    return s;
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.2.2: positive pairs are drawn with probability NS_ij and negatives
 * with probability proportional to the node weight.  The paper names no
 * sampler; both draws use Walker alias tables built by the "sweeping"
 * construction of Huebschle-Schneider and Sanders (2019, "Parallel weighted
 * random sampling"), in exact integer arithmetic:
 *   a_i = q_i * N, bucket capacity W = sum q;  light: a_i < W, heavy: a_i >= W.
 *   Lights are visited in index order and filled by the current heavy; a
 *   heavy whose residue drops to <= W becomes a bucket itself, filled by the
 *   next heavy.  own[b] is the exact mass item b keeps in its bucket.
 *   thresh[b] = min(floor(own[b] * 2^32 / W), 2^32 - 1); alias[b] = b when
 *   own[b] == W.
 * Returns 0, or -1 when N == 0 or W == 0 (nothing can be drawn).
 * Pinned by the exact mass invariant (every item's total mass over all
 * buckets equals a_i), brute-force enumeration of the draw probabilities on
 * small tables, and a chi-square test of draws.                             */
int orc_alias_build(uint64_t N, const uint32_t* q, uint32_t* thresh, uint32_t* alias, uint64_t* own)
{
    if (N == 0) return -1;
    uint64_t W = 0;
    for (uint64_t i = 0; i < N; ++i) W += q[i];
    if (W == 0) return -1;
    /* own mass per bucket, then thresholds */
    uint64_t* mass = own ? own : (uint64_t*)malloc(sizeof(uint64_t) * N);
    if (!mass) return -1;
    uint64_t li = 0, hj = 0;
    /* advance li to the first light, hj to the first heavy */
#define A_OF(x) ((uint64_t)q[(x)] * N)
    while (li < N && A_OF(li) >= W) ++li;
    while (hj < N && A_OF(hj) < W) ++hj;
    uint64_t w = A_OF(hj); /* residue of the current heavy */
    while (hj < N) {
        if (w > W && li < N) {
            /* light li is filled by heavy hj */
            mass[li] = A_OF(li);
            alias[li] = (uint32_t)hj;
            w = w - (W - A_OF(li));
            ++li;
            while (li < N && A_OF(li) >= W) ++li;
        } else {
            /* heavy hj becomes a bucket with its residue, filled by the next heavy */
            uint64_t nxt = hj + 1;
            while (nxt < N && A_OF(nxt) < W) ++nxt;
            mass[hj] = w;
            if (nxt < N && w < W) {
                alias[hj] = (uint32_t)nxt;
                w = A_OF(nxt) - (W - w);
            } else {
                alias[hj] = (uint32_t)hj;
                if (nxt < N) w = A_OF(nxt);
            }
            hj = nxt;
        }
    }
#undef A_OF
    for (uint64_t b = 0; b < N; ++b) {
        if (mass[b] >= W) {
            thresh[b] = 0xFFFFFFFFu;
            alias[b] = (uint32_t)b;
        } else {
            u128 t = ((u128)mass[b] << 32) / (u128)W;
            thresh[b] = t > 0xFFFFFFFFu ? 0xFFFFFFFFu : (uint32_t)t;
        }
    }
    if (!own) free(mass);
    return 0;
}

/* One alias draw: bucket = floor(R * N / 2^64) from a 64-bit uniform R,
 * keep the bucket's own item when U < thresh, else its alias.               */
uint64_t orc_alias_draw(uint64_t N, const uint32_t* thresh, const uint32_t* alias, uint64_t R, uint32_t U)
{
    uint64_t b = (uint64_t)(((u128)R * (u128)N) >> 64);
    return U < thresh[b] ? b : (uint64_t)alias[b];
}

/* The draws of one layout sample s of epoch t at level `level` (Sec. 3.2.2):
 * the positive pair (i, j) from the edge table, then M negatives from the node
 * table.  Random words: 0-1 edge bucket, 2 edge accept, 3+3m..5+3m negative m. */
void orc_sample_draws(uint64_t seed, uint32_t gid, uint32_t level, uint32_t t, uint32_t s, uint32_t M,
                      uint64_t nnz, const uint32_t* e_src, const uint32_t* e_dst,
                      const uint32_t* e_thresh, const uint32_t* e_alias,
                      uint32_t n0, const uint32_t* v_thresh, const uint32_t* v_alias,
                      uint32_t* out_i, uint32_t* out_j, uint32_t* out_neg)
{
    uint32_t tag = orc_tag(0, gid, level);
    uint64_t R = (uint64_t)orc_word(seed, s, t, tag, 0) | ((uint64_t)orc_word(seed, s, t, tag, 1) << 32);
    uint32_t U = orc_word(seed, s, t, tag, 2);
    uint64_t e = orc_alias_draw(nnz, e_thresh, e_alias, R, U);
    *out_i = e_src[e];
    *out_j = e_dst[e];
    for (uint32_t m = 0; m < M; ++m) {
        uint64_t Rm = (uint64_t)orc_word(seed, s, t, tag, 3 + 3 * m) |
                      ((uint64_t)orc_word(seed, s, t, tag, 4 + 3 * m) << 32);
        uint32_t Um = orc_word(seed, s, t, tag, 5 + 3 * m);
        out_neg[m] = (uint32_t)orc_alias_draw(n0, v_thresh, v_alias, Rm, Um);
    }
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.2.2 Eq. 12, with the readings: the attractive term is the exact
 * derivative of log (1 + d^{2b})^{-1}, i.e. -2b d^{2b-2} (y_i - y_j) /
 * (1 + d^{2b}); the repulsive term gamma 2b (y_i - y_m) / (d^2 (1 + d^{2b}));
 * a pair at distance 0 contributes nothing; each component of each pair force
 * is clipped to [-clip, clip].  FP64.  Pinned by finite differences of the
 * sampled objective (Eq. 11) and by the equilibrium distance d^{2b} = M gamma. */
static double orc_clip(double x, double c) { return x > c ? c : (x < -c ? -c : x); }

void orc_pair_force(double dx, double dy, int repulsive, double gamma, double b, double clip, double* fx, double* fy)
{
    double d2 = dx * dx + dy * dy;
    *fx = 0.0; *fy = 0.0;
    if (!(d2 > 0.0)) return;
    double d2b = pow(d2, b);
    double coef;
    if (repulsive)
        coef = gamma * 2.0 * b / (d2 * (1.0 + d2b));
    else
        coef = -2.0 * b * pow(d2, b - 1.0) / (1.0 + d2b);
    *fx = orc_clip(coef * dx, clip);
    *fy = orc_clip(coef * dy, clip);
}

/* The per-sample objective of Eq. 11 with the unnormalised t-kernel
 * LP = (1 + d^{2b})^{-1}: log LP_ij + sum_m gamma log(1 - LP_ijm).  Used by
 * the finite-difference pin only.                                            */
double orc_sample_objective(const double* yi, const double* yj, const double* yneg, uint32_t M, double gamma, double b)
{
    double dx = yi[0] - yj[0], dy = yi[1] - yj[1];
    double v = -log1p(pow(dx * dx + dy * dy, b));
    for (uint32_t m = 0; m < M; ++m) {
        double ex = yi[0] - yneg[2 * m], ey = yi[1] - yneg[2 * m + 1];
        double lp = 1.0 / (1.0 + pow(ex * ex + ey * ey, b));
        v += gamma * log(1.0 - lp);
    }
    return v;
}

/* ------------------------------------------------------------------------ */
/* The force terms of one sample (Sec. 3.2.2, Eqs. 11-12), computed from the
 * positions in Y.  The sampled term of Eq. 11 depends on y_a, y_c and every
 * y_cm, so its stochastic gradient moves all of them: the source by
 * attr + sum_m rep_m (Eq. 12), the positive target by -attr, each negative by
 * -rep_m.  Returns the number of (node, fx, fy) contributions written.      */
static uint32_t orc_sample_forces(const double* Y, uint32_t a, uint32_t c, const uint32_t* cneg, uint32_t M,
                                  double gamma, double b, double clip,
                                  uint32_t* node, double* fxs, double* fys)
{
    double Fx = 0.0, Fy = 0.0, fx, fy;
    uint32_t cnt = 1;
    orc_pair_force(Y[2 * a] - Y[2 * c], Y[2 * a + 1] - Y[2 * c + 1], 0, gamma, b, clip, &fx, &fy);
    Fx += fx; Fy += fy;
    node[cnt] = c; fxs[cnt] = -fx; fys[cnt] = -fy; ++cnt;
    for (uint32_t m = 0; m < M; ++m) {
        uint32_t cm = cneg[m];
        if (cm == a || cm == c) continue;
        orc_pair_force(Y[2 * a] - Y[2 * cm], Y[2 * a + 1] - Y[2 * cm + 1], 1, gamma, b, clip, &fx, &fy);
        Fx += fx; Fy += fy;
        node[cnt] = cm; fxs[cnt] = -fx; fys[cnt] = -fy; ++cnt;
    }
    node[0] = a; fxs[0] = Fx; fys[0] = Fy;
    return cnt;
}

/* One level of the layout optimisation (Sec. 3.2.2 "During optimization ...";
 * Sec. 3.2.3 "We optimize the graph layout jointly ...").
 *   Each epoch t in [t_begin, t_end) of T draws n_l samples s = 0..n_l-1 from
 *   the level-0 tables and maps every drawn node through anc (level-0 id ->
 *   level-l id; NULL = identity): a = anc(i), c = anc(j), c_m = anc(j_m);
 *   negatives with c_m == a or c_m == c are skipped.  lr_t = lr0 (1 - t/T).
 *   mode 0 (synchronous): the epoch's samples are cut into `substeps` equal
 *     consecutive runs of ceil(n_l / substeps) samples; the forces of one run
 *     are all computed from the positions at its start, summed per node (G),
 *     then applied: Y += lr_t G.
 *   mode 1 (sequential; the reference of the asynchronous GPU mode): the
 *     forces of each sample are computed from the current positions and
 *     applied at once, Y += lr_t F.
 * Y is n_l x 2, FP64, updated in place.  Returns 0.                        */
int orc_layout_level(uint64_t seed, uint32_t gid, uint32_t level,
                     uint64_t nnz, const uint32_t* e_src, const uint32_t* e_dst,
                     const uint32_t* e_thresh, const uint32_t* e_alias,
                     uint32_t n0, const uint32_t* v_thresh, const uint32_t* v_alias,
                     uint32_t nl, const uint32_t* anc, double* Y,
                     uint32_t T, uint32_t t_begin, uint32_t t_end, uint32_t M,
                     double gamma, double b, double lr0, double clip, int mode, uint32_t substeps)
{
    double* G = (double*)calloc((size_t)nl * 2 + 2, sizeof(double));
    uint32_t* neg = (uint32_t*)malloc(sizeof(uint32_t) * (M + 1));
    uint32_t* cneg = (uint32_t*)malloc(sizeof(uint32_t) * (M + 1));
    uint32_t* node = (uint32_t*)malloc(sizeof(uint32_t) * (M + 2));
    double* fxs = (double*)malloc(sizeof(double) * (M + 2));
    double* fys = (double*)malloc(sizeof(double) * (M + 2));
    if (!G || !neg || !cneg || !node || !fxs || !fys) {
        free(G); free(neg); free(cneg); free(node); free(fxs); free(fys);
        return -1;
    }
    if (substeps == 0) substeps = 1;
    uint32_t chunk = (uint32_t)(((uint64_t)nl + substeps - 1) / substeps);
    if (chunk == 0) chunk = 1;
    for (uint32_t t = t_begin; t < t_end; ++t) {
        double lr = lr0 * (1.0 - (double)t / (double)T);
        for (uint32_t s0 = 0; s0 < nl; s0 += chunk) {
            uint32_t s1 = (nl - s0 < chunk) ? nl : s0 + chunk;
            if (mode == 0) memset(G, 0, sizeof(double) * (size_t)nl * 2);
            for (uint32_t s = s0; s < s1; ++s) {
                uint32_t i, j;
                orc_sample_draws(seed, gid, level, t, s, M, nnz, e_src, e_dst, e_thresh, e_alias,
                                 n0, v_thresh, v_alias, &i, &j, neg);
                uint32_t a = anc ? anc[i] : i;
                uint32_t c = anc ? anc[j] : j;
                for (uint32_t m = 0; m < M; ++m) cneg[m] = anc ? anc[neg[m]] : neg[m];
                uint32_t cnt = orc_sample_forces(Y, a, c, cneg, M, gamma, b, clip, node, fxs, fys);
                for (uint32_t x = 0; x < cnt; ++x) {
                    if (mode == 0) {
                        G[2 * node[x]] += fxs[x];
                        G[2 * node[x] + 1] += fys[x];
                    } else {
                        Y[2 * node[x]] += lr * fxs[x];
                        Y[2 * node[x] + 1] += lr * fys[x];
                    }
                }
            }
            if (mode == 0)
                for (uint32_t v = 0; v < nl; ++v) {
                    Y[2 * v] += lr * G[2 * v];
                    Y[2 * v + 1] += lr * G[2 * v + 1];
                }
        }
    }
    free(G); free(neg); free(cneg); free(node); free(fxs); free(fys);
    return 0;
}

/* Sec. 3.2.3 "Layout of the coarsest graph": random initialisation, here
 * uniform in [-scale, scale]^2 from the Philox stream (purpose 1): word 0 ->
 * x, word 1 -> y; u = (w >> 8) 2^-24, coordinate = fl32((2u - 1) * scale),
 * then widened to FP64.                                                      */
void orc_init_positions(uint64_t seed, uint32_t gid, uint32_t level, uint32_t n, float scale, double* Y)
{
    uint32_t tag = orc_tag(1, gid, level);
    for (uint32_t v = 0; v < n; ++v) {
        for (uint32_t c = 0; c < 2; ++c) {
            uint32_t w = orc_word(seed, v, 0, tag, c);
            float u = (float)(w >> 8) * 5.9604644775390625e-08f; /* 2^-24 */
            float x = (2.0f * u - 1.0f) * scale;
            Y[2 * v + c] = (double)x;
        }
    }
}

/* Sec. 3.2.3 "Refinement": a fine node takes the position of the coarse node
 * it was merged into.                                                        */
void orc_interpolate(uint32_t n_fine, const uint32_t* parent, const double* Yc, double* Yf)
{
    for (uint32_t v = 0; v < n_fine; ++v) {
        Yf[2 * v] = Yc[2 * parent[v]];
        Yf[2 * v + 1] = Yc[2 * parent[v] + 1];
    }
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.2.3 "Coarsening" by heavy-edge matching (the default rule; the
 * paper's own star grouping is orc_star_group below).  Deterministic
 * handshake rounds: in round r every unmatched
 * node proposes to its unmatched neighbour with the largest key (edge weight,
 * then Philox hash of (min id, max id, round) under purpose 2, then the
 * smaller neighbour id); two nodes that propose to each other are matched.
 * Nodes still unmatched after `rounds` rounds stay single (match[v] = v).
 * Pinned by matching validity and by exact equality with brute force.       */
int orc_hem_match(uint32_t n, const uint64_t* rp, const uint32_t* col, const uint32_t* w,
                  uint64_t seed, uint32_t gid, uint32_t level, uint32_t rounds, uint32_t* match)
{
    uint32_t* prop = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n ? n : 1));
    if (!prop) return -1;
    uint32_t tag = orc_tag(2, gid, level);
    for (uint32_t v = 0; v < n; ++v) match[v] = ORC_NONE;
    for (uint32_t r = 0; r < rounds; ++r) {
        for (uint32_t v = 0; v < n; ++v) {
            prop[v] = ORC_NONE;
            if (match[v] != ORC_NONE) continue;
            uint32_t best = ORC_NONE, bw = 0, bh = 0;
            for (uint64_t e = rp[v]; e < rp[v + 1]; ++e) {
                uint32_t u = col[e];
                if (u == v || match[u] != ORC_NONE) continue;
                uint32_t lo = u < v ? u : v, hi = u < v ? v : u;
                uint32_t h = orc_word(seed, lo, hi, tag, 4u * r);
                uint32_t we = w ? w[e] : 1u;
                int better = 0;
                if (best == ORC_NONE) better = 1;
                else if (we != bw) better = we > bw;
                else if (h != bh) better = h > bh;
                else better = u < best;
                if (better) { best = u; bw = we; bh = h; }
            }
            prop[v] = best;
        }
        for (uint32_t v = 0; v < n; ++v) {
            uint32_t u = prop[v];
            if (u != ORC_NONE && prop[u] == v) match[v] = u;
        }
    }
    for (uint32_t v = 0; v < n; ++v)
        if (match[v] == ORC_NONE) match[v] = v;
    free(prop);
    return 0;
}

/* Cluster ids: the representative of v is min(v, match[v]); representatives
 * are numbered in increasing id order.  Returns the number of coarse nodes.  */
uint32_t orc_cluster_ids(uint32_t n, const uint32_t* match, uint32_t* cid)
{
    uint32_t nc = 0;
    for (uint32_t v = 0; v < n; ++v) {
        uint32_t m = match[v];
        if (m >= v) cid[v] = nc++;
    }
    for (uint32_t v = 0; v < n; ++v) {
        uint32_t m = match[v];
        if (m < v) cid[v] = cid[m];
    }
    return nc;
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.2.3 "Coarsening" as the paper states it (Fig. 3): pick a node at
 * random among those not yet grouped, make it and its still ungrouped
 * first-order neighbours one node of the coarser graph, and repeat until no
 * node is left.  Picking uniformly among the ungrouped nodes is the same as
 * walking one uniformly random order of all nodes and skipping the grouped
 * ones; the order is increasing (prio[v], v).  prio comes in as an input
 * (orc_star_priorities draws it) so that tests can set it by hand.
 * centre[v] = the picked node whose group v joined (centre[c] = c for a
 * picked node).  Pinned by hand-worked paths, stars, cycles and cliques and
 * by the independent-set characterisation on random graphs.               */
static int orc_cmp_u64(const void* a, const void* b)
{
    uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
    return (x > y) - (x < y);
}

int orc_star_group(uint32_t n, const uint64_t* rp, const uint32_t* col, const uint32_t* prio, uint32_t* centre)
{
    uint64_t* order = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(n ? n : 1));
    if (!order) return -1;
    for (uint32_t v = 0; v < n; ++v) {
        order[v] = ((uint64_t)prio[v] << 32) | v;
        centre[v] = ORC_NONE;
    }
    qsort(order, n, sizeof(uint64_t), orc_cmp_u64);
    for (uint32_t x = 0; x < n; ++x) {
        uint32_t v = (uint32_t)order[x];
        if (centre[v] != ORC_NONE) continue;      /* already grouped: skipped */
        centre[v] = v;
        for (uint64_t e = rp[v]; e < rp[v + 1]; ++e)
            if (centre[col[e]] == ORC_NONE) centre[col[e]] = v;
    }
    free(order);
    return 0;
}

/* The random order of the grouping at `level`: word 0 of the Philox stream
 * (v, 0, tag) with purpose 3.                                              */
void orc_star_priorities(uint32_t n, uint64_t seed, uint32_t gid, uint32_t level, uint32_t* prio)
{
    uint32_t tag = orc_tag(3, gid, level);
    for (uint32_t v = 0; v < n; ++v) prio[v] = orc_word(seed, v, 0, tag, 0);
}

/* Coarse node ids of a grouping: picked nodes numbered in increasing id
 * order, every node takes its centre's number.  Returns the number of groups. */
uint32_t orc_star_cluster_ids(uint32_t n, const uint32_t* centre, uint32_t* cid)
{
    uint32_t nc = 0;
    for (uint32_t v = 0; v < n; ++v)
        if (centre[v] == v) cid[v] = nc++;
    for (uint32_t v = 0; v < n; ++v)
        if (centre[v] != v) cid[v] = cid[centre[v]];
    return nc;
}

typedef struct { uint32_t a, b, w; } orc_triple;
static int orc_cmp_triple(const void* x, const void* y)
{
    const orc_triple* p = (const orc_triple*)x;
    const orc_triple* q = (const orc_triple*)y;
    if (p->a != q->a) return (p->a > q->a) - (p->a < q->a);
    return (p->b > q->b) - (p->b < q->b);
}

/* Coarse graph: edge (cid u, cid v) for every fine edge whose ends fall in
 * different clusters, weights summed; rows sorted by column.  Call with
 * out_col == NULL to get the coarse row pointer and the edge count only.    */
int64_t orc_contract(uint32_t n, const uint64_t* rp, const uint32_t* col, const uint32_t* w,
                     const uint32_t* cid, uint32_t nc, uint64_t* out_rp, uint32_t* out_col, uint32_t* out_w)
{
    uint64_t m = rp[n];
    orc_triple* t = (orc_triple*)malloc(sizeof(orc_triple) * (size_t)(m ? m : 1));
    if (!t) return -1;
    uint64_t cnt = 0;
    for (uint32_t u = 0; u < n; ++u)
        for (uint64_t e = rp[u]; e < rp[u + 1]; ++e) {
            uint32_t a = cid[u], b = cid[col[e]];
            if (a == b) continue;
            t[cnt].a = a; t[cnt].b = b; t[cnt].w = w ? w[e] : 1u;
            ++cnt;
        }
    qsort(t, cnt, sizeof(orc_triple), orc_cmp_triple);
    for (uint32_t c = 0; c <= nc; ++c) out_rp[c] = 0;
    uint64_t nout = 0;
    for (uint64_t x = 0; x < cnt; ++x) {
        if (x > 0 && t[x].a == t[x - 1].a && t[x].b == t[x - 1].b) {
            if (out_col) out_w[nout - 1] += t[x].w;
            continue;
        }
        if (out_col) { out_col[nout] = t[x].b; out_w[nout] = t[x].w; }
        out_rp[t[x].a + 1] += 1;
        ++nout;
    }
    for (uint32_t c = 0; c < nc; ++c) out_rp[c + 1] += out_rp[c];
    free(t);
    return (int64_t)nout;
}

/* ------------------------------------------------------------------------ */
/* Sec. 4.1 Eq. 15, neighbourhood preservation: mean Jaccard index of
 * NNG(v_i, k_eval) and the k_i nearest layout neighbours of y_i
 * (k_i = #NNG(v_i, k_eval)), layout ties broken by node id.  Evaluated over
 * the listed nodes (all nodes, or a sample).  Nodes with an empty NNG are
 * skipped.  Returns the mean over counted nodes; *counted gets their number. */
typedef struct { double d2; uint32_t id; } orc_nb;
static int orc_nb_less(const orc_nb* x, const orc_nb* y)
{
    return x->d2 < y->d2 || (x->d2 == y->d2 && x->id < y->id);
}
static void orc_select(orc_nb* a, int64_t lo, int64_t hi, int64_t k)
{
    /* quickselect: afterwards a[lo..k) are the k smallest (unordered) */
    while (hi - lo > 1) {
        orc_nb p = a[lo + (hi - lo) / 2];
        int64_t i = lo, j = hi - 1;
        while (i <= j) {
            while (orc_nb_less(&a[i], &p)) ++i;
            while (orc_nb_less(&p, &a[j])) --j;
            if (i <= j) { orc_nb tmp = a[i]; a[i] = a[j]; a[j] = tmp; ++i; --j; }
        }
        if (k <= j) hi = j + 1;
        else if (k >= i) lo = i;
        else return;
    }
}

double orc_neighbourhood_preservation(uint32_t n, const uint64_t* rp, const uint32_t* col, const double* Y,
                                      uint32_t k_eval, uint32_t nsel, const uint32_t* sel, uint32_t* counted)
{
    int32_t* dist = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
    uint32_t* queue = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n ? n : 1));
    orc_nb* nb = (orc_nb*)malloc(sizeof(orc_nb) * (size_t)(n ? n : 1));
    uint8_t* in_g = (uint8_t*)calloc(n ? n : 1, 1);
    if (!dist || !queue || !nb || !in_g) { free(dist); free(queue); free(nb); free(in_g); return -1.0; }
    for (uint32_t v = 0; v < n; ++v) dist[v] = -1;
    double acc = 0.0;
    uint32_t cntd = 0;
    for (uint32_t x = 0; x < nsel; ++x) {
        uint32_t i = sel ? sel[x] : x;
        uint32_t cnt = orc_bfs(n, rp, col, k_eval, i, dist, queue);
        uint32_t ki = cnt - 1;
        if (ki > 0) {
            for (uint32_t q = 1; q < cnt; ++q) in_g[queue[q]] = 1;
            uint32_t m = 0;
            for (uint32_t v = 0; v < n; ++v) {
                if (v == i) continue;
                double dx = Y[2 * v] - Y[2 * i], dy = Y[2 * v + 1] - Y[2 * i + 1];
                nb[m].d2 = dx * dx + dy * dy;
                nb[m].id = v;
                ++m;
            }
            orc_select(nb, 0, m, ki);
            uint32_t inter = 0;
            for (uint32_t q = 0; q < ki; ++q) inter += in_g[nb[q].id];
            acc += (double)inter / (double)(2 * ki - inter);
            ++cntd;
            for (uint32_t q = 1; q < cnt; ++q) in_g[queue[q]] = 0;
        }
        for (uint32_t q = 0; q < cnt; ++q) dist[queue[q]] = -1;
    }
    free(dist); free(queue); free(nb); free(in_g);
    if (counted) *counted = cntd;
    return cntd ? acc / cntd : 0.0;
}

/* Sec. 4.1 Eq. 16, normalised stress with w_ij = SPD^-2 and the optimal
 * scale alpha* = sum w SPD L / sum w L^2 (the closed-form minimiser), over the
 * connected pairs (i, j), i in the listed sources, j != i.  With all n nodes
 * as sources this is the paper's definition; with a sample of sources the
 * sum is scaled by n / nsel.                                                 */
double orc_stress(uint32_t n, const uint64_t* rp, const uint32_t* col, const double* Y,
                  uint32_t nsel, const uint32_t* sel)
{
    int32_t* dist = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
    uint32_t* queue = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n ? n : 1));
    if (!dist || !queue) { free(dist); free(queue); return -1.0; }
    for (uint32_t v = 0; v < n; ++v) dist[v] = -1;
    double swdl = 0.0, swll = 0.0, swdd = 0.0;
    for (uint32_t x = 0; x < nsel; ++x) {
        uint32_t i = sel ? sel[x] : x;
        uint32_t cnt = orc_bfs(n, rp, col, 0xFFFFFFFFu, i, dist, queue);
        for (uint32_t q = 1; q < cnt; ++q) {
            uint32_t j = queue[q];
            double d = (double)dist[j];
            double dx = Y[2 * i] - Y[2 * j], dy = Y[2 * i + 1] - Y[2 * j + 1];
            double L = sqrt(dx * dx + dy * dy);
            double wgt = 1.0 / (d * d);
            swdl += wgt * d * L;
            swll += wgt * L * L;
            swdd += wgt * d * d;
        }
        for (uint32_t q = 0; q < cnt; ++q) dist[queue[q]] = -1;
    }
    free(dist); free(queue);
    double alpha = swll > 0.0 ? swdl / swll : 0.0;
    /* sum w (alpha L - d)^2 = alpha^2 swll - 2 alpha swdl + swdd */
    double s = alpha * alpha * swll - 2.0 * alpha * swdl + swdd;
    if (s < 0.0) s = 0.0;
    double scale = nsel ? (double)n / (double)nsel : 0.0;
    return s * scale / ((double)n * (double)n);
}

/* ------------------------------------------------------------------------ */
/* Sec. 4.1 Eq. 17, crosslessness: 1 - sqrt(c / c_max) (1 when c_max = 0),
 * c the number of unordered pairs of edges that cross, c_max =
 * |E|(|E|-1)/2 - (1/2) sum_v deg(v)(deg(v)-1).  Edges are the graph's
 * undirected edges drawn as straight segments.  To decide crossings exactly,
 * positions are first snapped per axis to the grid 0..2^30-1 over the
 * layout's bounding box, q = floor((x - min) / (max - min) * (2^30 - 1) + 0.5)
 * in FP64 (q = 0 when max = min); an affine map changes no crossing, so only
 * near-degenerate pairs can be decided differently from the unsnapped
 * drawing.  Two edges without a common endpoint cross when each separates
 * the other's endpoints strictly: orient(a,b,c) and orient(a,b,d) have
 * opposite signs and so have orient(c,d,a) and orient(c,d,b), with
 * orient(a,b,c) = (bx-ax)(cy-ay) - (by-ay)(cx-ax) exact in 64-bit integers
 * (touching and collinear pairs do not count).  Brute force over all pairs.
 * Pinned by hand-drawn cases, closed forms on grids and stars, and exact
 * rational segment intersection (sympy) on random drawings.                 */
static void orc_snap(uint32_t n, const double* Y, int axis, int64_t* q)
{
    double lo = 0.0, hi = 0.0;
    for (uint32_t v = 0; v < n; ++v) {
        double x = Y[2 * v + axis];
        if (v == 0 || x < lo) lo = x;
        if (v == 0 || x > hi) hi = x;
    }
    double span = hi - lo;
    for (uint32_t v = 0; v < n; ++v)
        q[v] = span > 0.0 ? (int64_t)floor((Y[2 * v + axis] - lo) / span * 1073741823.0 + 0.5) : 0;
}

static int orc_sign(int64_t x) { return (x > 0) - (x < 0); }

static int64_t orc_orient(const int64_t* qx, const int64_t* qy, uint32_t a, uint32_t b, uint32_t c)
{
    return (qx[b] - qx[a]) * (qy[c] - qy[a]) - (qy[b] - qy[a]) * (qx[c] - qx[a]);
}

int orc_crossings(uint32_t n, const uint64_t* rp, const uint32_t* col, const double* Y,
                  uint64_t* crossings, double* crosslessness)
{
    int64_t* qx = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n ? n : 1));
    int64_t* qy = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n ? n : 1));
    uint64_t m = rp[n] / 2;
    uint32_t* eu = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(m ? m : 1));
    uint32_t* ev = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(m ? m : 1));
    if (!qx || !qy || !eu || !ev) { free(qx); free(qy); free(eu); free(ev); return -1; }
    orc_snap(n, Y, 0, qx);
    orc_snap(n, Y, 1, qy);
    uint64_t ne = 0;
    for (uint32_t u = 0; u < n; ++u)
        for (uint64_t e = rp[u]; e < rp[u + 1]; ++e)
            if (col[e] > u) { eu[ne] = u; ev[ne] = col[e]; ++ne; }
    uint64_t c = 0;
    for (uint64_t x = 0; x < ne; ++x)
        for (uint64_t y = x + 1; y < ne; ++y) {
            uint32_t a = eu[x], b = ev[x], p = eu[y], r = ev[y];
            if (a == p || a == r || b == p || b == r) continue;
            int s1 = orc_sign(orc_orient(qx, qy, a, b, p)), s2 = orc_sign(orc_orient(qx, qy, a, b, r));
            int s3 = orc_sign(orc_orient(qx, qy, p, r, a)), s4 = orc_sign(orc_orient(qx, qy, p, r, b));
            if (s1 * s2 < 0 && s3 * s4 < 0) ++c;
        }
    /* c_max = |E|(|E|-1)/2 - sum_v deg(v)(deg(v)-1)/2, exact */
    unsigned __int128 cmax = (unsigned __int128)ne * (ne ? ne - 1 : 0) / 2;
    unsigned __int128 adj = 0;
    for (uint32_t v = 0; v < n; ++v) {
        uint64_t d = rp[v + 1] - rp[v];
        adj += (unsigned __int128)d * (d ? d - 1 : 0) / 2;
    }
    cmax -= adj;
    *crossings = c;
    *crosslessness = cmax > 0 ? 1.0 - sqrt((double)c / (double)cmax) : 1.0;
    free(qx); free(qy); free(eu); free(ev);
    return 0;
}

/* Sec. 4.1 Eq. 19, minimum angle: 1 - mean over nodes of
 * |theta(v) - theta_min(v)| / theta(v), theta(v) = 2 pi / deg(v), theta_min(v)
 * the smallest angle between two edges at v that are consecutive around it
 * (directions atan2(y_u - y_v, x_u - x_v), sorted; the wrap-around gap
 * included).  The mean runs over nodes with an edge (isolated nodes are never
 * drawn); a node of degree 1 has no angle and deviates by 0.  Pinned by
 * closed forms on grids, regular stars and a path.                           */
static int orc_cmp_double(const void* a, const void* b)
{
    double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

double orc_min_angle(uint32_t n, const uint64_t* rp, const uint32_t* col, const double* Y)
{
    uint64_t dmax = 0;
    for (uint32_t v = 0; v < n; ++v)
        if (rp[v + 1] - rp[v] > dmax) dmax = rp[v + 1] - rp[v];
    double* ang = (double*)malloc(sizeof(double) * (size_t)(dmax ? dmax : 1));
    if (!ang) return -1.0;
    const double two_pi = 6.283185307179586;
    double dev = 0.0;
    uint64_t counted = 0;
    for (uint32_t v = 0; v < n; ++v) {
        uint64_t d = rp[v + 1] - rp[v];
        if (d == 0) continue;
        ++counted;
        if (d == 1) continue;
        for (uint64_t e = rp[v]; e < rp[v + 1]; ++e) {
            uint32_t u = col[e];
            ang[e - rp[v]] = atan2(Y[2 * u + 1] - Y[2 * v + 1], Y[2 * u] - Y[2 * v]);
        }
        qsort(ang, d, sizeof(double), orc_cmp_double);
        double mn = two_pi - (ang[d - 1] - ang[0]);
        for (uint64_t x = 1; x < d; ++x)
            if (ang[x] - ang[x - 1] < mn) mn = ang[x] - ang[x - 1];
        double theta = two_pi / (double)d;
        dev += fabs(theta - mn) / theta;
    }
    free(ang);
    return counted ? 1.0 - dev / (double)counted : 1.0;
}
