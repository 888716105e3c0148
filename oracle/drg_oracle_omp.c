/*
 * drg_oracle_omp.c -- the paper's multi-threaded optimisation (Sec. 4.3) as a
 * CPU performance baseline: the oracle's sequential level loop with each
 * epoch's samples shared out over OpenMP threads that read and update the
 * positions without locks (asynchronous SGD, "Hogwild").
 *
 * TEST INFRASTRUCTURE, like drg_oracle.c, whose arithmetic it reuses
 * unchanged (it is included below): only the test-suite and the benchmark's
 * optional CPU legs load it.  Each position update is an atomic add so that
 * concurrent updates are not lost; reads race with them, as in the paper's
 * lock-free threads.  With one thread the loop is orc_layout_level in
 * sequential mode exactly (same samples in the same order, same operations).
 * Build: gcc -fopenmp; optional (no OpenMP, no library).
 */
#include "drg_oracle.c"

#include <omp.h>

int orc_layout_level_omp(uint64_t seed, uint32_t gid, uint32_t level,
                         uint64_t nnz, const uint32_t* e_src, const uint32_t* e_dst,
                         const uint32_t* e_thresh, const uint32_t* e_alias,
                         uint32_t n0, const uint32_t* v_thresh, const uint32_t* v_alias,
                         uint32_t nl, const uint32_t* anc, double* Y,
                         uint32_t T, uint32_t t_begin, uint32_t t_end, uint32_t M,
                         double gamma, double b, double lr0, double clip, int threads)
{
    int fail = 0;
    for (uint32_t t = t_begin; t < t_end; ++t) {
        double lr = lr0 * (1.0 - (double)t / (double)T);
#pragma omp parallel num_threads(threads) reduction(| : fail)
        {
            uint32_t* neg = (uint32_t*)malloc(sizeof(uint32_t) * (M + 1));
            uint32_t* cneg = (uint32_t*)malloc(sizeof(uint32_t) * (M + 1));
            uint32_t* node = (uint32_t*)malloc(sizeof(uint32_t) * (M + 2));
            double* fxs = (double*)malloc(sizeof(double) * (M + 2));
            double* fys = (double*)malloc(sizeof(double) * (M + 2));
            int ok = neg && cneg && node && fxs && fys;
            if (!ok) fail = 1;
#pragma omp for schedule(static)
            for (uint32_t s = 0; s < nl; ++s) {
                if (!ok) continue;
                uint32_t i, j;
                orc_sample_draws(seed, gid, level, t, s, M, nnz, e_src, e_dst, e_thresh, e_alias,
                                 n0, v_thresh, v_alias, &i, &j, neg);
                uint32_t a = anc ? anc[i] : i;
                uint32_t c = anc ? anc[j] : j;
                for (uint32_t m = 0; m < M; ++m) cneg[m] = anc ? anc[neg[m]] : neg[m];
                uint32_t cnt = orc_sample_forces(Y, a, c, cneg, M, gamma, b, clip, node, fxs, fys);
                for (uint32_t x = 0; x < cnt; ++x) {
                    double ux = lr * fxs[x], uy = lr * fys[x];
#pragma omp atomic update
                    Y[2 * node[x]] += ux;
#pragma omp atomic update
                    Y[2 * node[x] + 1] += uy;
                }
            }
            free(neg); free(cneg); free(node); free(fxs); free(fys);
        }
        if (fail) return -1;
    }
    return 0;
}

int orc_omp_max_threads(void) { return omp_get_max_threads(); }
