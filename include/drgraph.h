/*
 * drgraph.h -- C ABI of the GB300 DRGraph layout library (libdrgraph.so).
 *
 * DRGraph (Zhu et al., arXiv 2008.07799) lays out a graph by negative-sampling
 * SGD on a sparse t-SNE-style objective, coarse to fine over a multilevel
 * hierarchy.  This library runs every step of that path in hand-written CUDA
 * kernels for sm_103a on one GPU:
 *
 *   drg_graph_from_edges       Sec. 3.1   undirected unweighted G = (V, E)
 *   drg_build_distance_matrix  Sec. 3.2.1 sparse k-order distance matrix (Eq. 8),
 *                                          similarity (Eqs. 4, 9) and the
 *                                          sampling tables of Sec. 3.2.2
 *                                          (_ex: sigma_i per node by perplexity)
 *   drg_coarsen / drg_build_hierarchy
 *                              Sec. 3.2.3 coarsening (the paper's star grouping
 *                                          or heavy-edge matching)
 *   drg_layout_level           Sec. 3.2.2-3.2.3  epochs of negative-sampling SGD
 *                                          (Eqs. 11-12) at one level, samples
 *                                          drawn on G^0, gradients forwarded to
 *                                          the level through the ancestor map
 *                                          (or on the level's own tables)
 *   drg_interpolate            Sec. 3.2.3 refinement: a fine node starts at its
 *                                          coarse node's position
 *   drg_layout / drg_layout_edges      the whole pipeline
 *   drg_layout_batch           many independent graphs in one launch per step
 *   drg_crossings / drg_min_angle
 *                              Sec. 4.1   crosslessness and minimum angle of a
 *                                          drawing
 *
 * Conventions
 *   - Every call returns a drg_status; nothing aborts.  On error the context's
 *     message (drg_last_error) says what failed.  Invalid arguments return
 *     DRG_EINVAL before any device work is queued.
 *   - Handles (drg_ctx, drg_graph, drg_dmat, drg_hier) are opaque and owned by
 *     the library; free each with its *_destroy call.  Destroying a context
 *     frees nothing else: destroy its handles first.
 *   - Position buffers are caller-owned, interleaved (x, y) FP32 pairs
 *     (float[2 * n]), on the device unless a call says otherwise.
 *   - All device work of a context is ordered on its CUDA stream (given to
 *     drg_create, or created by it).  Calls that must size an output read
 *     counts back from the device and therefore synchronise the stream; every
 *     such call says "synchronises".
 *   - Node ids are uint32 (n < 2^32 - 1); the distance matrix must have fewer
 *     than 2^32 entries.
 */
#ifndef DRGRAPH_H
#define DRGRAPH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DRG_OK = 0,
    DRG_EINVAL = 1,        /* invalid argument (null pointer, id out of range, bad size) */
    DRG_ENOMEM = 2,        /* device or host allocation failed */
    DRG_ECUDA = 3,         /* a CUDA runtime call failed */
    DRG_ETIMEOUT = 4,      /* a device-side wait exceeded its iteration limit */
    DRG_EUNSUPPORTED = 5,  /* the request exceeds a documented limit */
    DRG_EEMPTY = 6         /* the graph has no edge, so nothing can be sampled */
} drg_status;

typedef struct drg_ctx drg_ctx;
typedef struct drg_graph drg_graph;
typedef struct drg_dmat drg_dmat;
typedef struct drg_hier drg_hier;

/* Parameters of a layout run.  drg_params_default fills the paper's values
 * (Sec. 4 "Parameters": M = 5, gamma = 0.1, k = 1; Sec. 4.2: gamma = 0.01 on
 * the coarsest level; supplement: b) and the library's defaults for what the
 * paper leaves open. */
typedef struct {
    uint32_t k;              /* order of the distance matrix, 1..15 (Sec. 3.2.1) */
    uint32_t M;              /* negative samples per positive sample, 0..64 (Sec. 3.2.2) */
    uint32_t epochs;         /* epochs per level; an epoch draws n_l samples */
    float gamma;             /* weight of the negative samples (Eq. 10) */
    float gamma_coarsest;    /* gamma on the coarsest level of a hierarchy (Sec. 4.2) */
    float b;                 /* shape of the proximity kernel (1 + d^{2b})^{-1} (Eq. 5) */
    float lr0;               /* learning rate of epoch 0; epoch t uses lr0 (1 - t/epochs) */
    float sigma;             /* Gaussian width of the node similarity (Eq. 9) */
    float clip;              /* each component of each pair force is clipped to [-clip, clip] */
    float init_scale;        /* coarsest positions uniform in [-init_scale, init_scale]^2 */
    float rho;               /* stop coarsening when a level keeps more than rho of the nodes */
    uint64_t seed;           /* key of every Philox4x32-10 stream */
    uint32_t gid;            /* graph id folded into the random streams */
    int32_t mode;            /* 0 synchronous, 1 asynchronous (Hogwild) */
    int32_t precision;       /* 0 FP32; 1 FP16 and 2 BF16 copies for negative-sample gathers */
    uint32_t substeps;       /* synchronous sub-steps per epoch (>= 1) */
    uint32_t stop_nodes;     /* coarsen while a level has at least this many nodes */
    uint32_t match_rounds;   /* handshake rounds of heavy-edge matching */
    uint32_t max_levels;     /* at most this many levels, 1..64 */
    int32_t multilevel;      /* 0: lay out G^0 only */
    int32_t coarsen;         /* DRG_COARSEN_HEM or DRG_COARSEN_STAR (Sec. 3.2.3) */
    int32_t level_tables;    /* whole-path runs: 0 every level samples G^0's tables through the
                                ancestor map (Sec. 3.2.3, the paper's scheme); 1 each coarse level
                                samples its own distance matrix and tables, built just before the
                                level runs and freed after it (the conventional scheme) */
    float perplexity;        /* whole-path runs: > 0 sets sigma_i of Eq. 9 per node by this
                                perplexity (drg_build_distance_matrix_ex); 0 uses sigma */
    uint32_t row_cap;        /* whole-path runs: > 0 caps every row of the distance matrix to its
                                row_cap nearest nodes (drg_build_distance_matrix_capped); 0: none */
} drg_params;

/* Mode and precision values. */
#define DRG_MODE_SYNC 0
#define DRG_MODE_HOGWILD 1
#define DRG_PREC_FP32 0
#define DRG_PREC_FP16 1
#define DRG_PREC_BF16 2

/* Coarsening rules.  HEM: heavy-edge matching, handshake rounds (pairs of
 * nodes).  STAR: the paper's grouping (Sec. 3.2.3, Fig. 3): nodes taken in a
 * random order (Philox word 0 of counter (v, 0, tag), ties by id); each node
 * not yet grouped when taken forms a coarse node with its ungrouped
 * neighbours. */
#define DRG_COARSEN_HEM 0
#define DRG_COARSEN_STAR 1

void drg_params_default(drg_params* p);
const char* drg_status_string(drg_status s);

/* ---------------------------------------------------------------- context */
/* Create a context on `device`.  `stream` is a cudaStream_t to order all
 * work on (for example a torch stream), or NULL to create a private one. */
drg_status drg_create(drg_ctx** out, int device, void* stream);
drg_status drg_destroy(drg_ctx* ctx);
drg_status drg_synchronize(drg_ctx* ctx);
/* Last error message of the context (empty string when none). */
const char* drg_last_error(const drg_ctx* ctx);
/* Number of kernels this library has launched on the context so far. */
uint64_t drg_kernel_launches(const drg_ctx* ctx);

/* ---------------------------------------------------------------- graphs */
/* Sec. 3.1: G = (V, E) undirected and unweighted.  Builds the canonical CSR:
 * self-loops dropped, every edge stored in both directions, duplicates
 * removed, each row sorted by column.  src/dst hold m endpoint pairs (ids
 * < n) in host memory (on_device = 0) or device memory (on_device = 1); they
 * are read, not kept.  Ids >= n return DRG_EINVAL.  Synchronises. */
drg_status drg_graph_from_edges(drg_ctx* ctx, uint32_t n, uint64_t m, const uint32_t* src,
                                const uint32_t* dst, int on_device, drg_graph** out);
/* n nodes and nnz stored directed entries (2 |E|). */
drg_status drg_graph_info(const drg_graph* g, uint32_t* n, uint64_t* nnz);
/* Copy the CSR to host buffers: rp[n + 1], col[nnz], w[nnz] (edge weights,
 * all 1 on an input graph).  Any pointer may be NULL.  Synchronises. */
drg_status drg_graph_download(drg_ctx* ctx, const drg_graph* g, uint64_t* rp, uint32_t* col, uint32_t* w);
drg_status drg_graph_destroy(drg_graph* g);

/* ---------------------------------------------------------------- distance matrix */
/* Sec. 3.2.1 (Eqs. 8-9) and Sec. 3.2.2: the sparse distance matrix GD of G,
 * entry (i, j) = SPD(v_i, v_j) for every j in NNG(v_i, k), rows sorted by j;
 * the similarity weights and the two sampling tables drawn from in every
 * epoch:
 *   q[e]  = floor((fl(g(d)/Z_i) + fl(g(d)/Z_j)) * 2^30)  (FP32, correctly
 *           rounded, g(d) = exp(-d^2 / 2 sigma^2) rounded once to FP32,
 *           Z_i = sum over d = 1..k of count_i(d) * g(d) in that order) --
 *           proportional to NS_ij (Eq. 4) up to quantisation;
 *   r[i]  = sum of q over row i (u64); the node table uses r >> shift with
 *           the smallest shift that makes every value fit 32 bits;
 *   edge table: Walker alias table over the entries, weights q (the
 *           positive-sample distribution NS_ij); node table: alias table over
 *           the nodes, weights r >> shift (the negative-sample distribution,
 *           proportional to sum_l NS_il).  Both are built by the exact
 *           integer "sweep" construction (Huebschle-Schneider and Sanders,
 *           2019), so they are bit-identical to a sequential build.
 * k must be 1..15.  A graph without edges returns DRG_EEMPTY.  Synchronises. */
drg_status drg_build_distance_matrix(drg_ctx* ctx, const drg_graph* g, uint32_t k, float sigma,
                                     drg_dmat** out);
drg_status drg_dmat_info(const drg_dmat* d, uint32_t* n, uint64_t* nnz, uint32_t* node_shift);
/* Copy to host buffers (any may be NULL): rp[n+1], col[nnz], dist[nnz],
 * q[nnz], r[n], Z[n]; edge table e_thresh[nnz], e_alias[nnz] (entry ids);
 * node table v_thresh[n], v_alias[n].  The sampling path keeps no alias entry
 * ids (a record holds the alias's endpoints): e_alias is rebuilt for this
 * call by searching row i1 of the alias's endpoints (i1, j1) for j1, in a
 * temporary device buffer of 4 nnz bytes.  Synchronises. */
drg_status drg_dmat_download(drg_ctx* ctx, const drg_dmat* d, uint64_t* rp, uint32_t* col, uint8_t* dist,
                             uint32_t* q, uint64_t* r, float* Z, uint32_t* e_thresh, uint32_t* e_alias,
                             uint32_t* v_thresh, uint32_t* v_alias);
/* Host copies of the entries [e_begin, e_end) only (any pointer may be NULL):
 * col, dist, q, and the edge table's thresh and alias entry of those
 * buckets (rebuilt as for drg_dmat_download, 4 (e_end - e_begin) bytes of
 * temporary device memory).  e_end <= nnz.  Synchronises. */
drg_status drg_dmat_download_range(drg_ctx* ctx, const drg_dmat* d, uint64_t e_begin, uint64_t e_end, uint32_t* col,
                                   uint8_t* dist, uint32_t* q, uint32_t* e_thresh, uint32_t* e_alias);
/* drg_build_distance_matrix with Eq. 9's sigma_i set per node by perplexity
 * (perplexity > 0; sigma is then unused; 0 is the global-sigma build).  Row i
 * holds c_d nodes at hop distance d; beta_i = 1/(2 sigma_i^2) makes the
 * perplexity exp(H_i) = Z' exp(beta S'/Z') of NS_{.|i} equal `perplexity`,
 * with w_d = e^{-beta (d^2 - 1)}, Z' = sum_d c_d w_d and
 * S' = sum_d c_d (d^2 - 1) w_d (the factor e^{-beta} cancels in NS_{j|i});
 * it falls from the row size at beta = 0 to c_1, so rows smaller than
 * `perplexity` come out uniform and rows with c_1 >= perplexity keep only
 * their first-order neighbours.  beta_i: 60 bisection steps on [0, 512]
 * (mid = (lo + hi)/2; lo = mid when exp(H(mid)) > perplexity, else hi = mid;
 * beta_i = (lo + hi)/2), every step in FP64 with separately rounded
 * operations and the exponential e^x = p(r) 2^m, x = m ln2 + r (Cody-Waite
 * reduction with ln 2 = 0.6931471803691238 + 1.9082149292705877e-10,
 * m = floor(x * 1.4426950408889634 + 0.5), p the degree-13 Taylor polynomial
 * by Horner's rule with coefficients 1/n! computed by repeated division;
 * e^x = 0 below -700).  Then g_i(d) = fl32(e^{-beta_i (d^2 - 1)}),
 * Z_i = sum over d of count_i(d) * g_i(d) (FP32, in order) and
 *   q[e] = floor((fl(g_i(d)/Z_i) + fl(g_j(d)/Z_j)) * 2^30);
 * everything else as drg_build_distance_matrix.  DRG_EINVAL for a negative
 * or non-finite perplexity or one of 4.2e9 or more.  Synchronises. */
drg_status drg_build_distance_matrix_ex(drg_ctx* ctx, const drg_graph* g, uint32_t k, float sigma, float perplexity,
                                        drg_dmat** out);
/* drg_build_distance_matrix with a per-row neighbour cap, for graphs whose
 * k-order rows do not fit in memory (Sec. 3.2.1 notes that large k becomes
 * infeasible).  Row i keeps K_i, its row_cap nearest nodes of NNG(v_i, k) by
 * (hop distance, tie order of the node id): all nodes of the levels whose
 * cumulative count stays below row_cap, then the first nodes of the next level
 * in tie order.  The tie order is a fixed bijection t of [0, 2^28), applied to
 * a 28-bit id v as x = v ^ 0x2545F49; x = x * 0x9E3779B mod 2^28;
 * x ^= x >> 14; x = x * 0x85EBCA7 mod 2^28; t = x ^ (x >> 13); it keeps the
 * choice among equally near nodes unrelated to how ids were assigned (several
 * graph generators give their hubs the smallest ids).  The matrix's
 * pattern is the union K u K^T (an entry (i, j) for j in K_i or i in K_j,
 * rows sorted by j, dist the hop distance); the similarity of Eq. 9 is taken
 * over each row's kept set, Z_i = sum over d = 1..k of count of K_i at
 * distance d times g(d) (FP32, in order), and Eq. 4 symmetrises it over the
 * union:
 *   q[e] = floor((a + b) * 2^30), a = fl(g(d)/Z_i) when j is in K_i, else 0,
 *                                 b = fl(g(d)/Z_j) when i is in K_j, else 0;
 * r, the node table and the edge table as drg_build_distance_matrix.  With
 * row_cap at least the longest row it is that matrix bit for bit.  The
 * traversal stops at the level that fills the cap, so k = 3 stays feasible
 * where the full rows are not.  DRG_EINVAL for row_cap = 0;
 * DRG_EUNSUPPORTED for graphs of more than 2^28 nodes, for row_cap above 2016
 * unless it is at least n - 1 (then no row is cut: the uncapped matrix), and
 * when the kept entries reach 2^31.  Synchronises. */
drg_status drg_build_distance_matrix_capped(drg_ctx* ctx, const drg_graph* g, uint32_t k, float sigma,
                                            uint32_t row_cap, drg_dmat** out);
/* Host copy of beta_i = 1/(2 sigma_i^2) of every node (n doubles; 0 for an
 * empty row) of a perplexity-calibrated matrix; DRG_EINVAL for a matrix
 * built with a global sigma.  Synchronises. */
drg_status drg_dmat_calibration(drg_ctx* ctx, const drg_dmat* d, double* beta);
drg_status drg_dmat_destroy(drg_dmat* d);

/* ---------------------------------------------------------------- hierarchy */
/* Sec. 3.2.3 "Coarsening": one coarser level under the rule p->coarsen picks.
 * DRG_COARSEN_HEM: heavy-edge matching, p->match_rounds deterministic
 * handshake rounds (each unmatched node proposes to its unmatched neighbour of
 * largest (edge weight, Philox hash of the pair and round, smaller id); mutual
 * proposals match), unmatched nodes stay single; representative
 * min(v, mate(v)).  DRG_COARSEN_STAR: the paper's grouping (Fig. 3): nodes
 * taken in the order (Philox word 0 of counter (v, 0, tag), v) with purpose
 * 3; a node not yet grouped when taken becomes a centre and takes its
 * ungrouped neighbours, so every other node joins its neighbour centre
 * earliest in the order; representative = the centre.  Coarse ids are
 * numbered in representative id order; coarse edge weights are sums of fine
 * edge weights.  `level` selects the random stream.  parent (device, n_fine
 * uint32) receives the coarse id of every fine node.  DRG_EINVAL for an
 * unknown rule.  Synchronises. */
drg_status drg_coarsen(drg_ctx* ctx, const drg_graph* fine, uint32_t level, const drg_params* p,
                       drg_graph** coarse, uint32_t* parent);
/* Repeated drg_coarsen from G^0 while the level has >= p->stop_nodes nodes,
 * up to p->max_levels levels; a candidate level keeping more than p->rho of
 * its parent's nodes is discarded and ends the hierarchy.  The hierarchy
 * keeps each level's graph, parent map and ancestor map (G^0 node -> level
 * node).  Level 0 is `g0` itself (not copied; it must outlive the handle).
 * Synchronises. */
drg_status drg_build_hierarchy(drg_ctx* ctx, const drg_graph* g0, const drg_params* p, drg_hier** out);
drg_status drg_hier_info(const drg_hier* h, uint32_t* levels, uint32_t* sizes /* [levels], may be NULL */);
/* Host copies of level `level`'s parent map (n_level entries, level < levels-1)
 * and ancestor map (n_0 entries, level >= 1).  Either may be NULL.
 * Synchronises. */
drg_status drg_hier_download(drg_ctx* ctx, const drg_hier* h, uint32_t level, uint32_t* parent, uint32_t* anc);
/* Borrow the graph of one level (owned by the hierarchy). */
drg_status drg_hier_graph(const drg_hier* h, uint32_t level, const drg_graph** g);
drg_status drg_hier_destroy(drg_hier* h);

/* ---------------------------------------------------------------- layout */
/* Sec. 3.2.3 "Layout of the coarsest graph": pos[2 n] (device) uniform in
 * [-p->init_scale, p->init_scale]^2 from the Philox stream of
 * (p->seed, p->gid, level). */
drg_status drg_init_positions(drg_ctx* ctx, uint32_t n, uint32_t level, const drg_params* p, float* pos);

/* Epochs [t_begin, t_end) of p->epochs at one level (Sec. 3.2.2, Eqs. 11-12;
 * Sec. 3.2.3 gradient forwarding).  Sample s of epoch t draws from the
 * Philox stream counter (s, t, tag(level, gid), call): the positive entry
 * (i, j) from d's edge table and p->M negatives from its node table; the
 * level's nodes are a = anc(i), c = anc(j), c_m = anc(j_m) (identity at
 * level 0 or when h is NULL).  d is G^0's matrix or, at a coarse level, one
 * built on that level's graph (drg_hier_graph), whose entries are the
 * level's nodes themselves (identity map: the conventional multilevel scheme
 * the paper sets its forwarding against); negatives with c_m == a or c_m == c are
 * skipped.  The sample moves a by lr (attraction + sum of repulsions), c by
 * -lr attraction and each c_m by -lr repulsion_m, with
 *   attraction = -2b d^{2b-2} (y_a - y_c) / (1 + d^{2b}),
 *   repulsion  = gamma 2b (y_a - y_m) / (d^2 (1 + d^{2b})),
 * each component clipped to [-clip, clip], zero at distance 0, and
 * lr = p->lr0 (1 - t / p->epochs).  Synchronous mode cuts each epoch into
 * p->substeps runs of ceil(n_l / substeps) consecutive samples whose forces
 * all read the positions at the start of the run.  Hogwild mode (Sec. 4.3)
 * applies each sample's updates at once with atomic adds and keeps at most
 * ceil(n_l / substeps) samples in flight at any moment (bounding the
 * concurrency keeps asynchronous SGD close to the sequential method): with
 * FP32 positions, T <= ceil(n_l / substeps) threads each take every T-th
 * sample of an epoch, one at a time, in one cooperative launch in which a
 * warp starts epoch t only when every warp has finished epoch t - 2 (epochs
 * stay in step as in Sec. 4.3's shared epoch loop); with half-precision
 * copies, the synchronous runs' structure.  With substeps >= n_level one
 * sample is in flight and the run is the sequential method.  pos (device,
 * float[2 n_level]) is read and updated in place.  `gamma` overrides
 * p->gamma (use p->gamma_coarsest on the coarsest level).  DRG_ETIMEOUT: a
 * wait for the other warps exceeded 2 s (the positions are then partly
 * updated). */
drg_status drg_layout_level(drg_ctx* ctx, const drg_dmat* d, const drg_hier* h, uint32_t level, float* pos,
                            const drg_params* p, float gamma, uint32_t t_begin, uint32_t t_end);

/* Allocation-free variant of drg_layout_level (the paper has no counterpart:
 * this serves callers, not the method).  Some callers cannot allocate device
 * memory while they run -- for instance a serving process whose device
 * memory is fully reserved up front by another framework's allocator, or
 * code that must not grow its footprint after start-up -- and every other
 * layout call allocates its gradient buffer and epoch state per call.  This
 * one keeps them in a file-scope device array that every GPU loading the
 * library holds until the process exits: room for the epoch state and one
 * gradient pair per node, so levels of at most 1,048,576 nodes (8 MiB);
 * larger levels return DRG_EUNSUPPORTED.  It runs synchronous FP32 mode only
 * (other modes or precisions: DRG_EUNSUPPORTED) with the same kernels, random
 * streams and results as drg_layout_level, launched one by one instead of as
 * a graph.  d may be G^0's matrix or, at a coarse level, one built on that
 * level's graph, as for drg_layout_level.  It calls no allocating routine:
 * the first call on a device looks up the array's device address (the only
 * set-up; make that first call before any stream capture) and keeps it with
 * the id of the CUDA context it was read in, so a later call in another
 * context (for instance after the primary context was reset) repeats that
 * look-up; every call clears the gradient part, which keeps the previous
 * call's contents.  All calls share the one array per device, so calls that
 * overlap on the GPU (other streams, other contexts on the same device) race
 * and corrupt each other: serialise them. */
drg_status drg_layout_level_noalloc(drg_ctx* ctx, const drg_dmat* d, const drg_hier* h, uint32_t level, float* pos,
                                    const drg_params* p, float gamma, uint32_t t_begin, uint32_t t_end);

/* Sec. 3.2.3 "Refinement": fine_pos[v] = coarse_pos[parent(v)] for every node
 * of level coarse_level - 1.  Device buffers. */
drg_status drg_interpolate(drg_ctx* ctx, const drg_hier* h, uint32_t coarse_level, const float* coarse_pos,
                           float* fine_pos);

/* The whole path on a graph: distance matrix, hierarchy (when p->multilevel),
 * random coarsest layout, then for each level coarse to fine all epochs and
 * the refinement.  With p->level_tables each coarse level first gets its own
 * distance matrix and tables (freed after the level).  pos: device
 * float[2 n].  Synchronises. */
drg_status drg_layout(drg_ctx* ctx, const drg_graph* g, const drg_params* p, float* pos);

/* drg_graph_from_edges + drg_layout in one call.  Edges and positions live in
 * host memory when the matching *_on_device flag is 0 (copies are made on the
 * context stream) or in device memory when it is 1.  Synchronises. */
drg_status drg_layout_edges(drg_ctx* ctx, uint32_t n, uint64_t m, const uint32_t* src, const uint32_t* dst,
                            int edges_on_device, const drg_params* p, float* pos, int pos_on_device);

/* Lay out `count` independent graphs as one job.  Graph g uses p with
 * gid = g and shape b[g] (b may be NULL: p->b for all), i.e. its own random
 * streams, distance matrix, tables and hierarchy; in synchronous mode its
 * result equals drg_layout of that graph alone with those parameters up to
 * the order of FP32 atomic additions.  Levels run in rounds aligned at every
 * graph's coarsest level; in FP32 Hogwild mode all epochs of a round are one
 * cooperative launch (threads of every active graph, warps kept within two
 * epochs of each other by the same gates as drg_layout_level); otherwise
 * sub-step run c of every active graph is one kernel launch and all epochs
 * of the round are one CUDA graph launch.  pos[g] are device float[2 n_g].
 * p->level_tables must be 0 (DRG_EUNSUPPORTED).  Synchronises. */
drg_status drg_layout_batch(drg_ctx* ctx, uint32_t count, const drg_graph* const* graphs, const drg_params* p,
                            const float* b, float* const* pos);

/* ---------------------------------------------------------------- quality metrics */
/* Sec. 4.1 Eq. 17, crosslessness of a drawing of g: *crosslessness =
 * 1 - sqrt(c / c_max) (1 when c_max = 0), *crossings = c, the number of
 * unordered pairs of edges (straight segments) that cross, c_max =
 * |E|(|E|-1)/2 - (1/2) sum_v deg(v)(deg(v)-1).  Crossings are decided
 * exactly: positions snap per axis to the grid 0..2^30-1 over the drawing's
 * bounding box, q = floor((x - min) / (max - min) * (2^30 - 1) + 0.5) in FP64
 * (0 when max = min; an affine map changes no crossing), and two edges
 * without a common endpoint cross when each strictly separates the other's
 * endpoints by 64-bit integer orientation tests (touching and collinear
 * pairs do not count).  All pairs are tested (|E|^2 / 2 tests at about
 * 4 x 10^11 tests/s: 19 s for 4 million edges), in launches of at most 2^37
 * tests each; graphs with more than 2^23 edges return DRG_EUNSUPPORTED.
 * pos: device float[2 n].  DRG_EINVAL for a non-finite coordinate.
 * Synchronises. */
drg_status drg_crossings(drg_ctx* ctx, const drg_graph* g, const float* pos, uint64_t* crossings,
                         double* crosslessness);
/* Sec. 4.1 Eq. 19, minimum angle: *min_angle = 1 - mean over nodes of
 * |theta(v) - theta_min(v)| / theta(v), theta(v) = 2 pi / deg(v), theta_min(v)
 * the smallest angle between two edges consecutive around v (directions
 * atan2 in FP64; the wrap-around gap included).  The mean runs over nodes
 * with at least one edge; a node of degree 1 deviates by 0.  Directions
 * closer than 2 pi / 2^32 may be ordered either way (their gap then counts as
 * 0).  pos: device float[2 n].  Synchronises. */
drg_status drg_min_angle(drg_ctx* ctx, const drg_graph* g, const float* pos, double* min_angle);

/* Self-check of the epoch gates of the Hogwild level runs (no counterpart in
 * the paper).  `blocks` one-warp thread blocks (1 .. number of SMs), launched
 * so that all are resident at once, run `rounds` (1 .. 100000) empty epochs;
 * epoch e starts when `arrivals` warps have finished epoch e - 1, each wait
 * limited to timeout_ms (1 .. 10000).  arrivals == blocks: DRG_OK.
 * arrivals > blocks: no gate can open, every wait runs out, the warps leave
 * and the call returns DRG_ETIMEOUT (the GPU stays usable).
 * DRG_EUNSUPPORTED when the blocks cannot be resident together. */
drg_status drg_check_epoch_barrier(drg_ctx* ctx, uint32_t blocks, uint32_t arrivals, uint32_t rounds,
                                   uint32_t timeout_ms);

/* ---------------------------------------------------------------- profiling */
/* Per-kernel timing with CUDA events recorded on the context stream around
 * every launch of the named kernel family (costs a few microseconds per
 * launch; off by default).  Counters accumulate until reset. */
#define DRG_PROF_EPOCH 0   /* the sampling / gradient kernels (level runs); units = samples */
#define DRG_PROF_APPLY 1   /* k_apply: synchronous sub-step apply; units = nodes */
#define DRG_PROF_DMAT 2    /* drg_build_distance_matrix as a whole; units = entries */
#define DRG_PROF_HIER 3    /* hierarchy construction as a whole; units = levels */
#define DRG_PROF_GRAPH 4   /* drg_graph_from_edges; units = input edges */
#define DRG_PROF_BFS 5     /* the k-order BFS traversal kernel(s) of the distance matrix */
#define DRG_PROF_SIM 6     /* similarity and quantised weights; units = entries */
#define DRG_PROF_ALIAS 7   /* both alias tables and the edge records; units = entries + nodes */
#define DRG_PROF_ALLOC 8   /* host time inside device allocation calls; launches = calls, units = bytes */
#define DRG_PROF_COUNT 9
drg_status drg_profile_enable(drg_ctx* ctx, int on);
drg_status drg_profile_reset(drg_ctx* ctx);
/* Total milliseconds, number of timed launches and units of one family.
 * Synchronises. */
drg_status drg_profile_read(drg_ctx* ctx, int which, double* ms, uint64_t* launches, uint64_t* units);

/* ---------------------------------------------------------------- launch-shape autotuner */
/* The Hogwild level runs (drg_layout_level, drg_layout, drg_layout_batch)
 * use T threads, at most the in-flight bound; their launch shape is tuned
 * (no counterpart in the paper): the first run of at least 50 epochs for
 * each (device, kernel, M, precision, ancestor map, size bucket = bit length
 * of the level's nodes, or of a batch's total threads) times every candidate
 * -- 64, 128 or 256 threads per block, T = the bound, half or a quarter of it (a
 * smaller T only tightens the bound; batches tune the block size only) --
 * for 3 epochs on scratch copies of its positions, and every later run with
 * that key uses the fastest.  The table is process-wide.  Results of a run
 * depend on the shape only as far as Hogwild runs depend on thread timing.
 * drg_autotune_enable(ctx, 0) keeps the default shape (128 threads per
 * block, T = the bound) for the context's runs; on by default. */
drg_status drg_autotune_enable(drg_ctx* ctx, int on);
/* The tuned entries: *count receives their number; the first `cap` are
 * written (any array may be NULL): keys[6 i ..] = {kernel (0 single graph,
 * 1 batch), M (5, or 0 for any other), precision, ancestor map (0 or 1),
 * size bucket, device}, choice[2 i ..] = {threads per block, divisor of the
 * bound}, ms_per_epoch[i] = the choice's time per epoch in the tuning run. */
drg_status drg_autotune_read(uint32_t cap, uint32_t* keys, uint32_t* choice, float* ms_per_epoch, uint32_t* count);
/* Forget every tuned entry (the next long runs tune again). */
drg_status drg_autotune_clear(void);

/* ---------------------------------------------------------------- memory probes */
/* Measured ceilings for the roofline of the level kernels (no counterpart in
 * the paper, whose implementation runs on CPUs).  A sample of Sec. 3.2.2 is a
 * handful of random accesses: one 16-byte edge record from a table far larger
 * than L2, node records and position gathers that stay in L2, and vector
 * atomic adds; a streaming copy does not bound such accesses.  Each probe
 * allocates a zeroed buffer of buffer_bytes (1 MiB .. 64 GiB; DRG_ENOMEM when
 * it does not fit the free device memory), launches blocks_per_sm (1 .. 8)
 * blocks of 256 threads on every SM, each thread keeping 8 independent
 * accesses in flight, and times the launch with CUDA events on the context
 * stream:
 *   DRG_PROBE_LOAD8    random 8-byte loads through L2 (ld.global.cg.v2.f32),
 *                      the position gathers
 *   DRG_PROBE_LOAD16   random 16-byte loads (ld.global.nc.L2::64B.v4.u32: a
 *                      64-byte L2 prefetch size, as the edge records are read),
 *                      the table records
 *   DRG_PROBE_RED8     random 8-byte vector atomic adds (red of a float2),
 *                      the position updates
 *   DRG_PROBE_LOAD16_EVICT_FIRST  as LOAD16 with an L2 evict-first policy
 *   DRG_PROBE_COPY     streaming copy of the buffer's first half to its second
 *                      half (16-byte vectors; `accesses` is ignored)
 *   DRG_PROBE_MIX_LOAD8_RED8  a layout sample's mix, interleaved one to one
 *                      to one: random read-only 8-byte loads (ld.global.nc)
 *                      from the buffer's first half (the tables), random
 *                      8-byte loads through L2 (as LOAD8) and 8-byte atomic
 *                      adds (as RED8) on its second half (the positions); a
 *                      sample makes 5 to 7 table reads, 7 position reads and 7
 *                      atomic adds; all count as accesses
 * Random places are uniform over the buffer (a 32-bit linear congruential
 * stream per thread, scaled to the element count).  `accesses` (1 .. 1e11) is
 * rounded up to whole iterations; *done receives the accesses made (COPY: the
 * 16-byte vectors copied, each read once and written once) and *ms the kernel
 * time.  Synchronises. */
#define DRG_PROBE_LOAD8 0
#define DRG_PROBE_LOAD16 1
#define DRG_PROBE_RED8 2
#define DRG_PROBE_LOAD16_EVICT_FIRST 3
#define DRG_PROBE_COPY 4
#define DRG_PROBE_MIX_LOAD8_RED8 5
drg_status drg_probe_memory(drg_ctx* ctx, int kind, uint64_t buffer_bytes, uint64_t accesses, uint32_t blocks_per_sm,
                            double* ms, uint64_t* done);

/* ---------------------------------------------------------------- caller-given samples (tests) */
/* One synchronous step of Eqs. 11-12 over S samples fixed by the caller
 * instead of drawn (no counterpart in the paper's API: it serves closed-form
 * tests of the gradient).  Sample s is the term with source src[s], positive
 * target dst[s] and negatives neg[s M .. s M + M) (level node ids < n; device
 * arrays); negatives equal to the source or target are skipped.  Every force
 * is computed from the positions at the start of the call with the level
 * kernels' arithmetic (attraction -2b d^{2b-2} (y_a - y_c)/(1 + d^{2b}),
 * repulsion gamma 2b (y_a - y_m)/(d^2 (1 + d^{2b})), each component clipped
 * to [-clip, clip], zero at distance 0), moving the source by attraction +
 * sum of repulsions, the target by -attraction and each negative by -its
 * repulsion; the sums per node are then applied, pos += lr G.  pos: device
 * float[2 n], updated in place.  DRG_EINVAL for an id >= n, M > 64, b or clip
 * not positive or gamma negative.  Synchronises. */
drg_status drg_layout_step_explicit(drg_ctx* ctx, uint32_t n, float* pos, uint32_t S, const uint32_t* src,
                                    const uint32_t* dst, const uint32_t* neg, uint32_t M, float gamma, float b,
                                    float lr, float clip);

/* ---------------------------------------------------------------- inspection */
/* The draws of samples [s_begin, s_end) of epoch t at `level`: out_i, out_j
 * (level-0 ids of the positive entry) and out_neg[M per sample], device
 * buffers.  Same streams as drg_layout_level. */
drg_status drg_sample_draws(drg_ctx* ctx, const drg_dmat* d, uint32_t level, uint32_t t, uint32_t s_begin,
                            uint32_t s_end, const drg_params* p, uint32_t* out_i, uint32_t* out_j,
                            uint32_t* out_neg);

#ifdef __cplusplus
}
#endif

#endif /* DRGRAPH_H */
