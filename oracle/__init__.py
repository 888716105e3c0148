"""CPU oracle of the DRGraph layout path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The
product library (``paper_2008_07799_gb300``) never imports it and shares no
code with it.

The arithmetic lives in ``drg_oracle.c`` (plain C, FP64 layout math, exact
integer graph and index work, its own Philox4x32-10); this module only
marshals numpy arrays and runs the multilevel loop of Sec. 3.2.3 step by step:
canonical graph -> sparse distance matrix (Sec. 3.2.1) -> similarity and
quantised sampling weights (one sigma, or sigma_i per node by perplexity) ->
alias tables (Sec. 3.2.2) -> hierarchy by heavy-edge matching or the paper's
star grouping (Sec. 3.2.3) -> coarsest random layout -> for each level, coarse
to fine: epochs of negative-sampling SGD (Eqs. 11-12) on G^0's tables through
the ancestor map or on the level's own tables, then refinement.  The quality
metrics of Sec. 4.1 (NP, stress, crosslessness, minimum angle) evaluate the
result.

Parity status: every stage is pinned by ``tests/test_oracle_*.py`` against
closed forms, brute force, library routines or invariants.  Whole-run layout
quality against the paper's printed numbers is "parity unpinned" (the paper
states neither its random generator, sigma nor learning rate); only a loose
sanity range on a 17x17 grid is checked.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
import subprocess
import sysconfig

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "drg_oracle.c")
_LIB = os.path.join(_HERE, "_drg_oracle.so")
_lib = None

U32P = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
U64P = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")
U8P = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
F32P = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
F64P = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fused multiply-add: -ffp-contract=off)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-fno-fast-math", "-Wall", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_SRC_OMP = os.path.join(_HERE, "drg_oracle_omp.c")
_LIB_OMP = os.path.join(_HERE, "_drg_oracle_omp.so")
_lib_omp = None


def build_omp(force: bool = False):
    """Compile the optional multi-threaded baseline (gcc -fopenmp); returns
    its path, or None when the toolchain has no OpenMP."""
    newest = max(os.path.getmtime(_SRC_OMP), os.path.getmtime(_SRC))
    if force or not os.path.exists(_LIB_OMP) or os.path.getmtime(_LIB_OMP) < newest:
        tmp = _LIB_OMP + f".tmp{os.getpid()}"
        r = subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                            "-fno-fast-math", "-Wall", "-o", tmp, _SRC_OMP, "-lm"], capture_output=True, text=True)
        if r.returncode != 0:
            return None
        os.replace(tmp, _LIB_OMP)
    return _LIB_OMP


def lib_omp():
    """The multi-threaded baseline library (raises when it cannot be built)."""
    global _lib_omp
    if _lib_omp is not None:
        return _lib_omp
    path = build_omp()
    if path is None:
        raise RuntimeError("the OpenMP baseline needs gcc with OpenMP")
    L = C.CDLL(path)
    L.orc_layout_level_omp.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32,
                                       C.c_uint64, U32P, U32P, U32P, U32P,
                                       C.c_uint32, U32P, U32P,
                                       C.c_uint32, C.c_void_p, F64P,
                                       C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32,
                                       C.c_double, C.c_double, C.c_double, C.c_double, C.c_int]
    L.orc_omp_max_threads.restype = C.c_int
    _lib_omp = L
    return L


def lib():
    global _lib
    if _lib is not None:
        return _lib
    L = C.CDLL(build())
    L.orc_philox4x32_10.argtypes = [U32P, U32P, U32P]
    L.orc_tag.argtypes = [C.c_uint32] * 3
    L.orc_tag.restype = C.c_uint32
    L.orc_korder_counts.argtypes = [C.c_uint32, U64P, U32P, C.c_uint32, U64P]
    L.orc_korder_fill.argtypes = [C.c_uint32, U64P, U32P, C.c_uint32, U64P, U32P, U8P]
    L.orc_similarity.argtypes = [C.c_uint32, U64P, U32P, U8P, C.c_uint32, C.c_float,
                                 F32P, F32P, U32P, U64P, F64P]
    L.orc_korder_row.argtypes = [C.c_uint32, U64P, U32P, C.c_uint32, C.c_uint32, C.c_void_p, C.c_void_p,
                                 C.c_void_p, C.c_void_p]
    L.orc_korder_row.restype = C.c_uint32
    L.orc_class_counts.argtypes = [C.c_uint32, U64P, U32P, C.c_uint32, C.c_uint32, U32P, U64P]
    L.orc_normaliser.argtypes = [C.c_uint32, U64P, F32P]
    L.orc_normaliser.restype = C.c_float
    L.orc_entry_weight.argtypes = [C.c_float, C.c_float, C.c_float]
    L.orc_entry_weight.restype = C.c_uint32
    L.orc_node_weights_u32.argtypes = [C.c_uint32, U64P, U32P]
    L.orc_node_weights_u32.restype = C.c_uint32
    L.orc_alias_build.argtypes = [C.c_uint64, U32P, U32P, U32P, U64P]
    L.orc_alias_draw.argtypes = [C.c_uint64, U32P, U32P, C.c_uint64, C.c_uint32]
    L.orc_alias_draw.restype = C.c_uint64
    L.orc_sample_draws.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32,
                                   C.c_uint64, U32P, U32P, U32P, U32P, C.c_uint32, U32P, U32P,
                                   C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), U32P]
    L.orc_pair_force.argtypes = [C.c_double, C.c_double, C.c_int, C.c_double, C.c_double, C.c_double,
                                 C.POINTER(C.c_double), C.POINTER(C.c_double)]
    L.orc_sample_objective.argtypes = [F64P, F64P, F64P, C.c_uint32, C.c_double, C.c_double]
    L.orc_sample_objective.restype = C.c_double
    L.orc_layout_level.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32,
                                   C.c_uint64, U32P, U32P, U32P, U32P,
                                   C.c_uint32, U32P, U32P,
                                   C.c_uint32, C.c_void_p, F64P,
                                   C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32,
                                   C.c_double, C.c_double, C.c_double, C.c_double, C.c_int, C.c_uint32]
    L.orc_init_positions.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_float, F64P]
    L.orc_interpolate.argtypes = [C.c_uint32, U32P, F64P, F64P]
    L.orc_hem_match.argtypes = [C.c_uint32, U64P, U32P, C.c_void_p, C.c_uint64, C.c_uint32, C.c_uint32,
                                C.c_uint32, U32P]
    L.orc_cluster_ids.argtypes = [C.c_uint32, U32P, U32P]
    L.orc_cluster_ids.restype = C.c_uint32
    L.orc_exp.argtypes = [C.c_double]
    L.orc_exp.restype = C.c_double
    L.orc_row_perplexity.argtypes = [C.c_uint32, U64P, C.c_double]
    L.orc_row_perplexity.restype = C.c_double
    L.orc_calibrate_row.argtypes = [C.c_uint32, U64P, C.c_double]
    L.orc_calibrate_row.restype = C.c_double
    L.orc_similarity_perplexity.argtypes = [C.c_uint32, U64P, U32P, U8P, C.c_uint32, C.c_float, F64P, F32P, U32P,
                                            U64P, C.c_void_p]
    L.orc_crossings.argtypes = [C.c_uint32, U64P, U32P, F64P, C.POINTER(C.c_uint64), C.POINTER(C.c_double)]
    L.orc_min_angle.argtypes = [C.c_uint32, U64P, U32P, F64P]
    L.orc_min_angle.restype = C.c_double
    L.orc_star_group.argtypes = [C.c_uint32, U64P, U32P, U32P, U32P]
    L.orc_star_priorities.argtypes = [C.c_uint32, C.c_uint64, C.c_uint32, C.c_uint32, U32P]
    L.orc_star_priorities.restype = None
    L.orc_star_cluster_ids.argtypes = [C.c_uint32, U32P, U32P]
    L.orc_star_cluster_ids.restype = C.c_uint32
    L.orc_contract.argtypes = [C.c_uint32, U64P, U32P, C.c_void_p, U32P, C.c_uint32, U64P, C.c_void_p, C.c_void_p]
    L.orc_contract.restype = C.c_int64
    L.orc_neighbourhood_preservation.argtypes = [C.c_uint32, U64P, U32P, F64P, C.c_uint32, C.c_uint32,
                                                 C.c_void_p, C.POINTER(C.c_uint32)]
    L.orc_neighbourhood_preservation.restype = C.c_double
    L.orc_stress.argtypes = [C.c_uint32, U64P, U32P, F64P, C.c_uint32, C.c_void_p]
    L.orc_stress.restype = C.c_double
    _lib = L
    return L


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


# ---------------------------------------------------------------- parameters
@dataclasses.dataclass
class Params:
    """Layout parameters (Sec. 4 "Parameters"; Sec. 4.2; supplement on b)."""
    k: int = 1                 # order of the sparse distance matrix (Sec. 3.2.1)
    M: int = 5                 # negative samples per positive sample (Sec. 3.2.2)
    epochs: int = 400          # epochs per level
    gamma: float = 0.1         # negative-sample weight (Eq. 10)
    gamma_coarsest: float = 0.01   # early exaggeration on the coarsest level (Sec. 4.2)
    b: float = 1.0             # shape of the layout proximity kernel (Eq. 5)
    lr0: float = 1.0           # learning rate at epoch 0, linearly decayed to 0
    sigma: float = 1.0         # Gaussian width of the node similarity (Eq. 9)
    perplexity: float = 0.0    # > 0: sigma_i per node calibrated to this perplexity (sigma unused)
    clip: float = 5.0          # per-component clip of each pair force
    seed: int = 0
    gid: int = 0               # graph id in the random stream
    mode: int = 0              # 0 synchronous, 1 sequential (asynchronous reference)
    substeps: int = 16         # synchronous sub-steps per epoch
    stop_nodes: int = 1000     # coarsen while the level has at least this many nodes
    rho: float = 0.8           # stop when a coarser level keeps more than rho of the nodes
    match_rounds: int = 8      # handshake rounds of heavy-edge matching
    coarsen: int = 0           # 0 heavy-edge matching, 1 the paper's star grouping (Sec. 3.2.3)
    level_tables: int = 0      # 0 G^0's tables, samples forwarded to level l (Sec. 3.2.3);
                               # 1 each level its own distance matrix and tables (the conventional scheme)
    max_levels: int = 32
    init_scale: float = 1e-4   # coarsest positions uniform in [-s, s]^2
    multilevel: bool = True
    row_cap: int = 0           # > 0: each row keeps its row_cap nearest nodes, pattern K u K^T (korder_capped)


# ---------------------------------------------------------------- primitives
def philox(ctr, key):
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(np.asarray(ctr, np.uint32), np.asarray(key, np.uint32), out)
    return out


def canonical_graph(n, src, dst):
    """Sec. 3.1: undirected unweighted G = (V, E) -- drop self-loops, make
    every edge symmetric, remove duplicates; CSR rows sorted by column."""
    src = np.asarray(src, np.int64)
    dst = np.asarray(dst, np.int64)
    keep = src != dst
    a = np.r_[src[keep], dst[keep]]
    b = np.r_[dst[keep], src[keep]]
    key = np.unique(a * np.int64(n) + b)
    rows = key // n
    cols = key % n
    rp = np.zeros(n + 1, np.uint64)
    np.cumsum(np.bincount(rows, minlength=n), out=rp[1:])
    return rp, cols.astype(np.uint32)


def korder(rp, col, k):
    n = len(rp) - 1
    counts = np.zeros(max(n, 1), np.uint64)
    L = lib()
    assert L.orc_korder_counts(n, rp, col, k, counts) == 0
    gd_rp = np.zeros(n + 1, np.uint64)
    np.cumsum(counts[:n], out=gd_rp[1:])
    nnz = int(gd_rp[-1])
    gd_col = np.zeros(max(nnz, 1), np.uint32)
    gd_dist = np.zeros(max(nnz, 1), np.uint8)
    assert L.orc_korder_fill(n, rp, col, k, gd_rp, gd_col, gd_dist) == 0
    return gd_rp, gd_col[:nnz], gd_dist[:nnz]


TIE_BITS = 28
_TIE_MASK = (1 << TIE_BITS) - 1


def tie_order(v):
    """The order that breaks hop-distance ties in a capped row: a fixed
    bijection of [0, 2^28) (xor with a constant, multiplication by an odd
    constant mod 2^28, xor-shift, again, again), so that which nodes of a cut
    level are kept does not follow how the graph's ids were assigned (R-MAT
    and preferential-attachment generators give their hubs the smallest
    ids)."""
    x = (np.asarray(v, np.int64) ^ 0x2545F49) & _TIE_MASK
    x = (x * 0x9E3779B) & _TIE_MASK
    x ^= x >> 14
    x = (x * 0x85EBCA7) & _TIE_MASK
    x ^= x >> 13
    return x


def korder_capped(rp, col, k, cap):
    """Sec. 3.2.1 with a per-row neighbour cap (a reading for graphs whose
    k-order rows are too large): row i keeps K_i, its `cap` nearest entries by
    (hop distance, tie_order(node id)); the sampling pattern is the union of
    the kept entries and their transposes, rows sorted by column.  Returns the
    union CSR (rp, col, dist) and per entry (i, j) the flags own (j in K_i)
    and back (i in K_j).  Index work only; small graphs (the full rows are
    built first); node ids below 2^28."""
    n = len(rp) - 1
    if n > (1 << TIE_BITS):
        raise ValueError("capped rows need node ids below 2^28")
    g_rp, g_col, g_dist = korder(rp, col, k)
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(g_rp).astype(np.int64))
    c64 = g_col.astype(np.int64)
    # rank of every entry within its row by (distance, tie order of the column)
    order = np.lexsort((tie_order(c64), g_dist.astype(np.int64), rows))
    start = g_rp[:-1].astype(np.int64)
    rank = np.empty(len(order), np.int64)
    rank[order] = np.arange(len(order)) - start[rows[order]]
    kept = rank < cap
    fwd = rows[kept] * n + c64[kept]
    bwd = c64[kept] * n + rows[kept]
    keys = np.union1d(fwd, bwd)
    u_rows, u_col = keys // n, keys % n
    own = np.isin(keys, fwd)
    back = np.isin(keys, bwd)
    dist_of = dict(zip((rows * n + c64).tolist(), g_dist.tolist()))
    u_dist = np.array([dist_of[int(x)] for x in keys], np.uint8)
    u_rp = np.zeros(n + 1, np.uint64)
    np.cumsum(np.bincount(u_rows, minlength=n), out=u_rp[1:])
    return u_rp, u_col.astype(np.uint32), u_dist, own, back


def similarity_capped(u_rp, u_col, u_dist, own, back, k, sigma=1.0):
    """Eq. 9 over each row's kept set K_i and Eq. 4 over the union pattern:
    NS_{j|i} = g(d)/Z_i for j in K_i (else 0), Z_i = FP32 sum over d = 1..k of
    fl32(count of K_i at distance d) * g(d); q_e = floor((a + b) 2^30) in FP32
    with a = fl32(g/Z_i) when j in K_i else 0 and b = fl32(g/Z_j) when i in
    K_j else 0; r_i = row sums of q; ns the FP64 NS_ij."""
    n = len(u_rp) - 1
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(u_rp).astype(np.int64))
    d = u_dist.astype(np.int64)
    s32 = np.float64(np.float32(sigma))
    g64 = np.exp(-np.arange(1, k + 1, dtype=np.float64) ** 2 / (2.0 * s32 * s32))
    g32 = g64.astype(np.float32)
    Z = np.zeros(n, np.float32)
    Z64 = np.zeros(n, np.float64)
    for i in range(n):
        dd = d[int(u_rp[i]):int(u_rp[i + 1])][own[int(u_rp[i]):int(u_rp[i + 1])]]
        z = np.float32(0.0)
        for c in range(1, k + 1):
            cnt = np.float32(np.count_nonzero(dd == c))
            z = np.float32(z + np.float32(cnt * g32[c - 1]))
            Z64[i] += float(np.count_nonzero(dd == c)) * g64[c - 1]
        Z[i] = z
    j = u_col.astype(np.int64)
    gd = g32[d - 1]
    with np.errstate(divide="ignore", invalid="ignore"):
        a = np.where(own, gd / Z[rows], np.float32(0.0)).astype(np.float32)
        b = np.where(back, gd / Z[j], np.float32(0.0)).astype(np.float32)
    q = ((a + b).astype(np.float32) * np.float32(2.0 ** 30)).astype(np.float32).astype(np.uint32)
    r = np.bincount(rows, weights=q, minlength=n).astype(np.uint64)
    ns = (np.where(own, g64[d - 1] / np.where(Z64[rows] > 0, Z64[rows], 1.0), 0.0)
          + np.where(back, g64[d - 1] / np.where(Z64[j] > 0, Z64[j], 1.0), 0.0)) / (2.0 * n)
    return dict(Z=Z, q=q, r=r, ns=ns, g=g32)


class RowBFS:
    """Single rows of GD (spot checks of graphs too large for the full matrix)."""

    def __init__(self, rp, col, k):
        self.rp, self.col, self.k = rp, col, k
        n = len(rp) - 1
        self.dist = np.full(max(n, 1), -1, np.int32)
        self.queue = np.zeros(max(n, 1), np.uint32)
        self.out_col = np.zeros(max(n, 1), np.uint32)
        self.out_dist = np.zeros(max(n, 1), np.uint8)

    def row(self, src):
        L = lib()
        cnt = L.orc_korder_row(len(self.rp) - 1, self.rp, self.col, self.k, int(src),
                               self.dist.ctypes.data_as(C.c_void_p), self.queue.ctypes.data_as(C.c_void_p),
                               self.out_col.ctypes.data_as(C.c_void_p), self.out_dist.ctypes.data_as(C.c_void_p))
        return self.out_col[:cnt].copy(), self.out_dist[:cnt].copy()


def class_counts(rp, col, k, sources):
    """counts[x, d-1] = number of nodes at hop distance d from sources[x]."""
    sel = np.ascontiguousarray(sources, np.uint32)
    out = np.zeros((max(len(sel), 1), k), np.uint64)
    assert lib().orc_class_counts(len(rp) - 1, rp, col, k, len(sel), sel if len(sel) else np.zeros(1, np.uint32),
                                  out.reshape(-1)) == 0
    return out[:len(sel)]


def gaussians(k, sigma=1.0):
    """g(d) for d = 1..k as FP32 (FP64 exp of the FP32 sigma, rounded once)."""
    s = float(np.float32(sigma))
    return np.array([np.exp(-(d * d) / (2.0 * s * s)) for d in range(1, k + 1)]).astype(np.float32)


def normaliser(counts_row, g):
    c = np.ascontiguousarray(counts_row, np.uint64)
    return float(lib().orc_normaliser(len(g), c, np.ascontiguousarray(g, np.float32)))


def entry_weight(gd, zi, zj):
    return int(lib().orc_entry_weight(float(gd), float(zi), float(zj)))


def similarity(gd_rp, gd_col, gd_dist, k, sigma=1.0):
    n = len(gd_rp) - 1
    nnz = int(gd_rp[-1])
    g = np.zeros(k, np.float32)
    Z = np.zeros(max(n, 1), np.float32)
    q = np.zeros(max(nnz, 1), np.uint32)
    r = np.zeros(max(n, 1), np.uint64)
    ns = np.zeros(max(nnz, 1), np.float64)
    col = gd_col if nnz else np.zeros(1, np.uint32)
    dist = gd_dist if nnz else np.zeros(1, np.uint8)
    assert lib().orc_similarity(n, gd_rp, col, dist, k, sigma, g, Z, q, r, ns) == 0
    return dict(g=g, Z=Z[:n], q=q[:nnz], r=r[:n], ns=ns[:nnz])


def similarity_perplexity(gd_rp, gd_col, gd_dist, k, perplexity):
    """Eq. 9 with sigma_i calibrated per node to perplexity P (t-SNE rule)."""
    n = len(gd_rp) - 1
    nnz = int(gd_rp[-1])
    beta = np.zeros(max(n, 1), np.float64)
    Z = np.zeros(max(n, 1), np.float32)
    q = np.zeros(max(nnz, 1), np.uint32)
    r = np.zeros(max(n, 1), np.uint64)
    ns = np.zeros(max(nnz, 1), np.float64)
    col = gd_col if nnz else np.zeros(1, np.uint32)
    dist = gd_dist if nnz else np.zeros(1, np.uint8)
    assert lib().orc_similarity_perplexity(n, gd_rp, col, dist, k, perplexity, beta, Z, q, r,
                                           ns.ctypes.data) == 0
    return dict(beta=beta[:n], Z=Z[:n], q=q[:nnz], r=r[:n], ns=ns[:nnz])


def exp(x):
    """The oracle's own FP64 exponential (used by the calibration)."""
    return lib().orc_exp(float(x))


def row_perplexity(counts, beta):
    c = np.ascontiguousarray(counts, np.uint64)
    return lib().orc_row_perplexity(len(c), c, float(beta))


def calibrate_row(counts, perplexity):
    c = np.ascontiguousarray(counts, np.uint64)
    return lib().orc_calibrate_row(len(c), c, float(perplexity))


def node_weights_u32(r):
    r = np.ascontiguousarray(r, np.uint64)
    out = np.zeros(max(len(r), 1), np.uint32)
    s = lib().orc_node_weights_u32(len(r), r if len(r) else np.zeros(1, np.uint64), out)
    return out[:len(r)], int(s)


def alias_build(q):
    q = np.ascontiguousarray(q, np.uint32)
    N = len(q)
    th = np.zeros(max(N, 1), np.uint32)
    al = np.zeros(max(N, 1), np.uint32)
    own = np.zeros(max(N, 1), np.uint64)
    rc = lib().orc_alias_build(N, q if N else np.zeros(1, np.uint32), th, al, own)
    if rc != 0:
        return None
    return th[:N], al[:N], own[:N]


def alias_draw(thresh, alias, R, U):
    return int(lib().orc_alias_draw(len(thresh), thresh, alias, int(R), int(U)))


def edge_endpoints(gd_rp, gd_col):
    """Entry e of the distance matrix -> (source row, column)."""
    n = len(gd_rp) - 1
    src = np.repeat(np.arange(n, dtype=np.uint32), np.diff(gd_rp).astype(np.int64))
    return src, np.ascontiguousarray(gd_col, np.uint32)


@dataclasses.dataclass
class Tables:
    """Level-0 sampling state: edge table over distance-matrix entries and
    node table over nodes (Sec. 3.2.2)."""
    n0: int
    e_src: np.ndarray
    e_dst: np.ndarray
    e_thresh: np.ndarray
    e_alias: np.ndarray
    v_thresh: np.ndarray
    v_alias: np.ndarray
    q: np.ndarray
    r32: np.ndarray
    shift: int


def sampling_tables(gd_rp, gd_col, gd_dist, k, sigma=1.0, perplexity=0.0):
    if perplexity > 0:
        sim = similarity_perplexity(gd_rp, gd_col, gd_dist, k, perplexity)
    else:
        sim = similarity(gd_rp, gd_col, gd_dist, k, sigma)
    e_src, e_dst = edge_endpoints(gd_rp, gd_col)
    et = alias_build(sim["q"])
    r32, shift = node_weights_u32(sim["r"])
    vt = alias_build(r32)
    if et is None or vt is None:
        raise ValueError("graph has no edges: nothing to sample")
    return Tables(len(gd_rp) - 1, e_src, e_dst, et[0], et[1], vt[0], vt[1], sim["q"], r32, shift), sim


def sample_draws(tab: Tables, seed, gid, level, t, s, M):
    i = C.c_uint32()
    j = C.c_uint32()
    neg = np.zeros(max(M, 1), np.uint32)
    lib().orc_sample_draws(seed, gid, level, t, s, M, len(tab.e_thresh), tab.e_src, tab.e_dst,
                           tab.e_thresh, tab.e_alias, tab.n0, tab.v_thresh, tab.v_alias,
                           C.byref(i), C.byref(j), neg)
    return i.value, j.value, neg[:M].copy()


def pair_force(dx, dy, repulsive, gamma, b, clip):
    fx = C.c_double()
    fy = C.c_double()
    lib().orc_pair_force(dx, dy, int(repulsive), gamma, b, clip, C.byref(fx), C.byref(fy))
    return fx.value, fy.value


def sample_objective(yi, yj, yneg, gamma, b):
    yneg = np.ascontiguousarray(yneg, np.float64).reshape(-1)
    return lib().orc_sample_objective(np.ascontiguousarray(yi, np.float64), np.ascontiguousarray(yj, np.float64),
                                      yneg if len(yneg) else np.zeros(2), len(yneg) // 2, gamma, b)


def layout_level(tab: Tables, Y, level, anc, p: Params, gamma, t_begin=0, t_end=None):
    """Run epochs [t_begin, t_end) of one level in place on Y (n_l x 2 FP64)."""
    Y = np.ascontiguousarray(Y, np.float64)
    t_end = p.epochs if t_end is None else t_end
    anc_arr = None if anc is None else np.ascontiguousarray(anc, np.uint32)
    rc = lib().orc_layout_level(p.seed, p.gid, level, len(tab.e_thresh), tab.e_src, tab.e_dst,
                                tab.e_thresh, tab.e_alias, tab.n0, tab.v_thresh, tab.v_alias,
                                Y.shape[0], _ptr(anc_arr), Y.reshape(-1),
                                p.epochs, t_begin, t_end, p.M, gamma, p.b, p.lr0, p.clip, p.mode, p.substeps)
    assert rc == 0
    return Y


def layout_level_omp(tab: Tables, Y, level, anc, p: Params, gamma, threads, t_begin=0, t_end=None):
    """Sec. 4.3's multi-threaded optimisation: the sequential loop with each
    epoch's samples shared over `threads` lock-free threads (a CPU
    performance baseline; one thread is the sequential loop exactly)."""
    Y = np.ascontiguousarray(Y, np.float64)
    t_end = p.epochs if t_end is None else t_end
    anc_arr = None if anc is None else np.ascontiguousarray(anc, np.uint32)
    rc = lib_omp().orc_layout_level_omp(p.seed, p.gid, level, len(tab.e_thresh), tab.e_src, tab.e_dst,
                                        tab.e_thresh, tab.e_alias, tab.n0, tab.v_thresh, tab.v_alias,
                                        Y.shape[0], _ptr(anc_arr), Y.reshape(-1),
                                        p.epochs, t_begin, t_end, p.M, gamma, p.b, p.lr0, p.clip, int(threads))
    assert rc == 0
    return Y


def init_positions(p: Params, level, n):
    Y = np.zeros((n, 2), np.float64)
    lib().orc_init_positions(p.seed, p.gid, level, n, p.init_scale, Y.reshape(-1))
    return Y


def interpolate(parent, Yc):
    parent = np.ascontiguousarray(parent, np.uint32)
    Yf = np.zeros((len(parent), 2), np.float64)
    lib().orc_interpolate(len(parent), parent, np.ascontiguousarray(Yc, np.float64).reshape(-1), Yf.reshape(-1))
    return Yf


# ---------------------------------------------------------------- hierarchy
def hem_match(rp, col, w, p: Params, level):
    n = len(rp) - 1
    match = np.zeros(max(n, 1), np.uint32)
    w_arr = None if w is None else np.ascontiguousarray(w, np.uint32)
    assert lib().orc_hem_match(n, rp, col if len(col) else np.zeros(1, np.uint32), _ptr(w_arr),
                               p.seed, p.gid, level, p.match_rounds, match) == 0
    return match[:n]


def cluster_ids(match):
    cid = np.zeros(max(len(match), 1), np.uint32)
    nc = lib().orc_cluster_ids(len(match), np.ascontiguousarray(match, np.uint32), cid)
    return cid[:len(match)], int(nc)


def star_priorities(n, p: Params, level):
    """The random order of the star grouping at `level` (Philox purpose 3)."""
    prio = np.zeros(max(n, 1), np.uint32)
    lib().orc_star_priorities(n, p.seed, p.gid, level, prio)
    return prio[:n]


def star_group(rp, col, prio):
    """Sec. 3.2.3 grouping walked in the order (prio[v], v): centre[v] is the
    picked node whose group v joined."""
    n = len(rp) - 1
    centre = np.zeros(max(n, 1), np.uint32)
    assert lib().orc_star_group(n, np.ascontiguousarray(rp, np.uint64),
                                col if len(col) else np.zeros(1, np.uint32),
                                np.ascontiguousarray(prio, np.uint32) if n else np.zeros(1, np.uint32),
                                centre) == 0
    return centre[:n]


def star_cluster_ids(centre):
    cid = np.zeros(max(len(centre), 1), np.uint32)
    nc = lib().orc_star_cluster_ids(len(centre), np.ascontiguousarray(centre, np.uint32), cid)
    return cid[:len(centre)], int(nc)


def cluster(rp, col, w, p: Params, level):
    """Coarse node id of every node of a level, and their number, under the
    rule p.coarsen selects."""
    if p.coarsen == 1:
        return star_cluster_ids(star_group(rp, col, star_priorities(len(rp) - 1, p, level)))
    return cluster_ids(hem_match(rp, col, w, p, level))


def contract(rp, col, w, cid, nc):
    n = len(rp) - 1
    L = lib()
    colx = col if len(col) else np.zeros(1, np.uint32)
    w_arr = None if w is None else np.ascontiguousarray(w, np.uint32)
    out_rp = np.zeros(nc + 1, np.uint64)
    m = L.orc_contract(n, rp, colx, _ptr(w_arr), np.ascontiguousarray(cid, np.uint32), nc, out_rp, None, None)
    assert m >= 0
    out_col = np.zeros(max(m, 1), np.uint32)
    out_w = np.zeros(max(m, 1), np.uint32)
    L.orc_contract(n, rp, colx, _ptr(w_arr), np.ascontiguousarray(cid, np.uint32), nc, out_rp,
                   _ptr(out_col), _ptr(out_w))
    return out_rp, out_col[:m], out_w[:m]


@dataclasses.dataclass
class Level:
    rp: np.ndarray
    col: np.ndarray
    w: np.ndarray | None
    parent: np.ndarray | None = None   # this level -> next coarser level
    anc: np.ndarray | None = None      # level-0 node -> this level (None at level 0)

    @property
    def n(self):
        return len(self.rp) - 1


def hierarchy(rp, col, p: Params):
    """Sec. 3.2.3 coarsening: repeat while the level has >= stop_nodes nodes;
    stop (discarding the candidate) when it keeps more than rho of the nodes."""
    levels = [Level(rp, col, None)]
    while p.multilevel and len(levels) < p.max_levels and levels[-1].n >= p.stop_nodes:
        cur = levels[-1]
        lvl = len(levels) - 1
        cid, nc = cluster(cur.rp, cur.col, cur.w, p, lvl)
        if nc > p.rho * cur.n:
            break
        crp, ccol, cw = contract(cur.rp, cur.col, cur.w, cid, nc)
        cur.parent = cid
        anc = cid.copy() if cur.anc is None else cid[cur.anc]
        levels.append(Level(crp, ccol, cw, None, anc))
    return levels


def level_tables(level: Level, p: Params):
    """The conventional multilevel scheme the paper sets its own against
    (Sec. 3.2.3, last paragraph): level l's own sparse distance matrix (hop
    distances in G^l; the coarse edge weights play no part) and sampling
    tables, so that level l is laid out like an input graph of its own."""
    gd = korder(level.rp, level.col, p.k)
    return sampling_tables(*gd, p.k, p.sigma, p.perplexity)[0]


def sampling_tables_capped(rp, col, k, cap, sigma=1.0):
    """Sampling tables of the capped matrix (korder_capped, similarity_capped):
    the edge table over the union pattern's entries, the node table over the
    row sums of its weights."""
    u_rp, u_col, u_dist, own, back = korder_capped(rp, col, k, cap)
    sim = similarity_capped(u_rp, u_col, u_dist, own, back, k, sigma)
    e_src, e_dst = edge_endpoints(u_rp, u_col)
    et = alias_build(sim["q"])
    r32, shift = node_weights_u32(sim["r"])
    vt = alias_build(r32)
    if et is None or vt is None:
        raise ValueError("graph has no edges: nothing to sample")
    return Tables(len(u_rp) - 1, e_src, e_dst, et[0], et[1], vt[0], vt[1], sim["q"], r32, shift), \
        (u_rp, u_col, u_dist), sim


def run(n, src, dst, p: Params, return_state=False):
    """The whole layout path, coarse to fine (Sec. 3.2, Fig. 1 pipeline).
    With p.level_tables = 1 every coarse level samples its own tables
    (level_tables) instead of G^0's through the ancestor map; with
    p.row_cap > 0 the distance matrix's rows are capped (korder_capped)."""
    rp, col = canonical_graph(n, src, dst)
    if p.row_cap:
        assert not p.level_tables and p.perplexity == 0.0, "the row cap is for G^0's global-sigma tables"
        tab, (gd_rp, gd_col, gd_dist), sim = sampling_tables_capped(rp, col, p.k, p.row_cap, p.sigma)
    else:
        gd_rp, gd_col, gd_dist = korder(rp, col, p.k)
        tab, sim = sampling_tables(gd_rp, gd_col, gd_dist, p.k, p.sigma, p.perplexity)
    levels = hierarchy(rp, col, p)
    L = len(levels) - 1
    Y = init_positions(p, L, levels[L].n)
    level_tabs = {}
    for lvl in range(L, -1, -1):
        gamma = p.gamma_coarsest if (lvl == L and L > 0) else p.gamma
        if p.level_tables and lvl > 0:
            level_tabs[lvl] = level_tables(levels[lvl], p)
            Y = layout_level(level_tabs[lvl], Y, lvl, None, p, gamma)
        else:
            Y = layout_level(tab, Y, lvl, levels[lvl].anc, p, gamma)
        if lvl > 0:
            Y = interpolate(levels[lvl - 1].parent, Y)
    if return_state:
        return Y, dict(rp=rp, col=col, gd=(gd_rp, gd_col, gd_dist), tab=tab, sim=sim, levels=levels,
                       level_tabs=level_tabs)
    return Y


# ---------------------------------------------------------------- metrics
def neighbourhood_preservation(rp, col, Y, k_eval=2, nodes=None):
    n = len(rp) - 1
    sel = None if nodes is None else np.ascontiguousarray(nodes, np.uint32)
    cnt = C.c_uint32()
    v = lib().orc_neighbourhood_preservation(n, rp, col if len(col) else np.zeros(1, np.uint32),
                                             np.ascontiguousarray(Y, np.float64).reshape(-1), k_eval,
                                             n if sel is None else len(sel), _ptr(sel), C.byref(cnt))
    return v


def crossings(rp, col, Y):
    """Sec. 4.1 Eq. 17: (number of edge crossings, crosslessness), crossings
    decided exactly on positions snapped per axis to a 30-bit grid."""
    n = len(rp) - 1
    c = C.c_uint64()
    cl = C.c_double()
    assert lib().orc_crossings(n, np.ascontiguousarray(rp, np.uint64), col if len(col) else np.zeros(1, np.uint32),
                               np.ascontiguousarray(Y, np.float64).reshape(-1), C.byref(c), C.byref(cl)) == 0
    return int(c.value), float(cl.value)


def min_angle(rp, col, Y):
    """Sec. 4.1 Eq. 19, over nodes with at least one edge."""
    n = len(rp) - 1
    return lib().orc_min_angle(n, np.ascontiguousarray(rp, np.uint64), col if len(col) else np.zeros(1, np.uint32),
                               np.ascontiguousarray(Y, np.float64).reshape(-1))


def stress(rp, col, Y, sources=None):
    n = len(rp) - 1
    sel = None if sources is None else np.ascontiguousarray(sources, np.uint32)
    return lib().orc_stress(n, rp, col if len(col) else np.zeros(1, np.uint32),
                            np.ascontiguousarray(Y, np.float64).reshape(-1),
                            n if sel is None else len(sel), _ptr(sel))
