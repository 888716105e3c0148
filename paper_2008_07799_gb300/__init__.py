"""GB300 DRGraph layout library: Python binding of ``libdrgraph.so``.

Every step of the layout path runs in the library's CUDA kernels; this module
only marshals arguments (numpy arrays for host buffers, torch CUDA tensors for
device buffers) and turns status codes into exceptions.  The names follow the
C ABI in ``include/drgraph.h``:

    graph_from_edges, build_distance_matrix, coarsen, build_hierarchy,
    init_positions, layout_level, interpolate, layout, layout_edges,
    layout_batch, sample_draws, crossings, min_angle

There is no CPU fallback: without the built library (``build()``) every call
raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libdrgraph.so")

MODE_SYNC, MODE_HOGWILD = 0, 1
PREC_FP32, PREC_FP16, PREC_BF16 = 0, 1, 2

STATUS = {0: "ok", 1: "invalid argument", 2: "out of memory", 3: "CUDA error", 4: "device wait timed out",
          5: "unsupported size", 6: "graph has no edges"}

#: every symbol include/drgraph.h declares
EXPORTS = [
    "drg_params_default", "drg_status_string", "drg_create", "drg_destroy", "drg_synchronize", "drg_last_error",
    "drg_kernel_launches", "drg_graph_from_edges", "drg_graph_info", "drg_graph_download", "drg_graph_destroy",
    "drg_build_distance_matrix", "drg_dmat_info", "drg_dmat_download", "drg_dmat_destroy", "drg_coarsen",
    "drg_build_hierarchy", "drg_hier_info", "drg_hier_download", "drg_hier_graph", "drg_hier_destroy",
    "drg_init_positions", "drg_layout_level", "drg_interpolate", "drg_layout", "drg_layout_edges",
    "drg_layout_batch", "drg_sample_draws", "drg_profile_enable", "drg_profile_reset", "drg_profile_read",
    "drg_layout_level_noalloc", "drg_dmat_download_range", "drg_check_epoch_barrier",
    "drg_build_distance_matrix_ex", "drg_dmat_calibration", "drg_crossings", "drg_min_angle",
    "drg_probe_memory", "drg_autotune_enable", "drg_autotune_read", "drg_autotune_clear",
    "drg_build_distance_matrix_capped", "drg_layout_step_explicit",
]

PROBE_LOAD8, PROBE_LOAD16, PROBE_RED8, PROBE_LOAD16_EVICT_FIRST, PROBE_COPY, PROBE_MIX_LOAD8_RED8 = range(6)

PROF_EPOCH, PROF_APPLY, PROF_DMAT, PROF_HIER, PROF_GRAPH, PROF_BFS, PROF_SIM, PROF_ALIAS, PROF_ALLOC = range(9)


class DrgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Params(C.Structure):
    """Mirror of ``drg_params``."""
    _fields_ = [
        ("k", C.c_uint32), ("M", C.c_uint32), ("epochs", C.c_uint32),
        ("gamma", C.c_float), ("gamma_coarsest", C.c_float), ("b", C.c_float), ("lr0", C.c_float),
        ("sigma", C.c_float), ("clip", C.c_float), ("init_scale", C.c_float), ("rho", C.c_float),
        ("seed", C.c_uint64), ("gid", C.c_uint32), ("mode", C.c_int32), ("precision", C.c_int32),
        ("substeps", C.c_uint32), ("stop_nodes", C.c_uint32), ("match_rounds", C.c_uint32),
        ("max_levels", C.c_uint32), ("multilevel", C.c_int32), ("coarsen", C.c_int32),
        ("level_tables", C.c_int32), ("perplexity", C.c_float), ("row_cap", C.c_uint32),
    ]

    @classmethod
    def default(cls, **kw):
        p = cls()
        lib().drg_params_default(C.byref(p))
        for key, v in kw.items():
            if not hasattr(p, key):
                raise KeyError(key)
            setattr(p, key, v)
        return p

    def replace(self, **kw):
        q = Params()
        C.pointer(q)[0] = self
        for key, v in kw.items():
            setattr(q, key, v)
        return q


_lib = None
VP = C.c_void_p


def lib():
    """Load libdrgraph.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: run paper_2008_07799_gb300.build.build() (needs nvcc)")
    L = C.CDLL(LIB_PATH)
    st = C.c_int
    PP = C.POINTER(Params)
    sig = {
        "drg_params_default": (None, [PP]),
        "drg_status_string": (C.c_char_p, [st]),
        "drg_create": (st, [C.POINTER(VP), C.c_int, VP]),
        "drg_destroy": (st, [VP]),
        "drg_synchronize": (st, [VP]),
        "drg_last_error": (C.c_char_p, [VP]),
        "drg_kernel_launches": (C.c_uint64, [VP]),
        "drg_graph_from_edges": (st, [VP, C.c_uint32, C.c_uint64, VP, VP, C.c_int, C.POINTER(VP)]),
        "drg_graph_info": (st, [VP, C.POINTER(C.c_uint32), C.POINTER(C.c_uint64)]),
        "drg_graph_download": (st, [VP, VP, VP, VP, VP]),
        "drg_graph_destroy": (st, [VP]),
        "drg_build_distance_matrix": (st, [VP, VP, C.c_uint32, C.c_float, C.POINTER(VP)]),
        "drg_dmat_info": (st, [VP, C.POINTER(C.c_uint32), C.POINTER(C.c_uint64), C.POINTER(C.c_uint32)]),
        "drg_dmat_download": (st, [VP] * 12),
        "drg_dmat_destroy": (st, [VP]),
        "drg_build_distance_matrix_ex": (st, [VP, VP, C.c_uint32, C.c_float, C.c_float, C.POINTER(VP)]),
        "drg_dmat_calibration": (st, [VP, VP, VP]),
        "drg_build_distance_matrix_capped": (st, [VP, VP, C.c_uint32, C.c_float, C.c_uint32, C.POINTER(VP)]),
        "drg_crossings": (st, [VP, VP, VP, C.POINTER(C.c_uint64), C.POINTER(C.c_double)]),
        "drg_min_angle": (st, [VP, VP, VP, C.POINTER(C.c_double)]),
        "drg_dmat_download_range": (st, [VP, VP, C.c_uint64, C.c_uint64, VP, VP, VP, VP, VP]),
        "drg_coarsen": (st, [VP, VP, C.c_uint32, PP, C.POINTER(VP), VP]),
        "drg_build_hierarchy": (st, [VP, VP, PP, C.POINTER(VP)]),
        "drg_hier_info": (st, [VP, C.POINTER(C.c_uint32), VP]),
        "drg_hier_download": (st, [VP, VP, C.c_uint32, VP, VP]),
        "drg_hier_graph": (st, [VP, C.c_uint32, C.POINTER(VP)]),
        "drg_hier_destroy": (st, [VP]),
        "drg_init_positions": (st, [VP, C.c_uint32, C.c_uint32, PP, VP]),
        "drg_layout_level": (st, [VP, VP, VP, C.c_uint32, VP, PP, C.c_float, C.c_uint32, C.c_uint32]),
        "drg_layout_level_noalloc": (st, [VP, VP, VP, C.c_uint32, VP, PP, C.c_float, C.c_uint32, C.c_uint32]),
        "drg_check_epoch_barrier": (st, [VP, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32]),
        "drg_interpolate": (st, [VP, VP, C.c_uint32, VP, VP]),
        "drg_layout": (st, [VP, VP, PP, VP]),
        "drg_layout_edges": (st, [VP, C.c_uint32, C.c_uint64, VP, VP, C.c_int, PP, VP, C.c_int]),
        "drg_layout_batch": (st, [VP, C.c_uint32, VP, PP, VP, VP]),
        "drg_sample_draws": (st, [VP, VP, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32, PP, VP, VP, VP]),
        "drg_probe_memory": (st, [VP, C.c_int, C.c_uint64, C.c_uint64, C.c_uint32, C.POINTER(C.c_double),
                                  C.POINTER(C.c_uint64)]),
        "drg_layout_step_explicit": (st, [VP, C.c_uint32, VP, C.c_uint32, VP, VP, VP, C.c_uint32, C.c_float,
                                          C.c_float, C.c_float, C.c_float]),
        "drg_autotune_enable": (st, [VP, C.c_int]),
        "drg_autotune_read": (st, [C.c_uint32, VP, VP, VP, C.POINTER(C.c_uint32)]),
        "drg_autotune_clear": (st, []),
        "drg_profile_enable": (st, [VP, C.c_int]),
        "drg_profile_reset": (st, [VP]),
        "drg_profile_read": (st, [VP, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_uint64),
                                  C.POINTER(C.c_uint64)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _ptr(x):
    """Device or host address of a torch tensor / numpy array (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return x.ctypes.data
    assert x.is_contiguous()
    return x.data_ptr()


def _is_device(x):
    return not isinstance(x, np.ndarray) and getattr(x, "is_cuda", False)


def _host_u32(x):
    """numpy arrays become contiguous uint32; torch host tensors (e.g. pinned)
    are passed through untouched."""
    if isinstance(x, np.ndarray) or not hasattr(x, "data_ptr"):
        return np.ascontiguousarray(x, np.uint32)
    assert x.element_size() == 4 and x.is_contiguous()
    return x


class Context:
    """A library context on one GPU; ``stream`` is a cudaStream_t handle
    (e.g. ``torch.cuda.current_stream().cuda_stream``) or None."""

    def __init__(self, device=0, stream=None):
        self.h = VP()
        st = lib().drg_create(C.byref(self.h), int(device), stream)
        if st:
            raise DrgError(st, "drg_create failed")

    def check(self, st):
        if st:
            raise DrgError(st, lib().drg_last_error(self.h).decode())

    def synchronize(self):
        self.check(lib().drg_synchronize(self.h))

    @property
    def launches(self):
        return int(lib().drg_kernel_launches(self.h))

    def profile(self, on=True):
        self.check(lib().drg_profile_enable(self.h, int(on)))

    def autotune(self, on=True):
        """Tune the Hogwild kernels' launch shape (on by default)."""
        self.check(lib().drg_autotune_enable(self.h, int(on)))

    def profile_reset(self):
        self.check(lib().drg_profile_reset(self.h))

    def profile_read(self, which):
        """(milliseconds, launches, units) accumulated for one kernel family."""
        ms = C.c_double()
        n = C.c_uint64()
        u = C.c_uint64()
        self.check(lib().drg_profile_read(self.h, int(which), C.byref(ms), C.byref(n), C.byref(u)))
        return ms.value, n.value, u.value

    def close(self):
        if self.h:
            lib().drg_destroy(self.h)
            self.h = VP()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _Handle:
    _destroy = None

    def __init__(self, ctx, h):
        self.ctx = ctx
        self.h = h

    def close(self):
        if self.h and self._destroy:
            getattr(lib(), self._destroy)(self.h)
            self.h = VP()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Graph(_Handle):
    _destroy = "drg_graph_destroy"

    def info(self):
        n = C.c_uint32()
        nnz = C.c_uint64()
        lib().drg_graph_info(self.h, C.byref(n), C.byref(nnz))
        return n.value, nnz.value

    @property
    def n(self):
        return self.info()[0]

    def download(self):
        n, nnz = self.info()
        rp = np.zeros(n + 1, np.uint64)
        col = np.zeros(max(nnz, 1), np.uint32)
        w = np.zeros(max(nnz, 1), np.uint32)
        self.ctx.check(lib().drg_graph_download(self.ctx.h, self.h, _ptr(rp), _ptr(col), _ptr(w)))
        return rp, col[:nnz], w[:nnz]


class DistanceMatrix(_Handle):
    _destroy = "drg_dmat_destroy"

    def calibration(self):
        """beta_i = 1/(2 sigma_i^2) of every node (perplexity-calibrated matrices)."""
        n = self.info()[0]
        out = np.zeros(max(n, 1), np.float64)
        self.ctx.check(lib().drg_dmat_calibration(self.ctx.h, self.h, _ptr(out)))
        return out[:n]

    def info(self):
        n = C.c_uint32()
        nnz = C.c_uint64()
        s = C.c_uint32()
        lib().drg_dmat_info(self.h, C.byref(n), C.byref(nnz), C.byref(s))
        return n.value, nnz.value, s.value

    def download(self):
        n, nnz, shift = self.info()
        m = max(nnz, 1)
        out = dict(rp=np.zeros(n + 1, np.uint64), col=np.zeros(m, np.uint32), dist=np.zeros(m, np.uint8),
                   q=np.zeros(m, np.uint32), r=np.zeros(n, np.uint64), Z=np.zeros(n, np.float32),
                   e_thresh=np.zeros(m, np.uint32), e_alias=np.zeros(m, np.uint32),
                   v_thresh=np.zeros(n, np.uint32), v_alias=np.zeros(n, np.uint32))
        o = out
        self.ctx.check(lib().drg_dmat_download(self.ctx.h, self.h, _ptr(o["rp"]), _ptr(o["col"]), _ptr(o["dist"]),
                                               _ptr(o["q"]), _ptr(o["r"]), _ptr(o["Z"]), _ptr(o["e_thresh"]),
                                               _ptr(o["e_alias"]), _ptr(o["v_thresh"]), _ptr(o["v_alias"])))
        for key in ("col", "dist", "q", "e_thresh", "e_alias"):
            out[key] = out[key][:nnz]
        out["shift"] = shift
        return out

    def download_nodes(self):
        """The per-node arrays only: rp, r, Z and the node table."""
        n, nnz, shift = self.info()
        out = dict(rp=np.zeros(n + 1, np.uint64), r=np.zeros(n, np.uint64), Z=np.zeros(n, np.float32),
                   v_thresh=np.zeros(n, np.uint32), v_alias=np.zeros(n, np.uint32), shift=shift, nnz=nnz)
        self.ctx.check(lib().drg_dmat_download(self.ctx.h, self.h, _ptr(out["rp"]), None, None, None, _ptr(out["r"]),
                                               _ptr(out["Z"]), None, None, _ptr(out["v_thresh"]),
                                               _ptr(out["v_alias"])))
        return out

    def download_range(self, e0, e1):
        """Entries [e0, e1): col, dist, q and the edge table's thresh and alias."""
        m = max(e1 - e0, 1)
        out = dict(col=np.zeros(m, np.uint32), dist=np.zeros(m, np.uint8), q=np.zeros(m, np.uint32),
                   e_thresh=np.zeros(m, np.uint32), e_alias=np.zeros(m, np.uint32))
        self.ctx.check(lib().drg_dmat_download_range(self.ctx.h, self.h, int(e0), int(e1), _ptr(out["col"]),
                                                     _ptr(out["dist"]), _ptr(out["q"]), _ptr(out["e_thresh"]),
                                                     _ptr(out["e_alias"])))
        return {k: v[:e1 - e0] for k, v in out.items()}


class Hierarchy(_Handle):
    _destroy = "drg_hier_destroy"

    def __init__(self, ctx, h, g0):
        super().__init__(ctx, h)
        self.g0 = g0  # level 0 is borrowed: keep it alive

    def sizes(self):
        L = C.c_uint32()
        lib().drg_hier_info(self.h, C.byref(L), None)
        arr = np.zeros(L.value, np.uint32)
        lib().drg_hier_info(self.h, C.byref(L), _ptr(arr))
        return [int(x) for x in arr]

    def parent(self, level):
        sizes = self.sizes()
        out = np.zeros(sizes[level], np.uint32)
        self.ctx.check(lib().drg_hier_download(self.ctx.h, self.h, level, _ptr(out), None))
        return out

    def anc(self, level):
        sizes = self.sizes()
        out = np.zeros(sizes[0], np.uint32)
        self.ctx.check(lib().drg_hier_download(self.ctx.h, self.h, level, None, _ptr(out)))
        return out

    def graph(self, level):
        g = VP()
        self.ctx.check(lib().drg_hier_graph(self.h, level, C.byref(g)))
        view = Graph(self.ctx, g)
        view._destroy = None  # owned by the hierarchy
        view._owner = self
        return view


# ---------------------------------------------------------------- calls
def graph_from_edges(ctx: Context, n, src, dst) -> Graph:
    """numpy (host) or torch CUDA (device) uint32 arrays of equal length."""
    m = len(src)
    dev = _is_device(src)
    if not dev:
        src = _host_u32(src)
        dst = _host_u32(dst)
    h = VP()
    ctx.check(lib().drg_graph_from_edges(ctx.h, int(n), int(m), _ptr(src), _ptr(dst), int(dev), C.byref(h)))
    return Graph(ctx, h)


def build_distance_matrix(ctx: Context, g: Graph, k: int, sigma: float = 1.0,
                          perplexity: float = 0.0, row_cap: int = 0) -> DistanceMatrix:
    """perplexity > 0: sigma_i per node calibrated to that perplexity (any
    other non-zero value is refused by the library); row_cap > 0: every row
    keeps its row_cap nearest nodes, pattern K u K^T."""
    h = VP()
    if row_cap:
        ctx.check(lib().drg_build_distance_matrix_capped(ctx.h, g.h, int(k), float(sigma), int(row_cap), C.byref(h)))
    elif perplexity != 0.0:
        ctx.check(lib().drg_build_distance_matrix_ex(ctx.h, g.h, int(k), float(sigma), float(perplexity),
                                                     C.byref(h)))
    else:
        ctx.check(lib().drg_build_distance_matrix(ctx.h, g.h, int(k), float(sigma), C.byref(h)))
    d = DistanceMatrix(ctx, h)
    d.graph = g
    return d


def crossings(ctx: Context, g: Graph, pos):
    """Sec. 4.1 Eq. 17 of a drawing (device positions): (crossings, crosslessness)."""
    c = C.c_uint64()
    cl = C.c_double()
    ctx.check(lib().drg_crossings(ctx.h, g.h, _ptr(pos), C.byref(c), C.byref(cl)))
    return int(c.value), float(cl.value)


def min_angle(ctx: Context, g: Graph, pos) -> float:
    """Sec. 4.1 Eq. 19 of a drawing (device positions)."""
    out = C.c_double()
    ctx.check(lib().drg_min_angle(ctx.h, g.h, _ptr(pos), C.byref(out)))
    return float(out.value)


def coarsen(ctx: Context, g: Graph, level: int, p: Params, parent) -> Graph:
    """parent: torch CUDA uint32/int32 tensor of n entries (written)."""
    h = VP()
    ctx.check(lib().drg_coarsen(ctx.h, g.h, int(level), C.byref(p), C.byref(h), _ptr(parent)))
    return Graph(ctx, h)


def build_hierarchy(ctx: Context, g: Graph, p: Params) -> Hierarchy:
    h = VP()
    ctx.check(lib().drg_build_hierarchy(ctx.h, g.h, C.byref(p), C.byref(h)))
    return Hierarchy(ctx, h, g)


def init_positions(ctx: Context, n, level, p: Params, pos):
    ctx.check(lib().drg_init_positions(ctx.h, int(n), int(level), C.byref(p), _ptr(pos)))


def layout_level(ctx: Context, d: DistanceMatrix, h: Hierarchy | None, level, pos, p: Params, gamma,
                 t_begin=0, t_end=None):
    t_end = p.epochs if t_end is None else t_end
    ctx.check(lib().drg_layout_level(ctx.h, d.h, None if h is None else h.h, int(level), _ptr(pos), C.byref(p),
                                     float(gamma), int(t_begin), int(t_end)))


def interpolate(ctx: Context, h: Hierarchy, coarse_level, coarse_pos, fine_pos):
    ctx.check(lib().drg_interpolate(ctx.h, h.h, int(coarse_level), _ptr(coarse_pos), _ptr(fine_pos)))


def check_epoch_barrier(ctx: Context, blocks, arrivals, rounds=1, timeout_ms=50) -> int:
    """Status (0 ok, 4 timed out, ...) of the epoch-barrier self-check; does not raise."""
    return int(lib().drg_check_epoch_barrier(ctx.h, int(blocks), int(arrivals), int(rounds), int(timeout_ms)))


def layout(ctx: Context, g: Graph, p: Params, pos):
    ctx.check(lib().drg_layout(ctx.h, g.h, C.byref(p), _ptr(pos)))


def layout_edges(ctx: Context, n, src, dst, p: Params, pos):
    """Whole pipeline from an edge list; host (numpy) or device (torch) edges
    and positions, each copied on the context stream as needed."""
    e_dev = _is_device(src)
    if not e_dev:
        src = _host_u32(src)
        dst = _host_u32(dst)
    ctx.check(lib().drg_layout_edges(ctx.h, int(n), int(len(src)), _ptr(src), _ptr(dst), int(e_dev), C.byref(p),
                                     _ptr(pos), int(_is_device(pos))))


def layout_batch(ctx: Context, graphs, p: Params, positions, b=None):
    """b: optional per-graph kernel shapes (sequence of floats)."""
    n = len(graphs)
    garr = (VP * max(n, 1))(*[g.h for g in graphs])
    parr = (VP * max(n, 1))(*[_ptr(x) for x in positions])
    barr = None if b is None else np.ascontiguousarray(b, np.float32)
    ctx.check(lib().drg_layout_batch(ctx.h, n, garr, C.byref(p), _ptr(barr), parr))


def sample_draws(ctx: Context, d: DistanceMatrix, level, t, s_begin, s_end, p: Params, out_i, out_j, out_neg):
    ctx.check(lib().drg_sample_draws(ctx.h, d.h, int(level), int(t), int(s_begin), int(s_end), C.byref(p),
                                     _ptr(out_i), _ptr(out_j), _ptr(out_neg)))


def probe_memory(ctx: Context, kind, buffer_bytes, accesses, blocks_per_sm=6):
    """One memory probe (PROBE_*): (milliseconds, accesses made)."""
    ms = C.c_double()
    done = C.c_uint64()
    ctx.check(lib().drg_probe_memory(ctx.h, int(kind), int(buffer_bytes), int(accesses), int(blocks_per_sm),
                                     C.byref(ms), C.byref(done)))
    return ms.value, done.value


def autotune_table():
    """The process-wide tuned launch shapes: a list of dicts."""
    cnt = C.c_uint32()
    lib().drg_autotune_read(0, None, None, None, C.byref(cnt))
    n = cnt.value
    keys = np.zeros(6 * max(n, 1), np.uint32)
    choice = np.zeros(2 * max(n, 1), np.uint32)
    ms = np.zeros(max(n, 1), np.float32)
    lib().drg_autotune_read(n, _ptr(keys), _ptr(choice), _ptr(ms), C.byref(cnt))
    return [dict(kernel=("k_hogwild", "k_hogwild_batch")[int(keys[6 * i])], M=int(keys[6 * i + 1]),
                 precision=int(keys[6 * i + 2]), ancestors=int(keys[6 * i + 3]), bucket=int(keys[6 * i + 4]),
                 device=int(keys[6 * i + 5]), block=int(choice[2 * i]), divisor=int(choice[2 * i + 1]),
                 ms_per_epoch=float(ms[i])) for i in range(min(n, cnt.value))]


def autotune_clear():
    lib().drg_autotune_clear()


def layout_step_explicit(ctx: Context, pos, src, dst, neg, M, gamma, b, lr, clip=5.0):
    """One synchronous step over caller-given samples (device tensors: src,
    dst of S node ids, neg of S * M); pos is updated in place."""
    S = int(src.numel())
    n = int(pos.numel()) // 2
    ctx.check(lib().drg_layout_step_explicit(ctx.h, n, _ptr(pos), S, _ptr(src), _ptr(dst),
                                             _ptr(neg) if M else None, int(M), float(gamma), float(b), float(lr),
                                             float(clip)))
