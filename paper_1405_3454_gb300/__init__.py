"""GB300-native CudaPre: convex-hull preprocessing on the GPU (arXiv 1405.3454).

A thin ctypes binding over the C ABI in ``include/cudapre.h`` (library
``libcudapre.so`` built in-tree by ``_build.build()``).  This module only
marshals arguments: every step of the method runs in the CUDA kernels.
PyTorch provides device memory and streams.  There is no CPU fallback: if the
library is missing every call raises.

Entry points (same names as the C ABI):
  hull_prefilter  Steps 1-3 of section 2: survivors of the 16-extreme filter.
  hull_compute    the whole method: the convex hull via the filter.
Convenience wrappers ``prefilter`` and ``compute`` allocate outputs and a
workspace with torch.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcudapre.so")

HULL_OK = 0
HULL_ANGLES_CUMULATIVE = 0
HULL_ANGLES_ABSOLUTE = 1
HULL_FILTER_EXACT = 0
HULL_FILTER_FP32 = 1
HULL_DEVICE_DOMAIN = 1
HULL_DEVICE_TIMEOUT = 2
HULL_DEVICE_OVERFLOW = 4
NONE_IDX = 0xFFFFFFFF

# Exported symbols declared in include/cudapre.h.
ABI_SYMBOLS = (
    "hull_default_options", "hull_prefilter_workspace_bytes", "hull_workspace_bytes",
    "hull_prefilter", "hull_compute", "hull_read_counters", "hull_read_polygon",
    "hull_get_device_status", "hull_strerror", "hull_constants", "hull_abi_version", "hull_read_stats",
    "hull_timer_create", "hull_timer_destroy", "hull_timer_attach", "hull_timer_read", "hull_launch_count",
    "hull_compute_static", "hull_batch", "hull_batch_workspace_bytes", "hull_batch_ranges",
    "hull_selftest_wait", "hull_batch_read_set", "hull_graph_create", "hull_graph_destroy",
    "hull_graph_batch_ranges", "hull_graph_counts", "hull3_prefilter_workspace_bytes", "hull3_prefilter",
    "hull3_read_polyhedron",
)
HULL_STAGES = 6
STAGE_NAMES = ("validate", "extremes", "polygon", "filter", "hull", "final")


class HullOptions(ctypes.Structure):
    _fields_ = [("angles", ctypes.c_int32), ("filter", ctypes.c_int32), ("validate", ctypes.c_int32),
                ("block", ctypes.c_int32), ("grid", ctypes.c_int32), ("refine", ctypes.c_int32),
                ("no_prefilter", ctypes.c_int32), ("waves", ctypes.c_int32), ("unit_chunks", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 7)]


class HullStats(ctypes.Structure):
    _fields_ = [("n_survivors", ctypes.c_int64), ("n_escalated", ctypes.c_int64), ("n_refined", ctypes.c_int64),
                ("polygon_vertices", ctypes.c_int32), ("device_status", ctypes.c_uint32)]


class HullSetInfo(ctypes.Structure):
    _fields_ = [("polygon_vertices", ctypes.c_int32), ("polygon_xy", ctypes.c_int32 * 32),
                ("polygon_idx", ctypes.c_uint32 * 16), ("extreme_idx", ctypes.c_uint32 * 16),
                ("n_survivors", ctypes.c_int64), ("n_escalated", ctypes.c_int64), ("n_refined", ctypes.c_int64),
                ("device_status", ctypes.c_uint32), ("pad_", ctypes.c_uint32)]


class HullError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__("%s: %s" % (where, strerror(code)))


_lib = None


def load(path: str | None = None):
    """Load libcudapre.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError("libcudapre.so not built (run __graft_entry__.build() or "
                           "paper_1405_3454_gb300._build.build()): %s" % p)
    lib = ctypes.CDLL(p)
    P, i64, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_size_t
    OP = ctypes.POINTER(HullOptions)
    st = ctypes.c_int
    lib.hull_default_options.argtypes = [OP]
    lib.hull_default_options.restype = None
    lib.hull_prefilter_workspace_bytes.argtypes = [i64, OP]
    lib.hull_prefilter_workspace_bytes.restype = sz
    lib.hull_workspace_bytes.argtypes = [i64, OP]
    lib.hull_workspace_bytes.restype = sz
    lib.hull_prefilter.argtypes = [P, i64, P, sz, P, P, P, OP, P]
    lib.hull_prefilter.restype = st
    lib.hull_compute.argtypes = [P, i64, P, sz, P, P, OP, P]
    lib.hull_compute.restype = st
    lib.hull_read_counters.argtypes = [P, P, P, P]
    lib.hull_read_counters.restype = st
    lib.hull_read_polygon.argtypes = [P, P, P, P, P]
    lib.hull_read_polygon.restype = st
    lib.hull_get_device_status.argtypes = [P, P, P]
    lib.hull_get_device_status.restype = st
    lib.hull_strerror.argtypes = [st]
    lib.hull_strerror.restype = ctypes.c_char_p
    lib.hull_constants.argtypes = [P]
    lib.hull_constants.restype = None
    lib.hull_abi_version.argtypes = []
    lib.hull_abi_version.restype = ctypes.c_int32
    lib.hull_read_stats.argtypes = [P, ctypes.POINTER(HullStats), P]
    lib.hull_read_stats.restype = st
    lib.hull_timer_create.argtypes = [ctypes.c_int32]
    lib.hull_timer_create.restype = P
    lib.hull_timer_destroy.argtypes = [P]
    lib.hull_timer_destroy.restype = None
    lib.hull_timer_attach.argtypes = [P]
    lib.hull_timer_attach.restype = None
    lib.hull_timer_read.argtypes = [P, P, P]
    lib.hull_timer_read.restype = st
    lib.hull_launch_count.argtypes = []
    lib.hull_launch_count.restype = ctypes.c_int64
    lib.hull_compute_static.argtypes = [P, i64, P, P, OP, P]
    lib.hull_compute_static.restype = st
    lib.hull_batch_workspace_bytes.argtypes = [i64, ctypes.c_int32, OP]
    lib.hull_batch_workspace_bytes.restype = sz
    lib.hull_batch.argtypes = [P, P, ctypes.c_int32, i64, P, sz, P, P, OP, P]
    lib.hull_batch.restype = st
    lib.hull_batch_ranges.argtypes = [P, i64, P, P, ctypes.c_int32, i64, P, sz, P, P, OP, P]
    lib.hull_batch_ranges.restype = st
    lib.hull_selftest_wait.argtypes = [P, i64, P]
    lib.hull_selftest_wait.restype = st
    lib.hull_batch_read_set.argtypes = [P, i64, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(HullSetInfo), P]
    lib.hull_batch_read_set.restype = st
    lib.hull_graph_create.argtypes = []
    lib.hull_graph_create.restype = P
    lib.hull_graph_destroy.argtypes = [P]
    lib.hull_graph_destroy.restype = None
    lib.hull_graph_batch_ranges.argtypes = [P, P, i64, P, P, ctypes.c_int32, i64, P, sz, P, P, OP, P]
    lib.hull_graph_batch_ranges.restype = st
    lib.hull_graph_counts.argtypes = [P, P]
    lib.hull_graph_counts.restype = None
    lib.hull3_prefilter_workspace_bytes.argtypes = [i64, OP]
    lib.hull3_prefilter_workspace_bytes.restype = sz
    lib.hull3_prefilter.argtypes = [P, i64, P, sz, P, P, P, OP, P]
    lib.hull3_prefilter.restype = st
    lib.hull3_read_polyhedron.argtypes = [P, P, P, P, P, P]
    lib.hull3_read_polyhedron.restype = st
    _lib = lib
    return lib


def strerror(code: int) -> str:
    try:
        return load().hull_strerror(code).decode()
    except Exception:
        return "hull_status %d" % code


def _check(code: int, where: str):
    if code != HULL_OK:
        raise HullError(code, where)


@dataclass
class Options:
    angles: int = HULL_ANGLES_CUMULATIVE
    filter: int = HULL_FILTER_FP32
    validate: bool = False
    block: int = 0
    grid: int = 0
    refine: bool = True
    no_prefilter: bool = False
    waves: int = 0
    unit_chunks: int = 0

    def c(self) -> HullOptions:
        o = HullOptions()
        load().hull_default_options(ctypes.byref(o))
        o.angles, o.filter, o.validate = int(self.angles), int(self.filter), int(bool(self.validate))
        o.block, o.grid, o.refine = int(self.block), int(self.grid), int(bool(self.refine))
        o.no_prefilter = int(bool(self.no_prefilter))
        o.waves, o.unit_chunks = int(self.waves), int(self.unit_chunks)
        return o


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


def _stream_handle(stream) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _check_points(xy):
    import torch
    if not isinstance(xy, torch.Tensor) or not xy.is_cuda:
        raise TypeError("xy must be a CUDA torch.Tensor")
    if xy.dtype != torch.float32 or xy.dim() != 2 or xy.shape[1] != 2 or not xy.is_contiguous():
        raise ValueError("xy must be a contiguous float32 tensor of shape [n, 2]")
    return int(xy.shape[0])


# --------------------------------------------------------------------------
# C-ABI mirrors (raw pointers as ints, stream handle as int).

def hull_prefilter_workspace_bytes(n: int, opt: Options | None = None) -> int:
    return int(load().hull_prefilter_workspace_bytes(n, ctypes.byref((opt or Options()).c())))


def hull_workspace_bytes(n: int, opt: Options | None = None) -> int:
    return int(load().hull_workspace_bytes(n, ctypes.byref((opt or Options()).c())))


def hull_prefilter(d_xy: int, n: int, d_ws: int, ws_bytes: int, d_survivor_idx: int, d_n_survivors: int,
                   d_extreme_idx: int, opt: Options | None, stream: int) -> int:
    o = (opt or Options()).c()
    return load().hull_prefilter(d_xy, n, d_ws, ws_bytes, d_survivor_idx, d_n_survivors, d_extreme_idx or None,
                                 ctypes.byref(o), stream or None)


def hull_compute(d_xy: int, n: int, d_ws: int, ws_bytes: int, d_hull_idx: int, d_n_hull: int,
                 opt: Options | None, stream: int) -> int:
    o = (opt or Options()).c()
    return load().hull_compute(d_xy, n, d_ws, ws_bytes, d_hull_idx, d_n_hull, ctypes.byref(o), stream or None)


HULL_STATIC_MAX_POINTS = 1 << 20
HULL_DEVICE_OFFSETS = 8


def hull_batch_workspace_bytes(n_total: int, S: int, opt: Options | None = None) -> int:
    o = (opt or Options()).c()
    return int(load().hull_batch_workspace_bytes(n_total, S, ctypes.byref(o)))


def hull_batch(d_xy: int, d_offsets: int, S: int, n_total: int, d_ws: int, ws_bytes: int, d_hull_idx: int,
               d_hull_offsets: int, opt: Options | None, stream: int) -> int:
    o = (opt or Options()).c()
    return load().hull_batch(d_xy or None, d_offsets, S, n_total, d_ws, ws_bytes, d_hull_idx or None,
                             d_hull_offsets, ctypes.byref(o), stream or None)


def hull_compute_static(d_xy: int, n: int, d_hull_idx: int, d_n_hull: int, opt: Options | None,
                        stream: int) -> int:
    """hull_compute on the library's fixed per-device workspace (at most
    HULL_STATIC_MAX_POINTS points; the call allocates nothing)."""
    o = (opt or Options()).c()
    return load().hull_compute_static(d_xy, n, d_hull_idx, d_n_hull, ctypes.byref(o), stream or None)


# --------------------------------------------------------------------------
# Tensor-level wrappers.

def workspace(nbytes: int, device=None):
    import torch
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device or "cuda")


def prefilter(xy, opt: Options | None = None, ws=None, stream=None):
    """Steps 1-3 on one set.  Returns (survivor_idx int32 [n] (uint32 bits),
    n_survivors int64 [1], extreme_idx int32 [16] (uint32 bits), ws).
    Only the first n_survivors entries of survivor_idx are defined."""
    import torch
    n = _check_points(xy)
    opt = opt or Options()
    need = hull_prefilter_workspace_bytes(n, opt)
    if ws is None or ws.numel() < need:
        ws = workspace(need, xy.device)
    surv = torch.empty(max(n, 1), dtype=torch.int32, device=xy.device)
    cnt = torch.empty(1, dtype=torch.int64, device=xy.device)
    ext = torch.empty(16, dtype=torch.int32, device=xy.device)
    _check(hull_prefilter(_ptr(xy), n, _ptr(ws), ws.numel(), _ptr(surv), _ptr(cnt), _ptr(ext), opt,
                          _stream_handle(stream)), "hull_prefilter")
    return surv, cnt, ext, ws


def compute(xy, opt: Options | None = None, ws=None, stream=None):
    """The whole method on one set.  Returns (hull_idx int32 [n] (uint32 bits),
    n_hull int64 [1], ws).  Only the first n_hull entries are defined."""
    import torch
    n = _check_points(xy)
    opt = opt or Options()
    need = hull_workspace_bytes(n, opt)
    if ws is None or ws.numel() < need:
        ws = workspace(need, xy.device)
    out = torch.empty(max(n, 1), dtype=torch.int32, device=xy.device)
    cnt = torch.empty(1, dtype=torch.int64, device=xy.device)
    _check(hull_compute(_ptr(xy), n, _ptr(ws), ws.numel(), _ptr(out), _ptr(cnt), opt, _stream_handle(stream)),
           "hull_compute")
    return out, cnt, ws


def batch(xy, offsets, opt: Options | None = None, ws=None, stream=None):
    """The whole method on each set of a batch.  xy: float32 [n_total, 2] on
    the device; offsets: int64 [S+1] on the device (set s = rows offsets[s] ..
    offsets[s+1]).  Returns (hull_idx int64 [n_total] of global row indices,
    hull_offsets int64 [S+1], ws); set s's hull is
    hull_idx[hull_offsets[s]:hull_offsets[s+1]]."""
    import torch
    n_total = _check_points(xy)
    if offsets.dtype != torch.int64 or offsets.dim() != 1 or offsets.device != xy.device:
        raise ValueError("offsets must be a 1-D int64 tensor on the points' device")
    S = offsets.numel() - 1
    if S < 0:
        raise ValueError("offsets must hold S+1 >= 1 entries")
    opt = opt or Options()
    need = hull_batch_workspace_bytes(n_total, S, opt)
    if ws is None or ws.numel() < need:
        ws = workspace(need, xy.device)
    out = torch.empty(max(n_total, 1), dtype=torch.int64, device=xy.device)
    hoff = torch.empty(S + 1, dtype=torch.int64, device=xy.device)
    _check(hull_batch(_ptr(xy), _ptr(offsets), S, n_total, _ptr(ws), ws.numel(), _ptr(out), _ptr(hoff), opt,
                      _stream_handle(stream)), "hull_batch")
    return out, hoff, ws


def hull_batch_ranges(d_xy: int, n_xy: int, d_starts: int, d_offsets: int, S: int, n_total: int, d_ws: int,
                      ws_bytes: int, d_hull_idx: int, d_hull_offsets: int, opt: Options | None, stream: int) -> int:
    o = (opt or Options()).c()
    return load().hull_batch_ranges(d_xy or None, n_xy, d_starts or None, d_offsets, S, n_total, d_ws, ws_bytes,
                                    d_hull_idx or None, d_hull_offsets, ctypes.byref(o), stream or None)


def batch_ranges(pool, starts, sizes, opt: Options | None = None, ws=None, stream=None):
    """hull_batch_ranges on a resident pool: set s = pool rows starts[s] ..
    starts[s] + sizes[s].  pool float32 [n_xy, 2], starts / sizes int64 [S]
    on the pool's device.  Returns (hull_idx int64 (pool rows), hull_offsets
    int64 [S+1], ws)."""
    import torch
    n_xy = _check_points(pool)
    S = starts.numel()
    offsets = torch.zeros(S + 1, dtype=torch.int64, device=pool.device)
    if S:
        torch.cumsum(sizes, 0, out=offsets[1:])
    n_total = int(offsets[-1].item()) if S else 0
    opt = opt or Options()
    need = hull_batch_workspace_bytes(n_total, S, opt)
    if ws is None or ws.numel() < need:
        ws = workspace(need, pool.device)
    out = torch.empty(max(n_total, 1), dtype=torch.int64, device=pool.device)
    hoff = torch.empty(S + 1, dtype=torch.int64, device=pool.device)
    _check(hull_batch_ranges(_ptr(pool), n_xy, _ptr(starts), _ptr(offsets), S, n_total, _ptr(ws), ws.numel(),
                             _ptr(out), _ptr(hoff), opt, _stream_handle(stream)), "hull_batch_ranges")
    return out, hoff, ws


def hull_graph_batch_ranges(g: int, d_xy: int, n_xy: int, d_starts: int, d_offsets: int, S: int, n_total: int,
                            d_ws: int, ws_bytes: int, d_hull_idx: int, d_hull_offsets: int, opt: Options | None,
                            stream: int) -> int:
    o = (opt or Options()).c()
    return load().hull_graph_batch_ranges(g, d_xy or None, n_xy, d_starts or None, d_offsets, S, n_total, d_ws,
                                          ws_bytes, d_hull_idx or None, d_hull_offsets, ctypes.byref(o),
                                          stream or None)


class Graph:
    """Batches run as CUDA graphs (hull_graph_*): a call repeating the
    previous call's arguments replays its graph with one launch."""

    def __init__(self):
        self._g = load().hull_graph_create()
        if not self._g:
            raise RuntimeError("hull_graph_create failed")

    def batch_ranges(self, pool, starts, offsets, n_total: int, ws, out, hoff, opt: Options | None = None,
                     stream=None):
        """hull_batch_ranges through the graph; starts (or None for
        contiguous sets) and offsets are int64 device tensors, the outputs and
        workspace preallocated (sizes as for hull_batch_ranges)."""
        S = offsets.numel() - 1
        n_xy = _check_points(pool)
        code = hull_graph_batch_ranges(self._g, _ptr(pool), n_xy if starts is not None else n_total, _ptr(starts),
                                       _ptr(offsets), S, n_total, _ptr(ws), ws.numel(), _ptr(out), _ptr(hoff), opt,
                                       _stream_handle(stream))
        _check(code, "hull_graph_batch_ranges")

    def counts(self) -> dict:
        a = (ctypes.c_int64 * 6)()
        load().hull_graph_counts(self._g, a)
        return dict(zip(("calls", "captures", "updates", "instantiations", "replays", "kernels"), [int(v) for v in a]))

    def close(self):
        if self._g:
            load().hull_graph_destroy(self._g)
            self._g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --------------------------------------------------------------------------
# The 3D extension (section 5).

HULL3_SLOTS = 24
HULL3_MAX_FACETS = 48


def hull3_prefilter_workspace_bytes(n: int, opt: Options | None = None) -> int:
    return int(load().hull3_prefilter_workspace_bytes(n, ctypes.byref((opt or Options()).c())))


def hull3_prefilter(d_xyz: int, n: int, d_ws: int, ws_bytes: int, d_survivor_idx: int, d_n_survivors: int,
                    d_extreme_idx: int, opt: Options | None, stream: int) -> int:
    o = (opt or Options()).c()
    return load().hull3_prefilter(d_xyz or None, n, d_ws, ws_bytes, d_survivor_idx or None, d_n_survivors,
                                  d_extreme_idx or None, ctypes.byref(o), stream or None)


def _check_points3(xyz):
    import torch
    if not isinstance(xyz, torch.Tensor) or not xyz.is_cuda:
        raise TypeError("xyz must be a CUDA torch.Tensor")
    if xyz.dtype != torch.float32 or xyz.dim() != 2 or xyz.shape[1] != 3 or not xyz.is_contiguous():
        raise ValueError("xyz must be a contiguous float32 tensor of shape [n, 3]")
    return int(xyz.shape[0])


def prefilter3(xyz, opt: Options | None = None, ws=None, stream=None):
    """The 3D extension on one set.  Returns (survivor_idx int32 [n] (uint32
    bits), n_survivors int64 [1], extreme_idx int32 [24] (uint32 bits), ws)."""
    import torch
    n = _check_points3(xyz)
    opt = opt or Options()
    need = hull3_prefilter_workspace_bytes(n, opt)
    if ws is None or ws.numel() < need:
        ws = workspace(need, xyz.device)
    surv = torch.empty(max(n, 1), dtype=torch.int32, device=xyz.device)
    cnt = torch.empty(1, dtype=torch.int64, device=xyz.device)
    ext = torch.empty(HULL3_SLOTS, dtype=torch.int32, device=xyz.device)
    _check(hull3_prefilter(_ptr(xyz), n, _ptr(ws), ws.numel(), _ptr(surv), _ptr(cnt), _ptr(ext), opt,
                           _stream_handle(stream)), "hull3_prefilter")
    return surv, cnt, ext, ws


def read_polyhedron(ws, stream=None) -> dict:
    """The last hull3_prefilter's polyhedron: facet planes [m][4] (int),
    extremes [24], survivors, escalations, status bits."""
    nf = ctypes.c_int32(0)
    planes = (ctypes.c_int64 * (4 * HULL3_MAX_FACETS))()
    ext = (ctypes.c_uint32 * HULL3_SLOTS)()
    counts = (ctypes.c_int64 * 3)()
    _check(load().hull3_read_polyhedron(_ptr(ws), ctypes.byref(nf), planes, ext, counts, _stream_handle(stream)),
           "hull3_read_polyhedron")
    m = int(nf.value)
    return {"planes": [[int(planes[4 * k + q]) for q in range(4)] for k in range(m)],
            "extremes": [int(v) for v in ext], "n_survivors": int(counts[0]), "n_escalated": int(counts[1]),
            "device_status": int(counts[2])}


def read_counters(ws, stream=None):
    ns, ne = ctypes.c_int64(0), ctypes.c_int64(0)
    _check(load().hull_read_counters(_ptr(ws), ctypes.byref(ns), ctypes.byref(ne), _stream_handle(stream)),
           "hull_read_counters")
    return int(ns.value), int(ne.value)


def read_stats(ws, stream=None) -> dict:
    """Counters of the last call on this workspace."""
    o = HullStats()
    _check(load().hull_read_stats(_ptr(ws), ctypes.byref(o), _stream_handle(stream)), "hull_read_stats")
    return {k: int(getattr(o, k)) for k, _ in HullStats._fields_}


def read_polygon(ws, stream=None):
    """(m, xy [m][2] list, vertex point indices [m] list) of the last call's Step-2 polygon."""
    m = ctypes.c_int32(0)
    xy = (ctypes.c_int32 * 32)()
    idx = (ctypes.c_uint32 * 16)()
    _check(load().hull_read_polygon(_ptr(ws), ctypes.byref(m), xy, idx, _stream_handle(stream)),
           "hull_read_polygon")
    k = int(m.value)
    return k, [[xy[2 * i], xy[2 * i + 1]] for i in range(k)], [int(idx[i]) for i in range(k)]


def batch_read_set(ws, n_total: int, S: int, s: int, stream=None) -> dict:
    """Set s of the last batch call on a batch workspace laid out for
    (n_total, S): its polygon (m, xy, point indices within the set), its 16
    extremes (indices within the set), its counters and status bits."""
    o = HullSetInfo()
    _check(load().hull_batch_read_set(_ptr(ws), int(n_total), int(S), int(s), ctypes.byref(o),
                                      _stream_handle(stream)), "hull_batch_read_set")
    m = int(o.polygon_vertices)
    return {"m": m, "poly_xy": [[o.polygon_xy[2 * k], o.polygon_xy[2 * k + 1]] for k in range(m)],
            "poly_idx": [int(o.polygon_idx[k]) for k in range(m)],
            "extremes": [int(v) for v in o.extreme_idx], "n_survivors": int(o.n_survivors),
            "n_escalated": int(o.n_escalated), "n_refined": int(o.n_refined),
            "device_status": int(o.device_status)}


def device_status(ws, stream=None):
    bits = ctypes.c_uint32(0)
    code = load().hull_get_device_status(_ptr(ws), ctypes.byref(bits), _stream_handle(stream))
    return int(code), int(bits.value)


def selftest_wait(ws, limit_cycles: int = 1 << 20, stream=None):
    """Run one bounded device wait that nothing releases (a test of the
    timeout path); the workspace's status then reads HULL_ERR_TIMEOUT."""
    _check(load().hull_selftest_wait(_ptr(ws), int(limit_cycles), _stream_handle(stream)), "hull_selftest_wait")


def constants():
    arr = (ctypes.c_double * 4)()
    load().hull_constants(arr)
    return {"s3": arr[0], "c75": arr[1], "s75": arr[2], "h": arr[3]}


def as_index(t, count=None):
    """uint32 bits stored in an int32 tensor -> int64 indices (host numpy)."""
    import numpy as np
    a = t.cpu().numpy().view(np.uint32).astype(np.int64)
    return a if count is None else a[: int(count)]


class StageTimer:
    """Per-stage device time of the calls made on this host thread while attached."""

    def __init__(self, max_calls: int = 256):
        self._t = load().hull_timer_create(max_calls)
        if not self._t:
            raise RuntimeError("hull_timer_create failed")

    def attach(self):
        load().hull_timer_attach(self._t)

    def detach(self):
        load().hull_timer_attach(None)

    def read(self):
        """(dict stage -> total ms, number of recorded calls); clears the timer."""
        ms = (ctypes.c_float * HULL_STAGES)()
        calls = ctypes.c_int32(0)
        _check(load().hull_timer_read(self._t, ms, ctypes.byref(calls)), "hull_timer_read")
        return {STAGE_NAMES[i]: float(ms[i]) for i in range(HULL_STAGES)}, int(calls.value)

    def close(self):
        if self._t:
            load().hull_timer_destroy(self._t)
            self._t = None


def launch_count() -> int:
    return int(load().hull_launch_count())
