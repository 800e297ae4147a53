"""Python access to the CPU oracle (``oracle.cpp``).

TEST INFRASTRUCTURE ONLY: imported by the test suite, by the smoke check in
``__graft_entry__`` and by the CPU-baseline leg of ``bench.py``, never by the
product package.  It shares no code with the CUDA path.

Every function follows a step of the paper (arXiv 1405.3454, section 2):
``extremes`` (Step 1), ``hull16`` (Step 2, Andrew's monotone chain),
``prefilter`` (Step 3) and ``hull`` (the hull of the remaining points,
section 3 case (2); on all points it is the plain definition of the hull).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

ANGLES_CUMULATIVE = 0  # 0, 30, 75, 120 degrees
ANGLES_ABSOLUTE = 1  # 0, 30, 45, 60 degrees


def build(force: bool = False) -> str:
    """Compile liboracle.so with g++ -O2 -ffp-contract=off (no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        subprocess.check_call(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-Wno-stringop-overflow", "-shared", "-fPIC",
                               "-pthread", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _get():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i64 = ctypes.c_int64
        lib.oracle_constants.argtypes = [P]
        lib.oracle_rotate.argtypes = [ctypes.c_float, ctypes.c_float, ctypes.c_int, ctypes.c_int, P]
        lib.oracle_check_domain.argtypes = [P, i64]
        lib.oracle_check_domain.restype = ctypes.c_int
        lib.oracle_extremes.argtypes = [P, i64, ctypes.c_int, P]
        lib.oracle_hull16.argtypes = [P, P, P, P]
        lib.oracle_hull16.restype = ctypes.c_int
        lib.oracle_strictly_inside.argtypes = [P, ctypes.c_int, i64, i64]
        lib.oracle_strictly_inside.restype = ctypes.c_int
        lib.oracle_prefilter.argtypes = [P, i64, P, ctypes.c_int, P]
        lib.oracle_prefilter.restype = i64
        lib.oracle_hull.argtypes = [P, P, i64, P]
        lib.oracle_hull.restype = i64
        lib.oracle_brute_hull.argtypes = [P, i64, P]
        lib.oracle_brute_hull.restype = i64
        lib.oracle_cudapre.argtypes = [P, i64, ctypes.c_int, P, P, P, P, P, P, P]
        lib.oracle_cudapre_mt.argtypes = [P, i64, ctypes.c_int, ctypes.c_int, P, P, P, P, P, P, P]
        lib.oracle_cudapre_mt.restype = ctypes.c_int
        lib.oracle3_extremes.argtypes = [P, i64, ctypes.c_int, P]
        lib.oracle3_facets.argtypes = [P, P, ctypes.c_int, P, ctypes.c_int]
        lib.oracle3_facets.restype = ctypes.c_int
        lib.oracle3_prefilter.argtypes = [P, i64, P, ctypes.c_int, P]
        lib.oracle3_prefilter.restype = i64
        lib.oracle3_check_domain.argtypes = [P, i64]
        lib.oracle3_check_domain.restype = ctypes.c_int
        _lib = lib
    return _lib


def _pts(xy) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(xy, dtype=np.float32).reshape(-1, 2))
    return a


def constants() -> dict:
    out = np.zeros(4, dtype=np.float64)
    _get().oracle_constants(out.ctypes.data)
    return {"s3": float(out[0]), "c75": float(out[1]), "s75": float(out[2]), "h": float(out[3])}


def rotate(x: float, y: float, group: int, angles: int = ANGLES_CUMULATIVE):
    out = np.zeros(2, dtype=np.float64)
    _get().oracle_rotate(float(x), float(y), angles, group, out.ctypes.data)
    return float(out[0]), float(out[1])


def check_domain(xy) -> bool:
    a = _pts(xy)
    return bool(_get().oracle_check_domain(a.ctypes.data, a.shape[0]))


def extremes(xy, angles: int = ANGLES_CUMULATIVE) -> np.ndarray:
    """Step 1: 16 extreme indices, slot 4g+{0,1,2,3} = argmin x', argmax x', argmin y', argmax y'."""
    a = _pts(xy)
    out = np.full(16, -1, dtype=np.int64)
    _get().oracle_extremes(a.ctypes.data, a.shape[0], angles, out.ctypes.data)
    return out


def hull16(xy, ext_idx) -> tuple[np.ndarray, np.ndarray]:
    """Step 2: polygon of the extremes; returns (vertex indices [m], vertex coords [m, 2] int32)."""
    a = _pts(xy)
    e = np.ascontiguousarray(np.asarray(ext_idx, dtype=np.int64))
    pidx = np.zeros(16, dtype=np.int64)
    pxy = np.zeros(32, dtype=np.int32)
    m = _get().oracle_hull16(a.ctypes.data, e.ctypes.data, pidx.ctypes.data, pxy.ctypes.data)
    return pidx[:m].copy(), pxy[: 2 * m].reshape(m, 2).copy()


def strictly_inside(poly_xy, px: int, py: int) -> bool:
    p = np.ascontiguousarray(np.asarray(poly_xy, dtype=np.int32).reshape(-1, 2))
    return bool(_get().oracle_strictly_inside(p.ctypes.data, p.shape[0], int(px), int(py)))


def prefilter(xy, poly_xy) -> np.ndarray:
    """Step 3: ascending indices of the points not strictly inside the polygon."""
    a = _pts(xy)
    p = np.ascontiguousarray(np.asarray(poly_xy, dtype=np.int32).reshape(-1, 2))
    out = np.empty(max(a.shape[0], 1), dtype=np.int64)
    c = _get().oracle_prefilter(a.ctypes.data, a.shape[0], p.ctypes.data, p.shape[0], out.ctypes.data)
    return out[:c].copy()


def hull(xy, idx=None) -> np.ndarray:
    """Convex hull (CCW from the lexicographic minimum, strictly convex) of xy[idx] (all if None)."""
    a = _pts(xy)
    if idx is None:
        k = a.shape[0]
        ip = None
    else:
        ia = np.ascontiguousarray(np.asarray(idx, dtype=np.int64))
        k = ia.shape[0]
        ip = ia.ctypes.data
    out = np.empty(max(k, 1), dtype=np.int64)
    c = _get().oracle_hull(a.ctypes.data, ip, k, out.ctypes.data)
    return out[:c].copy()


def brute_hull(xy) -> np.ndarray:
    a = _pts(xy)
    out = np.empty(max(a.shape[0], 1), dtype=np.int64)
    c = _get().oracle_brute_hull(a.ctypes.data, a.shape[0], out.ctypes.data)
    if c < 0:
        raise ValueError("brute_hull: input too large or malformed (%d)" % c)
    return out[:c].copy()


def cudapre(xy, angles: int = ANGLES_CUMULATIVE) -> dict:
    """The whole method in the paper's order: extremes, polygon, survivors, hull of survivors."""
    a = _pts(xy)
    n = a.shape[0]
    ext = np.full(16, -1, dtype=np.int64)
    m = np.zeros(1, dtype=np.int32)
    pxy = np.zeros(32, dtype=np.int32)
    surv = np.empty(max(n, 1), dtype=np.int64)
    ns = np.zeros(1, dtype=np.int64)
    hl = np.empty(max(n, 1), dtype=np.int64)
    nh = np.zeros(1, dtype=np.int64)
    _get().oracle_cudapre(a.ctypes.data, n, angles, ext.ctypes.data, m.ctypes.data, pxy.ctypes.data,
                          surv.ctypes.data, ns.ctypes.data, hl.ctypes.data, nh.ctypes.data)
    mm = int(m[0])
    return {
        "extremes": ext,
        "poly_xy": pxy[: 2 * mm].reshape(mm, 2).copy(),
        "survivors": surv[: int(ns[0])].copy(),
        "hull": hl[: int(nh[0])].copy(),
    }


def cudapre_mt(xy, angles: int = ANGLES_CUMULATIVE, threads: int = 0) -> tuple[dict, int]:
    """cudapre() with the point loops split over host threads (0: all
    hardware threads); returns (the same dict as cudapre, threads used)."""
    a = _pts(xy)
    n = a.shape[0]
    ext = np.full(16, -1, dtype=np.int64)
    m = np.zeros(1, dtype=np.int32)
    pxy = np.zeros(32, dtype=np.int32)
    surv = np.empty(max(n, 1), dtype=np.int64)
    ns = np.zeros(1, dtype=np.int64)
    hl = np.empty(max(n, 1), dtype=np.int64)
    nh = np.zeros(1, dtype=np.int64)
    t = _get().oracle_cudapre_mt(a.ctypes.data, n, angles, int(threads), ext.ctypes.data, m.ctypes.data,
                                 pxy.ctypes.data, surv.ctypes.data, ns.ctypes.data, hl.ctypes.data, nh.ctypes.data)
    mm = int(m[0])
    return ({"extremes": ext, "poly_xy": pxy[: 2 * mm].reshape(mm, 2).copy(),
             "survivors": surv[: int(ns[0])].copy(), "hull": hl[: int(nh[0])].copy()}, int(t))


# ---- the 3D extension (section 5) -------------------------------------------

def _pts3(xyz) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(xyz, dtype=np.float32).reshape(-1, 3))


def extremes3(xyz, angles: int = ANGLES_CUMULATIVE) -> np.ndarray:
    """24 extreme indices: slot 6g + {0..5} = argmin/argmax of x', y', z' of rotation group g (about z)."""
    a = _pts3(xyz)
    out = np.full(24, -1, dtype=np.int64)
    _get().oracle3_extremes(a.ctypes.data, a.shape[0], angles, out.ctypes.data)
    return out


def facets3(xyz, ext_idx, max_planes: int = 256) -> np.ndarray:
    """Facet planes [m, 4] (Nx, Ny, Nz, d; N.p <= d on the polyhedron, reduced, sorted)."""
    a = _pts3(xyz)
    e = np.ascontiguousarray(np.asarray(ext_idx, dtype=np.int64))
    out = np.zeros(4 * max_planes, dtype=np.int64)
    m = _get().oracle3_facets(a.ctypes.data, e.ctypes.data, e.shape[0], out.ctypes.data, max_planes)
    if m < 0:
        raise ValueError("more facets than max_planes")
    return out[:4 * m].reshape(m, 4).copy()


def prefilter3(xyz, planes) -> np.ndarray:
    """Ascending indices of the points not strictly inside the polyhedron."""
    a = _pts3(xyz)
    p = np.ascontiguousarray(np.asarray(planes, dtype=np.int64).reshape(-1, 4))
    out = np.empty(max(a.shape[0], 1), dtype=np.int64)
    c = _get().oracle3_prefilter(a.ctypes.data, a.shape[0], p.ctypes.data, p.shape[0], out.ctypes.data)
    return out[:c].copy()


def check_domain3(xyz) -> bool:
    a = _pts3(xyz)
    return bool(_get().oracle3_check_domain(a.ctypes.data, a.shape[0]))


def cudapre3(xyz, angles: int = ANGLES_CUMULATIVE) -> dict:
    """The 3D extension in order: extremes, polyhedron, survivors."""
    ext = extremes3(xyz, angles)
    planes = facets3(xyz, ext) if _pts3(xyz).shape[0] else np.zeros((0, 4), np.int64)
    return {"extremes": ext, "planes": planes, "survivors": prefilter3(xyz, planes)}
