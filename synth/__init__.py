"""Seeded synthetic point sets (float32 xy, integer-valued, |v| <= 2^24).

Input generators only: nothing here computes an extreme point, a hull or an
inside test.  The arrays feed both the CPU oracle and the CUDA path.  The C
source (``synth.c``) is compiled on first use with gcc.

Shapes follow the paper's data groups (section 3): uniform square and uniform
circle (its rbox data) and Gaussian clusters in place of the projected mesh
vertices of Table 3, which are not available.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libsynth.so")
_lib = None

BASE_SEED = 1405345
R24 = 1 << 24


def build(force: bool = False) -> str:
    """Compile libsynth.so next to the source (gcc, OpenMP, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _get():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i64, u64 = ctypes.c_int64, ctypes.c_uint64
        lib.synth_square.argtypes = [P, i64, u64, u64, i64]
        lib.synth_disk.argtypes = [P, i64, u64, u64, i64]
        lib.synth_gaussian.argtypes = [P, i64, u64, u64, ctypes.c_double, i64]
        lib.synth_near_edge.argtypes = [P, i64, u64, u64, P, ctypes.c_int]
        lib.synth_near_edge.restype = ctypes.c_int
        lib.synth_permute.argtypes = [P, P, i64, u64]
        lib.synth_set_plan.argtypes = [i64, u64, ctypes.c_double, ctypes.c_double, P, P]
        lib.synth_mix64.argtypes = [u64]
        lib.synth_mix64.restype = u64
        lib.synth_draw.argtypes = [u64, u64, u64, u64]
        lib.synth_draw.restype = u64
        lib.synth_cube3.argtypes = [P, i64, u64, u64, i64]
        lib.synth_ball3.argtypes = [P, i64, u64, u64, i64]
        lib.synth_gauss3.argtypes = [P, i64, u64, u64, ctypes.c_double, i64]
        _lib = lib
    return _lib


def _out(n: int, out=None) -> np.ndarray:
    if out is None:
        return np.empty((n, 2), dtype=np.float32)
    assert out.dtype == np.float32 and out.shape == (n, 2) and out.flags.c_contiguous
    return out


def square(n: int, seed: int = BASE_SEED, r: int = 1 << 20, stream: int = 0, out=None) -> np.ndarray:
    """n points uniform on the integer lattice of [-r, r]^2."""
    a = _out(n, out)
    _get().synth_square(a.ctypes.data, n, seed, stream, r)
    return a


def disk(n: int, seed: int = BASE_SEED, r: int = R24, stream: int = 1, out=None) -> np.ndarray:
    """n lattice points uniform in the disk x^2 + y^2 <= r^2."""
    a = _out(n, out)
    _get().synth_disk(a.ctypes.data, n, seed, stream, r)
    return a


def gaussian(n: int, seed: int = BASE_SEED, sigma: float = float(1 << 22), clip: int = R24,
             stream: int = 2, out=None) -> np.ndarray:
    """n integer-valued Gaussian points (sigma per axis), clipped to [-clip, clip]."""
    a = _out(n, out)
    _get().synth_gaussian(a.ctypes.data, n, seed, stream, float(sigma), clip)
    return a


def near_edge(n: int, poly_xy: np.ndarray, seed: int = BASE_SEED, stream: int = 3, out=None) -> np.ndarray:
    """n points on, or within one unit inside of, the edges of a CCW polygon."""
    poly = np.ascontiguousarray(np.asarray(poly_xy, dtype=np.int32).reshape(-1, 2))
    a = _out(n, out)
    ok = _get().synth_near_edge(a.ctypes.data, n, seed, stream, poly.ctypes.data, poly.shape[0])
    if not ok:
        raise ValueError("near_edge needs a polygon with at least 3 vertices")
    return a


def permute(xy: np.ndarray, seed: int = BASE_SEED) -> np.ndarray:
    """Seeded affine permutation of the points (a cheap invertible shuffle)."""
    xy = np.ascontiguousarray(xy, dtype=np.float32)
    out = np.empty_like(xy)
    _get().synth_permute(xy.ctypes.data, out.ctypes.data, xy.shape[0], seed)
    return out


def interleave(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Even indices from a, odd indices from b (len(a) == len(b) or len(a) == len(b) + 1).

    Both inputs keep their relative order, so lowest-index tie-breaking among
    the points of `a` is unchanged."""
    assert len(a) - len(b) in (0, 1)
    out = np.empty((len(a) + len(b), 2), dtype=np.float32)
    out[0::2] = a
    out[1::2] = b
    return out


def near_edge_mix(n: int, seed: int, polygon_of) -> tuple[np.ndarray, np.ndarray]:
    """The FP32-escalation workload: n points, half integer-valued Gaussian
    (sigma 2^22, clipped to +-2^24) at even indices, half on or within one unit
    inside the edges of the Gaussian half's Step-2 polygon at odd indices.
    `polygon_of(xy) -> [m, 2] int` supplies that polygon (the generator
    computes no polygon itself).  Returns (xy, polygon)."""
    g = gaussian(n - n // 2, seed, stream=40)
    poly = np.asarray(polygon_of(g), dtype=np.int32).reshape(-1, 2)
    ne = near_edge(n // 2, poly, seed, stream=41)
    return interleave(g, ne), poly


def shape(kind: int, n: int, seed: int, stream: int, out=None) -> np.ndarray:
    """Shape id 0 = square r=2^24, 1 = disk r=2^24, 2 = Gaussian sigma=2^22 clipped at 2^24."""
    if kind == 0:
        return square(n, seed, R24, stream, out)
    if kind == 1:
        return disk(n, seed, R24, stream, out)
    return gaussian(n, seed, float(1 << 22), R24, stream, out)


def set_plan(s: int, seed: int = BASE_SEED, lo: float = 1e3, hi: float = 4e6):
    """Sizes floor(exp(U(ln lo, ln hi))) and shape ids for s independent sets."""
    sizes = np.empty(s, dtype=np.int64)
    shapes = np.empty(s, dtype=np.int32)
    _get().synth_set_plan(s, seed, float(lo), float(hi), sizes.ctypes.data, shapes.ctypes.data)
    return sizes, shapes


def batch(s: int, seed: int = BASE_SEED, lo: float = 1e3, hi: float = 4e6, out=None):
    """Concatenated point sets of the batched workload.

    Returns (xy [N, 2] float32, offsets [s + 1] int64, shapes [s] int32).
    Set k is shape(shapes[k]) with its own stream, so any set can be
    regenerated alone.
    """
    sizes, shapes = set_plan(s, seed, lo, hi)
    offsets = np.zeros(s + 1, dtype=np.int64)
    np.cumsum(sizes, out=offsets[1:])
    total = int(offsets[-1])
    xy = _out(total, out)
    for k in range(s):
        shape(int(shapes[k]), int(sizes[k]), seed, 1000 + k, out=xy[offsets[k]:offsets[k + 1]])
    return xy, offsets, shapes


def one_set(k: int, s: int, seed: int = BASE_SEED, lo: float = 1e3, hi: float = 4e6) -> np.ndarray:
    """Set k of batch(s, seed, lo, hi), generated alone."""
    sizes, shapes = set_plan(s, seed, lo, hi)
    return shape(int(shapes[k]), int(sizes[k]), seed, 1000 + k)


def mix64(z: int) -> int:
    return int(_get().synth_mix64(z & 0xFFFFFFFFFFFFFFFF))


def draw(seed: int, stream: int, i: int, k: int) -> int:
    return int(_get().synth_draw(seed, stream, i, k))


def _unit(seed: int, stream: int, i: int, k: int) -> float:
    """U(0, 1) from one counter-based draw (53 bits, never 0)."""
    return ((draw(seed, stream, i, k) >> 11) + 0.5) * 2.0 ** -53


def serving_pool(per_decile: int, seed: int = BASE_SEED, lo: float = 1e4, hi: float = 1.6e7):
    """The dataset pool of the serving workload: per_decile sets in each of
    the 10 log-size deciles of [lo, hi) (size floor(exp(U)) within its
    decile, shape drawn per set as in the batched workload), concatenated.
    Returns (xy [N, 2] float32, starts [K] int64, sizes [K] int64, shapes [K])."""
    k_sets = 10 * per_decile
    a, b = np.log(lo), np.log(hi)
    sizes = np.empty(k_sets, np.int64)
    shapes = np.empty(k_sets, np.int32)
    for j in range(k_sets):
        d = j // per_decile
        u = _unit(seed, 60, j, 0)
        sizes[j] = int(np.floor(np.exp(a + (b - a) * (d + u) / 10.0)))
        shapes[j] = int(draw(seed, 61, j, 0) % 3)
    starts = np.zeros(k_sets, np.int64)
    np.cumsum(sizes[:-1], out=starts[1:])
    xy = _out(int(sizes.sum()))
    for j in range(k_sets):
        shape(int(shapes[j]), int(sizes[j]), seed, 2000 + j, out=xy[starts[j]:starts[j] + sizes[j]])
    return xy, starts, sizes, shapes


def serving_requests(n: int, k_sets: int, seed: int = BASE_SEED):
    """n requests over a pool of k_sets sets: the set of each request
    (uniform, so request sizes follow the pool's log-uniform deciles) and
    unit-rate Poisson arrival times (divide by the rate to scale).
    Returns (set index [n] int64, arrival [n] float64)."""
    sets = np.fromiter((draw(seed, 62, r, 0) % k_sets for r in range(n)), dtype=np.int64, count=n)
    gaps = np.fromiter((-np.log(_unit(seed, 63, r, 0)) for r in range(n)), dtype=np.float64, count=n)
    return sets, np.cumsum(gaps)


# ---- 3D point sets (float32 xyz [n][3], integer-valued, |v| <= 2^19) -------

R19 = 1 << 19


def _out3(n: int, out=None) -> np.ndarray:
    if out is None:
        return np.empty((n, 3), dtype=np.float32)
    assert out.dtype == np.float32 and out.shape == (n, 3) and out.flags.c_contiguous
    return out


def cube3(n: int, seed: int = BASE_SEED, r: int = R19, stream: int = 0, out=None) -> np.ndarray:
    """Uniform integer points in [-r, r]^3."""
    a = _out3(n, out)
    _get().synth_cube3(a.ctypes.data, n, seed, stream, r)
    return a


def ball3(n: int, seed: int = BASE_SEED, r: int = R19, stream: int = 0, out=None) -> np.ndarray:
    """Uniform integer points in the ball of radius r (indexed rejection)."""
    a = _out3(n, out)
    _get().synth_ball3(a.ctypes.data, n, seed, stream, r)
    return a


def gauss3(n: int, seed: int = BASE_SEED, sigma: float = float(1 << 17), clip: int = R19, stream: int = 0,
           out=None) -> np.ndarray:
    """Integer-valued Gaussian points, sigma per axis, clipped to [-clip, clip]."""
    a = _out3(n, out)
    _get().synth_gauss3(a.ctypes.data, n, seed, stream, float(sigma), clip)
    return a


def shape3(kind: int, n: int, seed: int, stream: int = 0) -> np.ndarray:
    """3D shape id 0 = cube r=2^19, 1 = ball r=2^19, 2 = Gaussian sigma=2^17 clipped at 2^19."""
    return (cube3, ball3, gauss3)[kind](n, seed, stream=stream)
