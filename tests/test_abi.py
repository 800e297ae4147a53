"""The C-ABI library loads and exports every symbol the header declares.

No compute call here (no GPU needed): only loading, symbol lookup, option
defaults, error strings, workspace sizing and the projection constants.
"""
import ctypes
import os
import re
from decimal import Decimal, getcontext

import pytest

import paper_1405_3454_gb300 as cp
from paper_1405_3454_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return cp.load()


def declared_functions():
    names = set()
    for h in HEADERS:
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z_][a-z0-9_]*)\s*\(", src, re.M):
            names.add(m.group(1))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 10
    for nm in names:
        assert hasattr(lib, nm), nm
    assert set(cp.ABI_SYMBOLS) <= set(names)


def test_defaults_and_strings(lib):
    o = cp.HullOptions()
    lib.hull_default_options(ctypes.byref(o))
    assert o.angles == cp.HULL_ANGLES_CUMULATIVE and o.filter == cp.HULL_FILTER_FP32 and o.validate == 0
    assert o.refine == 1 and ctypes.sizeof(o) == 16 * 4
    for code in range(8):
        assert lib.hull_strerror(code).decode().startswith("HULL_")
    assert lib.hull_abi_version() == 1


def test_workspace_sizes_monotone(lib):
    a = cp.hull_workspace_bytes(1000)
    b = cp.hull_workspace_bytes(1 << 20)
    assert 0 < a < b
    assert cp.hull_prefilter_workspace_bytes(1 << 28) < cp.hull_workspace_bytes(1 << 28)
    # the full pipeline keeps two (u64 key, u32 index) buffers of n entries
    assert cp.hull_workspace_bytes(1 << 28) >= 24 * (1 << 28)


def test_library_constants_are_correctly_rounded(lib):
    getcontext().prec = 60
    s3 = Decimal(3).sqrt() / 2
    s6, s2 = Decimal(6).sqrt(), Decimal(2).sqrt()
    c = cp.constants()
    assert c["s3"] == float(s3)
    assert c["c75"] == float((s6 - s2) / 4)
    assert c["s75"] == float((s6 + s2) / 4)
    assert c["h"] == float(s2 / 2)


def test_argument_errors_without_gpu(lib):
    # invalid arguments are rejected before any CUDA call
    P = 256 * 1024
    assert cp.hull_prefilter(0, 10, P, 1 << 30, P, P, 0, None, 0) == 1      # null xy
    assert cp.hull_prefilter(P + 4, 10, P, 1 << 30, P, P, 0, None, 0) == 1  # misaligned xy
    assert cp.hull_prefilter(P, -1, P, 1 << 30, P, P, 0, None, 0) == 1      # negative n
    assert cp.hull_prefilter(P, 1 << 32, P, 1 << 30, P, P, 0, None, 0) == 1 # n too large
    assert cp.hull_compute(P, 10, P + 8, 1 << 30, P, P, None, 0) == 1       # misaligned workspace
    assert cp.hull_compute(P, 1000, P, 16, P, P, None, 0) == 3               # workspace too small
    o = cp.Options(angles=7)
    assert cp.hull_compute(P, 10, P, 1 << 30, P, P, o, 0) == 7               # unsupported option
    # the no-prefilter comparator is for hull_compute only
    assert cp.hull_prefilter(P, 10, P, 1 << 30, P, P, 0, cp.Options(no_prefilter=True), 0) == 7
    assert cp.hull_batch(P, P, 1, 10, P, 1 << 30, P, P, cp.Options(no_prefilter=True), 0) == 7
    # the timeout self-test checks its workspace and its limit first
    lib_ = cp.load()
    assert lib_.hull_selftest_wait(0, 1000, 0) == 1
    assert lib_.hull_selftest_wait(P + 16, 1000, 0) == 1
    assert lib_.hull_selftest_wait(P, 0, 0) == 1
    assert lib_.hull_selftest_wait(P, (1 << 31) + 1, 0) == 1


def test_compute_workspace_has_room_for_reserved_slots(lib):
    # hull_compute on 2^24 points or more may reserve up to 4096 warps x 256
    # survivor slots beyond n: its workspace holds that many more (key, index)
    # entries in both buffer pairs; hull_prefilter's workspace does not change
    a, b = cp.hull_workspace_bytes((1 << 24) - 1), cp.hull_workspace_bytes(1 << 24)
    assert b - a >= 2 * (8 + 4) * 4096 * 256
    assert cp.hull_prefilter_workspace_bytes(1 << 24) == cp.hull_prefilter_workspace_bytes((1 << 24) - 1)
    # the largest sets do without (survivor positions stay below 2^32)
    top = (1 << 32) - 1
    assert cp.hull_workspace_bytes(top) - cp.hull_workspace_bytes(top - 1) < 64


def test_graph_rejects_the_default_stream_before_any_cuda_call(lib):
    # the legacy default stream cannot be captured: refused up front
    g = lib.hull_graph_create()
    assert g
    P = 256 * 1024
    code = cp.hull_graph_batch_ranges(g, P, 10, 0, P, 1, 10, P, 1 << 20, P, P, None, 0)
    assert code == 1
    counts = (ctypes.c_int64 * 6)()
    lib.hull_graph_counts(g, counts)
    assert list(counts) == [0, 0, 0, 0, 0, 0]
    lib.hull_graph_destroy(g)


def test_static_entry_point_holds_its_largest_set(lib):
    # hull_compute_static runs hull_compute on one fixed 26 MiB array per
    # device: the workspace of its largest set must fit there, and one point
    # more is refused before any CUDA call
    assert cp.hull_workspace_bytes(cp.HULL_STATIC_MAX_POINTS) <= 26 << 20
    P = 256 * 1024
    assert lib.hull_compute_static(P, cp.HULL_STATIC_MAX_POINTS + 1, P, P, None, 0) == 6  # HULL_ERR_BUDGET
