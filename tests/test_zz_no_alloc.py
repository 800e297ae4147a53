"""hull_compute_static: the whole method on the library's fixed per-device
workspace, called through the C ABI and compared with hull_compute.

Collected last (file name), so it runs both alone and after every other test
of the session.  Two calls in a row on different inputs, with no
synchronisation between them, must each match hull_compute bit for bit; the
second also shows that the counters left by the first are cleared.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth

HULL_ERR_INVALID_ARG = 1
HULL_ERR_BUDGET = 6


@pytest.fixture(scope="module")
def lib():
    from paper_1405_3454_gb300 import _build
    import paper_1405_3454_gb300 as cp
    _build.build()
    return cp


def test_static_limit_and_rejections(lib):
    # no CUDA call is made on these paths
    cp = lib
    assert cp.HULL_STATIC_MAX_POINTS == 1 << 20
    assert cp.hull_workspace_bytes(cp.HULL_STATIC_MAX_POINTS) <= 26 << 20
    P = 256 * 1024
    assert cp.hull_compute_static(P, cp.HULL_STATIC_MAX_POINTS + 1, P, P, None, 0) == HULL_ERR_BUDGET
    assert cp.hull_compute_static(P, 1 << 28, P, P, None, 0) == HULL_ERR_BUDGET
    assert cp.hull_compute_static(P, -1, P, P, None, 0) == HULL_ERR_INVALID_ARG


def inputs():
    n_max = 1 << 20
    a = synth.disk(n_max, synth.BASE_SEED + 71)          # the largest accepted set
    b = synth.square(100_003, synth.BASE_SEED + 72)      # ragged size
    c = synth.gaussian(65_537, synth.BASE_SEED + 73)
    return [a, b, c]


def reference_hulls(cp, sets, opt):
    import torch
    outs = []
    for xy in sets:
        d = torch.from_numpy(np.ascontiguousarray(xy)).cuda()
        out, cnt, _ = cp.compute(d, opt)
        torch.cuda.synchronize()
        outs.append(cp.as_index(out, int(cnt.item())).tolist())
    return outs


@pytest.mark.gpu
@pytest.mark.parametrize("filt", [1, 0])
def test_static_matches_hull_compute(gpu_lib, filt):
    import torch
    cp = gpu_lib
    opt = cp.Options(filter=filt)
    sets = inputs()
    want = reference_hulls(cp, sets, opt)
    # the first set also against the oracle
    assert want[0] == oracle.cudapre(sets[0])["hull"].tolist()
    dev = [torch.from_numpy(np.ascontiguousarray(xy)).cuda() for xy in sets]
    outs = [torch.full((xy.shape[0],), -1, dtype=torch.int32, device="cuda") for xy in sets]
    cnts = [torch.full((1,), -1, dtype=torch.int64, device="cuda") for _ in sets]
    stream = torch.cuda.current_stream().cuda_stream
    torch.cuda.synchronize()
    # first call: set-up of the workspace address on this device
    assert cp.hull_compute_static(dev[0].data_ptr(), sets[0].shape[0], outs[0].data_ptr(), cnts[0].data_ptr(),
                                  opt, stream) == 0
    torch.cuda.synchronize()
    assert cp.as_index(outs[0], int(cnts[0].item())).tolist() == want[0]
    alloc0 = torch.cuda.memory_allocated()
    free0 = torch.cuda.mem_get_info()[0]
    # two calls in a row on one stream, no synchronisation between them
    for k in (1, 2):
        rc = cp.hull_compute_static(dev[k].data_ptr(), sets[k].shape[0], outs[k].data_ptr(), cnts[k].data_ptr(),
                                    opt, stream)
        assert rc == 0, cp.strerror(rc)
    torch.cuda.synchronize()
    for k in (1, 2):
        assert cp.as_index(outs[k], int(cnts[k].item())).tolist() == want[k], k
    # the calls allocated nothing, from torch or from the device
    assert torch.cuda.memory_allocated() == alloc0
    assert torch.cuda.mem_get_info()[0] == free0


@pytest.mark.gpu
def test_static_empty_and_tiny(gpu_lib):
    import torch
    cp = gpu_lib
    out = torch.full((4,), -1, dtype=torch.int32, device="cuda")
    cnt = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    xy = torch.zeros((1, 2), dtype=torch.float32, device="cuda")
    assert cp.hull_compute_static(xy.data_ptr(), 0, out.data_ptr(), cnt.data_ptr(), None, stream) == 0
    torch.cuda.synchronize()
    assert int(cnt.item()) == 0
    tri = np.array([[0, 0], [5, 0], [0, 5], [1, 1]], dtype=np.float32)
    d = torch.from_numpy(tri).cuda()
    assert cp.hull_compute_static(d.data_ptr(), 4, out.data_ptr(), cnt.data_ptr(), None, stream) == 0
    torch.cuda.synchronize()
    assert cp.as_index(out, int(cnt.item())).tolist() == oracle.cudapre(tri)["hull"].tolist() == [0, 1, 2]
