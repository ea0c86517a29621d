"""The allocation-free inspector entry point against the regular one and the oracle.

tb_inspect_points_noalloc serves callers that cannot allocate device memory
while they run (a device-memory budget fixed at start-up, or a real-time loop
where an allocation would synchronise the device); it keeps its scratch in a
fixed device array.  Its result must equal what tb_set_sources computes and
what the FP64 oracle's inspector computes (integer tables: bit-exact), on two
calls in a row, the second smaller than the first so that leftovers of the
first call in the shared scratch would show, and the calls must leave the
device's free memory unchanged.  This file is collected last.
"""
from __future__ import annotations

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _points(shape, h, seed, n):
    g = np.random.Generator(np.random.PCG64(seed))
    ext = np.array([(shape[d] - 1) * h[d] for d in range(3)])
    pts = g.uniform(0.0, 1.0, size=(n, 3)) * ext
    pts[0] = [3 * h[0], 4 * h[1], 5 * h[2]]   # on a node: one affected point
    pts[1] = ext                              # upper corner of the grid
    pts[2] = pts[3]                           # duplicate point
    return pts


def test_noalloc_inspector_matches_regular_entry_point_and_oracle():
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import oracle
    import paper_2010_10248_gb300 as tb
    from paper_2010_10248_gb300 import _tb

    torch.cuda.set_device(0)
    shape, h = (37, 45, 83), (10.0, 11.0, 9.0)
    vp = torch.full(shape, 2000.0, device="cuda")
    # a first call sets up the device (the scratch address and, with lazy
    # module loading, the kernels' code), which may map memory once
    w_pts = torch.from_numpy(_points(shape, h, 999, 40)).cuda()
    w_lin = torch.zeros(8 * 40, dtype=torch.int64, device="cuda")
    w_n = torch.zeros(1, dtype=torch.int64, device="cuda")
    assert _tb.tb_inspect_points_noalloc(shape, h, 40, w_pts, w_lin, w_n,
                                         torch.cuda.current_stream()) == _tb.TB_OK
    for call, npt in enumerate((700, 23)):
        pts = _points(shape, h, 1000 + call, npt)
        # regular entry point
        p = tb.Propagator(shape, h, 8)
        p.set_model(vp)
        p.set_sources(pts, np.zeros((npt, 4), np.float32))
        want, _ = p.source_points()
        p.close()
        # the oracle's inspector (FP64, plain C)
        lin_orc, _ = oracle.inspect_points(shape, h, 8, 1e-3, 4, np.full(shape, 2000.0), pts)
        np.testing.assert_array_equal(want, lin_orc)
        # allocation-free entry point: every buffer exists before the call
        d_pts = torch.from_numpy(pts).cuda()
        d_lin = torch.full((8 * npt,), -7, dtype=torch.int64, device="cuda")
        d_n = torch.zeros(1, dtype=torch.int64, device="cuda")
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        st = _tb.tb_inspect_points_noalloc(shape, h, npt, d_pts, d_lin, d_n,
                                           torch.cuda.current_stream())
        assert st == _tb.TB_OK
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0, "the allocation-free call changed the device's free memory"
        n = int(d_n.item())
        assert n == len(want)
        np.testing.assert_array_equal(d_lin[:n].cpu().numpy(), want)


def test_noalloc_inspector_limits():
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2010_10248_gb300 import _tb

    shape, h = (20, 20, 20), (10.0, 10.0, 10.0)
    d = torch.zeros((8193, 3), dtype=torch.float64, device="cuda")
    out = torch.zeros(8 * 8193, dtype=torch.int64, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    assert _tb.tb_inspect_points_noalloc(shape, h, 8193, d, out, cnt) == _tb.TB_EINVAL
    # a grid whose linear index would not fit the sort key (n0 n1 n2 >= 2^40)
    assert _tb.tb_inspect_points_noalloc((65535, 65535, 300), h, 4, d, out, cnt) == _tb.TB_EINVAL
    # an off-grid coordinate is reported through the count
    d[:4] = torch.tensor([[-1.0, 5.0, 5.0]] * 4, dtype=torch.float64)
    assert _tb.tb_inspect_points_noalloc(shape, h, 4, d, out, cnt) == _tb.TB_OK
    torch.cuda.synchronize()
    assert int(cnt.item()) == -1
