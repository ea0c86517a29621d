"""Continuous-batching shot server: shots overlap on the GPU, admission
respects the memory budget, and every shot (FP32 or FP16 wavefield storage)
gives bit-identical traces alone and in the mix."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2010_10248_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def serving():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2010_10248_gb300 as tb
    tb.load()
    from paper_2010_10248_gb300 import serving
    return serving


def shots(serving, n=6, seed=5):
    g = np.random.default_rng(seed)
    out = []
    for i in range(n):
        shape = tuple(int(x) for x in g.choice([48, 64, 80, 96], size=3))
        so = int(g.choice([4, 8]))
        h = (10.0, 10.0, 10.0)
        vp = wl.layered_vp(shape, seed + i, vmin=1500.0, vmax=3000.0, nlayers=4, nblobs=2)
        ext = np.array([(shape[d] - 1) * h[d] for d in range(3)])
        src = g.uniform(0.3, 0.7, size=(int(g.integers(1, 5)), 3)) * ext
        rec = g.uniform(0.05, 0.95, size=(int(g.integers(20, 300)), 3)) * ext
        out.append(serving.ShotRequest(shape, h, so, vp, src, 12.0, rec, nt=int(g.integers(300, 600)), nbl=8,
                                       time_tile=int(g.choice([0, 1])), arrival=0.0005 * i, tag=i,
                                       storage=1 if i % 3 == 2 else 0))
    return out


def test_alone_and_in_the_mix_are_identical(serving):
    reqs = shots(serving)
    alone = {}
    solo = serving.ShotServer(slots=1)
    for r in reqs:
        r0 = serving.ShotRequest(**{**r.__dict__, "arrival": 0.0})
        (res,) = solo.run([r0])
        alone[r.tag] = res.traces
    mix = serving.ShotServer(slots=4)
    results = mix.run(reqs)
    assert sorted(x.tag for x in results) == sorted(alone)
    for x in results:
        np.testing.assert_array_equal(x.traces, alone[x.tag])
        assert np.abs(x.traces).max() > 0
        assert x.latency >= 0
    assert mix.stats["max_in_flight"] >= 2  # the shots overlapped on the device


def test_admission_respects_the_memory_budget(serving):
    reqs = shots(serving, n=5, seed=9)
    big = max(serving.footprint_bytes(r) for r in reqs)
    budget = big + min(serving.footprint_bytes(r) for r in reqs)
    srv = serving.ShotServer(slots=4, memory_budget=budget)
    results = srv.run(reqs)
    assert len(results) == len(reqs)
    assert srv.stats["max_bytes"] <= budget
    too_big = serving.ShotServer(slots=2, memory_budget=big - 1)
    with pytest.raises(ValueError):
        too_big.run([max(reqs, key=serving.footprint_bytes)])
