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
    # small FP32 shots go to batch lanes (one launch per step for all of them)
    mix = serving.ShotServer(slots=4, batch_points=96 ** 3, batch_chunk=16)
    results = mix.run(reqs)
    assert sum(ln["max_shots"] for ln in mix.stats["lanes"].values()) >= 2
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


def test_batched_shots_equal_alone_and_the_oracle(serving):
    """Shots of different grids, lengths and geometries advanced together (one
    launch per step for all of them), admitted at different steps: traces and
    final wavefields bit-identical to each shot's one-step run alone, and the
    first shot within the FP32 bar of the FP64 oracle."""
    import torch

    import oracle
    import paper_2010_10248_gb300 as tb
    g = np.random.default_rng(21)
    cases = []
    for shape, nt in (((40, 48, 70), 37), ((64, 64, 64), 60), ((33, 50, 90), 45)):
        h = (10.0, 10.0, 10.0)
        vp = wl.layered_vp(shape, int(g.integers(1000)), vmin=1600.0, vmax=3200.0, nlayers=3, nblobs=2)
        ext = np.array([(shape[d] - 1) * h[d] for d in range(3)])
        src = g.uniform(0.3, 0.7, size=(2, 3)) * ext
        rec = np.concatenate([g.uniform(0.05, 0.95, size=(50, 3)) * ext, ext[None, :]])
        dt = 0.8 * oracle.cfl_dt_max(8, h, float(vp.max()))
        wav = np.repeat(wl.ricker(25.0, dt, nt, t0=5 * dt)[None, :], 2, axis=0).astype(np.float32)
        cases.append((shape, h, vp, src, rec, dt, wav, nt))

    def prop(c):
        shape, h, vp, src, rec, dt, wav, nt = c
        p = tb.Propagator(shape, h, 8, nbl=6)
        p.set_model(torch.from_numpy(vp).cuda(), dt=dt)
        p.set_sources(src, wav)
        p.set_receivers(rec)
        return p

    alone = []
    for c in cases:
        p = prop(c)
        tr = p.forward(c[7], schedule="onestep").clone()
        alone.append((tr, p.field(0).clone(), p.field(1).clone()))
        p.close()
    st = torch.cuda.current_stream()
    b = tb._tb.Batch(4)
    props = [prop(c) for c in cases]
    outs = [torch.full((c[7], len(c[4])), float("nan"), device="cuda") for c in cases]
    b.add(props[0].h, cases[0][7], outs[0], st)
    b.step(10, st)
    b.add(props[1].h, cases[1][7], outs[1], st)
    b.step(7, st)
    b.add(props[2].h, cases[2][7], outs[2], st)
    done = []
    while b.active():
        b.step(5, st)
        done += b.finished()
    torch.cuda.synchronize()
    assert sorted(done) == sorted(p.h for p in props)
    for p, o, (tr, u0, u1) in zip(props, outs, alone):
        assert torch.equal(o, tr)
        assert torch.equal(p.field(0), u0) and torch.equal(p.field(1), u1)
        assert float(tr.abs().max()) > 0
    shape, h, vp, src, rec, dt, wav, nt = cases[0]
    tr_o, u_o, _ = oracle.acoustic_forward(shape, h, 8, dt, nt, vp.astype(np.float64), nbl=6, src_xyz=src,
                                           src_wav=wav.astype(np.float64), rec_xyz=rec)
    e_tr = np.linalg.norm(outs[0].cpu().numpy() - tr_o) / np.linalg.norm(tr_o)
    e_u = np.linalg.norm(props[0].field(0).cpu().numpy() - u_o) / np.linalg.norm(u_o)
    assert e_tr <= 1e-4 and e_u <= 1e-4, (e_tr, e_u)
    for p in props:
        p.close()
    b.close()


@pytest.mark.parametrize("kind", ["blocked", "onestep", "f16"])
def test_footprint_bounds_the_library_bytes(serving, kind):
    """The admission estimate holds what the library reports for the shot
    (tb_workspace_bytes after its forward) plus the device trace tensor, and
    is not far above it."""
    import torch
    from paper_2010_10248_gb300 import _tb
    g = np.random.default_rng(11)
    shape, h = (80, 64, 96), (10.0, 10.0, 10.0)
    vp = wl.layered_vp(shape, 3, vmin=1500.0, vmax=3000.0, nlayers=4, nblobs=2)
    ext = np.array([(shape[d] - 1) * h[d] for d in range(3)])
    src = g.uniform(0.3, 0.7, size=(3, 3)) * ext
    rec = g.uniform(0.05, 0.95, size=(250, 3)) * ext
    req = serving.ShotRequest(shape, h, 8, vp, src, 12.0, rec, nt=200, nbl=8,
                              time_tile=0 if kind == "blocked" else 1, storage=1 if kind == "f16" else 0)
    st = torch.cuda.current_stream()
    p, dt, keep = serving._setup(torch, req, st, req.time_tile if req.storage == 0 else 1)
    tr = torch.empty((req.nt, len(rec)), dtype=torch.float32, device="cuda")
    _tb.tb_forward(p.h, req.nt, tr, _tb.TB_BLOCKED if kind == "blocked" else _tb.TB_ONESTEP, st)
    torch.cuda.synchronize()
    used = p.workspace_bytes() + 4 * tr.numel()
    est = serving.footprint_bytes(req)
    print(f"{kind}: library {used / 2**20:.1f} MiB, estimate {est / 2**20:.1f} MiB")
    assert used <= est <= 1.3 * used + (16 << 20)
    p.close()


_ALLOC_PROBE = """
import json, sys, torch
import paper_2010_10248_gb300 as tb
tb.load()
opt = {"f32": {}, "f16": {"storage": tb.TB_F16}, "plain": {"storage": tb.TB_F32_PLAIN},
       "tti": {"physics": tb.TB_TTI}, "elastic": {"physics": tb.TB_ELASTIC}}[sys.argv[1]]
torch.cuda.init()
tb.Propagator((32, 32, 32), (10.0, 10.0, 10.0), 8, **opt).close()  # first-use costs of the allocator
torch.cuda.synchronize()
free0 = torch.cuda.mem_get_info()[0]
p = tb.Propagator((320, 320, 320), (10.0, 10.0, 10.0), 8, **opt)
torch.cuda.synchronize()
free1 = torch.cuda.mem_get_info()[0]
print(json.dumps([free0 - free1, p.workspace_bytes()]))
"""


@pytest.mark.parametrize("kind", ["f32", "f16", "plain", "tti", "elastic"])
def test_workspace_bytes_match_device_allocations(serving, kind):
    """tb_workspace_bytes after tb_create against the drop in free device
    memory around it, in a fresh process (its allocation pool holds only a
    small handle's memory), to the pool's growth granularity."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _ALLOC_PROBE, kind], cwd=root, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    drop, reported = json.loads(r.stdout.strip().splitlines()[-1])
    field = 4 * 320 ** 3
    print(f"{kind}: free memory dropped {drop / 2**20:.1f} MiB, reported {reported / 2**20:.1f} MiB")
    assert reported >= 2 * field  # at least two FP32 wavefields' worth
    assert abs(drop - reported) <= 64 << 20
