"""GPU parity of the TTI (Sec. III-B, Eq. 2) and elastic (Sec. III-C, Eq. 3)
propagators against the FP64 oracle, through the C ABI: one step per launch,
and the temporally blocked wavefront (Sec. II-B, Fig. 7b), which must equal
the one-step path bit for bit.

Tolerance: rel-L2 <= 1e-4 on receiver traces and wavefields (FP32 against
FP64), as for the acoustic path."""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from paper_2010_10248_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = 1e-4


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def tb():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2010_10248_gb300 as tb
    tb.load()
    return tb


def geometry(shape, h, seed, nrec=24):
    g = np.random.default_rng(seed)
    ext = np.array([(shape[d] - 1) * h[d] for d in range(3)])
    src = (g.uniform(0.35, 0.65, size=(1, 3)) * ext)
    rec = g.uniform(0.1, 0.9, size=(nrec, 3)) * ext
    rec[:4, 0] = 0.0            # receivers on the low faces
    rec[4:6, 2] = ext[2]        # and on the high face (upper-edge clamp)
    return src, rec


def tti_case(shape, so, seed, nt):
    h = (12.0, 10.0, 11.0)
    vp = wl.layered_vp(shape, seed, vmin=1500.0, vmax=2500.0, nlayers=4, nblobs=4)
    eps = wl.smooth_field(shape, seed + 1, 0.05, 0.3)
    delta = np.minimum(wl.smooth_field(shape, seed + 2, 0.0, 0.2), eps)
    theta = wl.smooth_field(shape, seed + 3, 0.0, math.pi / 4)
    phi = wl.smooth_field(shape, seed + 4, -0.3, math.pi / 4)
    src, rec = geometry(shape, h, seed + 5)
    return h, vp, (eps, delta, theta, phi), src, rec


@pytest.mark.parametrize("schedule", ["onestep", "blocked"])
@pytest.mark.parametrize("shape,so,nt", [((30, 33, 40), 4, 70), ((28, 31, 37), 8, 60),
                                         ((30, 29, 35), 12, 40)])
def test_tti_matches_oracle(tb, shape, so, nt, schedule):
    import torch
    h, vp, aux, src, rec = tti_case(shape, so, 101 + so, nt)
    p = tb.Propagator(shape, h, so, physics=tb.TB_TTI, nbl=5, time_tile=3, slab_planes=so)
    p.set_model(torch.from_numpy(vp).cuda(), aux=np.stack(aux))
    dt = p.dt
    assert dt == pytest.approx(0.8 * oracle.tti_dt_max(so, h, float(vp.max()), float(aux[0].max())),
                               rel=1e-5)
    wav = wl.ricker(30.0, dt, nt, t0=8 * dt)[None, :].astype(np.float32)
    p.set_sources(src, wav)
    p.set_receivers(rec)
    tr = p.forward(nt, schedule=schedule).cpu().numpy()
    tr_o, st_o = oracle.tti_forward(shape, h, so, dt, nt, vp.astype(np.float64),
                                    *[a.astype(np.float64) for a in aux], nbl=5,
                                    src_xyz=src, src_wav=wav.astype(np.float64), rec_xyz=rec)
    e_tr = rel_l2(tr, tr_o)
    fields = [p.field(i).cpu().numpy() for i in range(4)]
    e_f = [rel_l2(f, st_o[i]) for i, f in enumerate(fields)]
    print(f"TTI so{so} {schedule}: traces rel-L2 {e_tr:.2e}, fields {[f'{x:.1e}' for x in e_f]}")
    assert np.abs(tr_o).max() > 0
    assert e_tr <= TOL
    assert max(e_f) <= TOL


def elastic_case(shape, so, seed):
    h = (10.0, 11.0, 9.0)
    vp = wl.layered_vp(shape, seed, vmin=2000.0, vmax=3500.0, nlayers=4, nblobs=4)
    vs = (vp / wl.smooth_field(shape, seed + 1, 1.6, 2.0)).astype(np.float32)
    rho = wl.smooth_field(shape, seed + 2, 1.0, 2.5)
    src, rec = geometry(shape, h, seed + 5)
    return h, vp, (vs, rho), src, rec


@pytest.mark.parametrize("schedule", ["onestep", "blocked"])
@pytest.mark.parametrize("shape,so,nt", [((30, 33, 40), 4, 70), ((28, 31, 37), 8, 60),
                                         ((30, 29, 35), 12, 40)])
def test_elastic_matches_oracle(tb, shape, so, nt, schedule):
    import torch
    h, vp, aux, src, rec = elastic_case(shape, so, 201 + so)
    p = tb.Propagator(shape, h, so, physics=tb.TB_ELASTIC, nbl=5, time_tile=3, slab_planes=so // 2)
    p.set_model(torch.from_numpy(vp).cuda(), aux=np.stack(aux))
    dt = p.dt
    assert dt == pytest.approx(0.8 * oracle.elastic_dt_max(so, h, float(vp.max())), rel=1e-9)
    wav = wl.ricker(40.0, dt, nt, t0=8 * dt)[None, :].astype(np.float32)
    p.set_sources(src, wav)
    p.set_receivers(rec)
    tr = p.forward(nt, schedule=schedule).cpu().numpy()
    tr_o, st_o = oracle.elastic_forward(shape, h, so, dt, nt, vp.astype(np.float64),
                                        *[a.astype(np.float64) for a in aux], nbl=5, src_xyz=src,
                                        src_wav=wav.astype(np.float64), rec_xyz=rec)
    e_tr = rel_l2(tr, tr_o)
    e_f = [rel_l2(p.field(i).cpu().numpy(), st_o[i]) for i in range(9)]
    print(f"elastic so{so} {schedule}: traces rel-L2 {e_tr:.2e}, fields {[f'{x:.1e}' for x in e_f]}")
    assert np.abs(tr_o).max() > 0
    assert e_tr <= TOL
    assert max(e_f) <= TOL


def _run(tb, physics, case, so, nt, schedule, **opt):
    import torch
    h, vp, aux, src, rec = case
    p = tb.Propagator(vp.shape, h, so, physics=physics, nbl=4, **opt)
    p.set_model(torch.from_numpy(vp).cuda(), aux=np.stack(aux))
    wav = np.stack([wl.ricker(f, p.dt, nt, t0=(6 + i) * p.dt) for i, f in enumerate((35.0, 25.0, 45.0))])
    g = np.random.default_rng(so + nt)
    ext = np.array([(vp.shape[d] - 1) * h[d] for d in range(3)])
    srcs = np.concatenate([src, g.uniform(0.05, 0.95, size=(2, 3)) * ext])
    srcs[1, 0] = 0.0      # a source on the first plane
    srcs[2, 0] = ext[0]   # and one on the last
    p.set_sources(srcs, wav.astype(np.float32))
    p.set_receivers(rec)
    tr = p.forward(nt, schedule=schedule).cpu().numpy()
    nf = 4 if physics == tb.TB_TTI else 9
    return tr, [p.field(i).cpu().numpy() for i in range(nf)]


@pytest.mark.parametrize("physics", ["tti", "tti_l1", "tti_fused", "elastic", "elastic_l1"])
@pytest.mark.parametrize("shape,so,T,slab,nt", [((30, 33, 40), 4, 2, 0, 23), ((37, 31, 36), 8, 3, 4, 20),
                                                ((29, 33, 35), 8, 2, 5, 17), ((41, 29, 35), 12, 2, 6, 15),
                                                ((33, 30, 34), 4, 8, 3, 19), ((19, 30, 34), 8, 4, 0, 13),
                                                ((70, 28, 33), 4, 16, 2, 37)])
def test_blocked_bitwise_equals_onestep(tb, physics, shape, so, T, slab, nt):
    """Ragged slabs (n0 not a multiple of the slab), nt not a multiple of T
    (the rest one step per launch), sources on the first and last planes.
    The fused TTI step reaches 2r planes, so its slabs are at least so."""
    ela = physics.startswith("elastic")
    phys = tb.TB_ELASTIC if ela else tb.TB_TTI
    opt = dict(tti_fused=physics == "tti_fused", stream_l1=physics.endswith("_l1"))
    if opt["tti_fused"] and slab:
        slab = max(slab, so)
    case = (elastic_case(shape, so, 400 + so) if ela else tti_case(shape, so, 300 + so, nt))
    ref_tr, ref_f = _run(tb, phys, case, so, nt, "onestep", **opt)
    got_tr, got_f = _run(tb, phys, case, so, nt, "blocked", time_tile=T, slab_planes=slab, **opt)
    assert np.abs(ref_tr).max() > 0
    assert np.array_equal(got_tr, ref_tr)
    for a, b in zip(got_f, ref_f):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("shape,so", [((30, 33, 40), 4), ((70, 19, 71), 8), ((45, 26, 33), 12), ((96, 40, 66), 8)])
def test_tti_fused_step_equals_two_pass(tb, shape, so):
    """The fused TTI step (fluxes on chip, tiles of 8 x 32 columns, chunks
    along axis 0) against the flux and update kernels: traces and fields bit
    for bit, on grids with ragged tiles and several chunks."""
    nt = 21
    case = tti_case(shape, so, 500 + so, nt)
    ref_tr, ref_f = _run(tb, tb.TB_TTI, case, so, nt, "onestep")
    got_tr, got_f = _run(tb, tb.TB_TTI, case, so, nt, "onestep", tti_fused=True)
    assert np.abs(ref_tr).max() > 0
    assert np.array_equal(got_tr, ref_tr)
    for a, b in zip(got_f, ref_f):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("shape,so", [((30, 33, 40), 4), ((70, 19, 71), 8), ((45, 26, 33), 12), ((96, 40, 66), 8)])
def test_elastic_tma_equals_l1(tb, shape, so):
    """The TMA-staged elastic updates (8 x 32 tiles, chunks along axis 0,
    halos and out-of-grid cells filled by the copy engine) against the L1
    streaming kernels: traces and every field bit for bit, on grids with
    ragged tiles and several chunks."""
    nt = 21
    case = elastic_case(shape, so, 600 + so)
    ref_tr, ref_f = _run(tb, tb.TB_ELASTIC, case, so, nt, "onestep", stream_l1=True)
    got_tr, got_f = _run(tb, tb.TB_ELASTIC, case, so, nt, "onestep")
    assert np.abs(ref_tr).max() > 0
    assert np.array_equal(got_tr, ref_tr)
    for a, b in zip(got_f, ref_f):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("shape,so", [((30, 33, 40), 4), ((70, 19, 71), 8), ((45, 26, 33), 12), ((96, 40, 66), 8)])
def test_tti_tma_equals_l1(tb, shape, so):
    """The TMA-staged TTI passes against the L1 streaming kernels: traces and
    every field bit for bit, ragged tiles and several chunks."""
    nt = 21
    case = tti_case(shape, so, 700 + so, nt)
    ref_tr, ref_f = _run(tb, tb.TB_TTI, case, so, nt, "onestep", stream_l1=True)
    got_tr, got_f = _run(tb, tb.TB_TTI, case, so, nt, "onestep")
    assert np.abs(ref_tr).max() > 0
    assert np.array_equal(got_tr, ref_tr)
    for a, b in zip(got_f, ref_f):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("physics", ["tti", "elastic"])
@pytest.mark.parametrize("shape,so", [((6, 7, 8), 4), ((10, 10, 10), 8), ((14, 15, 14), 12), ((40, 10, 70), 8)])
def test_smallest_grids_all_paths_agree(tb, physics, shape, so):
    """Grids at the minimum size (n = so + 2) and thinner than one tile: the
    TMA boxes reach past every edge (zeros from the copy engine).  TMA-staged
    one-step and blocked, and the L1 streaming kernels, agree bit for bit, and
    with the oracle within 1e-4."""
    nt = 9
    phys = tb.TB_TTI if physics == "tti" else tb.TB_ELASTIC
    case = tti_case(shape, so, 800 + so, nt) if physics == "tti" else elastic_case(shape, so, 900 + so)
    h, vp, aux, src, rec = case
    ref_tr, ref_f = _run(tb, phys, case, so, nt, "onestep", stream_l1=True)
    for sched, opt in [("onestep", {}), ("blocked", dict(time_tile=2, slab_planes=so))]:
        got_tr, got_f = _run(tb, phys, case, so, nt, sched, **opt)
        assert np.array_equal(got_tr, ref_tr), sched
        for a, b in zip(got_f, ref_f):
            assert np.array_equal(a, b), sched
    # the oracle with the same sources (the three of _run) and receivers
    import torch
    p = tb.Propagator(shape, h, so, physics=phys, nbl=4)
    p.set_model(torch.from_numpy(vp).cuda(), aux=np.stack(aux))
    dt = p.dt
    p.close()
    wav = np.stack([wl.ricker(f, dt, nt, t0=(6 + i) * dt) for i, f in enumerate((35.0, 25.0, 45.0))])
    g = np.random.default_rng(so + nt)
    ext = np.array([(shape[d] - 1) * h[d] for d in range(3)])
    srcs = np.concatenate([src, g.uniform(0.05, 0.95, size=(2, 3)) * ext])
    srcs[1, 0] = 0.0
    srcs[2, 0] = ext[0]
    fn = oracle.tti_forward if physics == "tti" else oracle.elastic_forward
    tr_o, _ = fn(shape, h, so, dt, nt, vp.astype(np.float64), *[a.astype(np.float64) for a in aux], nbl=4,
                 src_xyz=srcs, src_wav=wav.astype(np.float32).astype(np.float64), rec_xyz=rec)
    assert rel_l2(ref_tr, tr_o) <= TOL


def test_tti_and_elastic_reject_bad_options_and_models(tb):
    import torch
    shape, h = (20, 20, 20), (10.0, 10.0, 10.0)
    vp = torch.full(shape, 2000.0, device="cuda")
    one = np.ones(shape, dtype=np.float32)
    p = tb.Propagator(shape, h, 4, physics=tb.TB_TTI)
    with pytest.raises(tb.TBError) as e:  # eps < delta
        p.set_model(vp, aux=np.stack([0.05 * one, 0.1 * one, 0 * one, 0 * one]))
    assert e.value.status == 4  # TB_EUNSTABLE
    with pytest.raises(tb.TBError):  # aux required
        p.set_model(vp)
    p.set_model(vp, aux=np.stack([0.2 * one, 0.1 * one, 0 * one, 0 * one]))
    q = tb.Propagator(shape, h, 4, physics=tb.TB_ELASTIC)
    with pytest.raises(tb.TBError):  # vs too large (2 vs^2 > vp^2)
        q.set_model(vp, aux=np.stack([1500.0 * one, one]))
    for opt in [dict(time_tile=17), dict(slab_planes=1), dict(slab_planes=-1)]:
        with pytest.raises(tb.TBError):  # at most 16 fused steps; slabs of at least r planes
            tb.Propagator(shape, h, 4, physics=tb.TB_ELASTIC, **opt)
    with pytest.raises(tb.TBError):  # the fused TTI step reaches 2r planes
        tb.Propagator(shape, h, 8, physics=tb.TB_TTI, slab_planes=7, tti_fused=True)
    tb.Propagator(shape, h, 8, physics=tb.TB_TTI, slab_planes=4).close()


def _subbox_parity(tb, physics, w, nsteps, radius, schedule="onestep"):
    """Full-size run in the benchmark's configuration (same kernels and
    launch shapes) for nsteps; the oracle runs on the sub-box around the
    source that holds the whole domain of dependence (radius cells), with the
    full grid's damping values, so its fields are exact there."""
    import torch
    shape, h = w.shape, w.spacing
    p = tb.Propagator(shape, h, w.so, physics=physics, nbl=w.nbl)
    vp = torch.from_numpy(w.vp).cuda()
    p.set_model(vp, aux=torch.from_numpy(np.stack(w.meta["aux"])).cuda())
    dt = p.dt
    nt = nsteps
    wav = wl.ricker(w.f0, dt, nt, t0=3 * dt)[None, :].astype(np.float32)
    p.set_sources(w.src_xyz, wav)
    p.set_receivers(w.rec_xyz)
    tr = p.forward(nt, schedule=schedule).cpu().numpy()
    c = np.floor(w.src_xyz[0] / np.array(h)).astype(int)
    lo = np.maximum(c - radius, 0)
    hi = np.minimum(c + radius + 2, np.array(shape))
    sl = tuple(slice(lo[d], hi[d]) for d in range(3))
    sub = tuple(int(hi[d] - lo[d]) for d in range(3))
    # damping of the full grid, restricted to the box
    eta = np.zeros(sub)
    vmax = float(w.vp.max())
    for d in range(3):
        e = oracle.damping_axis(shape[d], w.nbl, h[d], vmax)[lo[d]:hi[d]]
        eta += e.reshape([-1 if k == d else 1 for k in range(3)])
    shift = lo * np.array(h)
    inbox = np.all((w.rec_xyz >= shift) & (w.rec_xyz <= (hi - 1) * np.array(h)), axis=1)
    aux = [a[sl].astype(np.float64) for a in w.meta["aux"]]
    fn = oracle.tti_forward if physics == tb.TB_TTI else oracle.elastic_forward
    tr_o, st_o = fn(sub, h, w.so, dt, nt, w.vp[sl].astype(np.float64), *aux, eta=eta,
                    src_xyz=w.src_xyz - shift, src_wav=wav.astype(np.float64),
                    rec_xyz=w.rec_xyz[inbox] - shift, nthreads=0)
    nf = 4 if physics == tb.TB_TTI else 9
    errs = [rel_l2(p.field(i).cpu().numpy()[sl], st_o[i]) for i in range(nf)]
    e_tr = rel_l2(tr[:, inbox], tr_o)
    print(f"{w.name}: {nt} steps, box {sub}: fields {max(errs):.2e}, traces {e_tr:.2e}")
    assert max(errs) <= TOL and e_tr <= TOL
    assert np.abs(tr_o).max() > 0
    # receivers outside the box are outside the domain of dependence
    assert np.all(tr[:, ~inbox] == 0.0)


@pytest.mark.slow
@pytest.mark.parametrize("schedule", ["onestep", "blocked"])
def test_tti_full_size_subbox(tb, schedule):
    w = wl.tti_384_so8()
    _subbox_parity(tb, tb.TB_TTI, w, nsteps=5, radius=5 * w.so + 4, schedule=schedule)


@pytest.mark.slow
@pytest.mark.parametrize("schedule", ["onestep", "blocked"])
def test_elastic_full_size_subbox(tb, schedule):
    w = wl.elastic_384_so8()
    _subbox_parity(tb, tb.TB_ELASTIC, w, nsteps=6, radius=6 * w.so + 4, schedule=schedule)


@pytest.mark.slow
@pytest.mark.parametrize("physics", ["tti", "elastic"])
def test_full_size_blocked_bitwise_equals_onestep(tb, physics):
    """The benchmark's grid, model and default wavefront (time tile 16, slabs
    of 32 planes) over 26 steps (one wavefront and ten single steps):
    traces and every field bit for bit."""
    import torch
    w = wl.tti_384_so8() if physics == "tti" else wl.elastic_384_so8()
    phys = tb.TB_TTI if physics == "tti" else tb.TB_ELASTIC
    out = []
    for schedule in ("onestep", "blocked"):
        p = tb.Propagator(w.shape, w.spacing, w.so, physics=phys, nbl=w.nbl)
        p.set_model(torch.from_numpy(w.vp).cuda(), aux=torch.from_numpy(np.stack(w.meta["aux"])).cuda())
        nt = 26
        wav = wl.ricker(w.f0, p.dt, nt, t0=3 * p.dt)[None, :].astype(np.float32)
        p.set_sources(w.src_xyz, wav)
        p.set_receivers(w.rec_xyz)
        tr = p.forward(nt, schedule=schedule)
        fields = [p.field(i) for i in range(4 if physics == "tti" else 9)]
        out.append((tr, fields))
        p.close()
    (a_tr, a_f), (b_tr, b_f) = out
    assert torch.equal(a_tr, b_tr) and bool(a_tr.abs().max() > 0)
    for a, b in zip(a_f, b_f):
        assert torch.equal(a, b)
