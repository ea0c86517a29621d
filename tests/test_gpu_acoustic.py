"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances: rel-L2 <= 1e-4 against the oracle (FP32 arithmetic), and the
temporally blocked schedule bitwise equal to the one-step kernel (every
point update uses the same round-to-nearest operation sequence).
Integer inspector tables are compared bit-exactly.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2010_10248_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = 1e-4


def rel(a, b):
    nb = np.linalg.norm(b)
    assert nb > 0
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / nb)


@pytest.fixture(scope="module")
def tb():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    import paper_2010_10248_gb300 as tb
    return tb


def make_case(name):
    if name == "cfg64_so4":
        w = wl.acoustic_64_so4()
        return dict(shape=w.shape, h=w.spacing, so=w.so, nt=w.nt, nbl=w.nbl, vp=w.vp,
                    src=w.src_xyz, rec=w.rec_xyz, f0=w.f0)
    if name == "ragged_so8":
        shape, h = (37, 45, 83), (10.0, 11.0, 9.0)
        vp = wl.layered_vp(shape, 17, nlayers=5, nblobs=4)
        src = np.array([[171.3, 240.9, 371.4],                 # generic off-grid point
                        [200.0, 220.0, 360.0],                 # exactly on a node
                        [360.0, 484.0, 738.0],                 # upper corner of the grid
                        [175.0, 237.0, 369.0]])                # shares corners with the first
        rec = np.concatenate([wl.receiver_line(shape, h, 5, 20),
                              np.array([[0.0, 0.0, 0.0], [360.0, 484.0, 738.0],
                                        [181.1, 200.5, 400.2]])])
        return dict(shape=shape, h=h, so=8, nt=60, nbl=5, vp=vp, src=src, rec=rec, f0=55.0)
    if name == "ragged_so12":
        shape, h = (30, 33, 70), (10.0, 10.0, 10.0)
        vp = wl.layered_vp(shape, 23, nlayers=3, nblobs=2)
        src = np.array([[145.5, 161.2, 300.7]])
        rec = wl.receiver_line(shape, h, 7, 12)
        return dict(shape=shape, h=h, so=12, nt=40, nbl=4, vp=vp, src=src, rec=rec, f0=60.0)
    if name == "ragged_so4":
        shape, h = (26, 70, 131), (10.0, 10.0, 10.0)
        vp = wl.layered_vp(shape, 29, nlayers=4, nblobs=3)
        src = np.array([[121.1, 345.6, 650.2], [40.0, 100.0, 1300.0]])
        rec = wl.receiver_plane(shape, h, 31, 12, 34, depth_cells=20)
        return dict(shape=shape, h=h, so=4, nt=50, nbl=6, vp=vp, src=src, rec=rec, f0=50.0)
    if name == "sources_so8":
        # many sources: twelve along axis 0 in one column (its plane range has
        # gaps; the axis-2 corners straddle two column pairs), a cloud of 40,
        # and two on the last, unpaired column of an odd axis 2
        shape, h = (40, 26, 37), (10.0, 10.0, 10.0)
        vp = wl.layered_vp(shape, 37, nlayers=3, nblobs=2)
        g = np.random.default_rng(41)
        ext = np.array([(shape[d] - 1) * h[d] for d in range(3)])
        line = np.array([[20.0 + 31.0 * i, 101.3, 152.7] for i in range(12)])
        cloud = g.uniform(0.1, 0.9, size=(40, 3)) * ext
        edge = np.array([[133.3, 57.1, 360.0], [250.0, 200.0, 360.0]])
        src = np.concatenate([line, cloud, edge])
        rec = wl.receiver_line(shape, h, 9, 16)
        return dict(shape=shape, h=h, so=8, nt=60, nbl=5, vp=vp, src=src, rec=rec, f0=55.0)
    if name == "tall_so8":
        # a grid tall along axis 1, so that with few CTAs per launch the
        # blocked sweep's bands are pipelined across time tiles
        shape, h = (30, 96, 70), (10.0, 10.0, 10.0)
        vp = wl.layered_vp(shape, 43, nlayers=4, nblobs=3)
        src = np.array([[150.3, 100.7, 340.2], [120.0, 830.0, 95.5], [41.0, 520.2, 600.9]])
        rec = np.concatenate([wl.receiver_line(shape, h, 11, 24),
                              np.array([[10.0, 945.0, 100.0], [250.0, 15.0, 680.0]])])
        return dict(shape=shape, h=h, so=8, nt=61, nbl=5, vp=vp, src=src, rec=rec, f0=55.0)
    raise KeyError(name)


_oracle_cache = {}


def oracle_run(name, c, dt, wav):
    if name not in _oracle_cache:
        _oracle_cache[name] = oracle.acoustic_forward(
            c["shape"], c["h"], c["so"], dt, c["nt"], c["vp"].astype(np.float64), nbl=c["nbl"],
            src_xyz=c["src"], src_wav=wav, rec_xyz=c["rec"])
    return _oracle_cache[name]


def gpu_run(tb, c, dt, wav, schedule, **opt):
    import torch
    p = tb.Propagator(c["shape"], c["h"], c["so"], nbl=c["nbl"], **opt)
    p.set_model(torch.from_numpy(np.ascontiguousarray(c["vp"])).cuda(), dt=dt)
    p.set_sources(c["src"], wav)
    p.set_receivers(c["rec"])
    tr = p.forward(c["nt"], schedule=schedule)
    torch.cuda.synchronize()
    out = tr.cpu().numpy(), p.field(0).cpu().numpy(), p.field(1).cpu().numpy()
    p.close()
    return out


def setup(name):
    c = make_case(name)
    dt = 0.8 * oracle.cfl_dt_max(c["so"], c["h"], float(c["vp"].max()))
    wav = np.repeat(wl.ricker(c["f0"], dt, c["nt"])[None, :], len(c["src"]), axis=0)
    return c, dt, wav


CASES = ["cfg64_so4", "ragged_so8", "ragged_so12", "ragged_so4", "sources_so8"]


@pytest.mark.parametrize("name", CASES)
def test_onestep_matches_oracle(tb, name):
    c, dt, wav = setup(name)
    tr_o, u_o, up_o = oracle_run(name, c, dt, wav)
    tr, u, up = gpu_run(tb, c, dt, wav, "onestep")
    assert rel(u, u_o) <= TOL, rel(u, u_o)
    assert rel(up, up_o) <= TOL
    assert rel(tr, tr_o) <= TOL, rel(tr, tr_o)


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("T,opts", [(2, {}), (3, {}), (4, {}),
                                    (4, dict(y_bands=2, x_chunks=3)),
                                    (3, dict(y_bands=3, x_chunks=2)),
                                    (2, dict(y_bands=2))])
def test_blocked_bitwise_equals_onestep(tb, name, T, opts):
    c, dt, wav = setup(name)
    if c["so"] == 12 and T > 2:
        T = 2  # the longest fused sweep that fits shared memory at space order 12
    ref = gpu_run(tb, c, dt, wav, "onestep", x_chunks=1)
    got = gpu_run(tb, c, dt, wav, "blocked", time_tile=T, **opts)
    for a, b in zip(got, ref):
        np.testing.assert_array_equal(a, b)
    tr_o, u_o, _ = oracle_run(name, c, dt, wav)
    assert rel(got[1], u_o) <= TOL and rel(got[0], tr_o) <= TOL


# Launches limited to a few CTAs: bands pipelined across time tiles, most
# launches holding the last band of one time tile and the first rows of the
# next (two time tiles in flight, receiver rows recorded out of step order).
@pytest.mark.parametrize("name,T,band_ctas", [("tall_so8", 3, 10), ("tall_so8", 2, 8), ("tall_so8", 4, 10),
                                              ("tall_so8", 3, 6), ("ragged_so4", 2, 9), ("ragged_so4", 4, 12)])
def test_pipelined_bands_bitwise_equal_onestep(tb, name, T, band_ctas):
    c, dt, wav = setup(name)
    ref = gpu_run(tb, c, dt, wav, "onestep", x_chunks=1)
    got = gpu_run(tb, c, dt, wav, "blocked", time_tile=T, band_ctas=band_ctas)
    for a, b in zip(got, ref):
        np.testing.assert_array_equal(a, b)
    tr_o, u_o, _ = oracle_run(name, c, dt, wav)
    assert rel(got[1], u_o) <= TOL and rel(got[0], tr_o) <= TOL


@pytest.mark.parametrize("layout,nsrc", [("plane", 150), ("dense", 400)])
def test_many_sources_match_oracle(tb, layout, nsrc):
    """Sec. V-C's corner cases at a small size: many sources on a horizontal
    plane (few column pairs with long plane ranges) and spread through the
    grid (many column pairs, gaps inside their ranges), each with its own
    amplitude; pipelined blocked sweeps bitwise equal to the one-step kernel,
    both against the FP64 oracle."""
    shape, h = (30, 64, 44), (10.0, 11.0, 9.0)
    vp = wl.layered_vp(shape, 53, nlayers=3, nblobs=2)
    if layout == "plane":
        src = wl.source_plane(shape, h, 55, nsrc, depth_cells=9, margin_cells=3)
    else:
        src = wl.source_cloud(shape, h, 56, nsrc, margin_cells=1)
    rec = np.concatenate([wl.receiver_line(shape, h, 57, 30), wl.source_cloud(shape, h, 58, 40, 0.5)])
    c = dict(shape=shape, h=h, so=8, nt=40, nbl=4, vp=vp, src=src, rec=rec, f0=55.0)
    dt = 0.8 * oracle.cfl_dt_max(c["so"], c["h"], float(c["vp"].max()))
    amp = wl.rng(59).uniform(-1.0, 1.0, size=(nsrc, 1))
    wav = (amp * wl.ricker(c["f0"], dt, c["nt"])[None, :]).astype(np.float64)
    ref = gpu_run(tb, c, dt, wav, "onestep", x_chunks=1)
    got = gpu_run(tb, c, dt, wav, "blocked", time_tile=3, band_ctas=3)
    for a, b in zip(got, ref):
        np.testing.assert_array_equal(a, b)
    tr_o, u_o, _ = oracle.acoustic_forward(shape, h, c["so"], dt, c["nt"], vp.astype(np.float64), nbl=c["nbl"],
                                           src_xyz=src, src_wav=wav, rec_xyz=rec)
    assert np.abs(u_o).max() > 0
    assert rel(got[1], u_o) <= TOL and rel(got[0], tr_o) <= TOL


def test_pipelined_launch_too_small_is_rejected(tb):
    import torch
    c, dt, wav = setup("tall_so8")
    p = tb.Propagator(c["shape"], c["h"], c["so"], nbl=c["nbl"], time_tile=3, band_ctas=2)
    p.set_model(torch.from_numpy(np.ascontiguousarray(c["vp"])).cuda(), dt=dt)
    with pytest.raises(tb.TBError):
        p.forward(6, schedule="blocked")
    p.close()


@pytest.mark.parametrize("opts", [dict(x_chunks=1), dict(x_chunks=5), dict(y_bands=2, x_chunks=2)])
def test_onestep_decompositions_agree(tb, opts):
    c, dt, wav = setup("ragged_so8")
    ref = gpu_run(tb, c, dt, wav, "onestep", x_chunks=1)
    got = gpu_run(tb, c, dt, wav, "onestep", **opts)
    for a, b in zip(got, ref):
        np.testing.assert_array_equal(a, b)


def test_inspector_tables_match_oracle(tb):
    import torch
    c, dt, wav = setup("ragged_so8")
    p = tb.Propagator(c["shape"], c["h"], c["so"], nbl=c["nbl"])
    p.set_model(torch.from_numpy(c["vp"]).cuda(), dt=dt)
    p.set_sources(c["src"], wav)
    p.set_receivers(c["rec"])
    lin, dcmp = p.source_points()
    lin_o, dcmp_o = oracle.inspect_points(c["shape"], c["h"], c["so"], dt, c["nt"],
                                          c["vp"].astype(np.float64), c["src"], wav)
    np.testing.assert_array_equal(lin, lin_o)
    np.testing.assert_allclose(dcmp, dcmp_o, rtol=2e-6, atol=2e-6 * np.abs(dcmp_o).max())
    rlin, cid, cw = p.receiver_points()
    rlin_o, _ = oracle.inspect_points(c["shape"], c["h"], c["so"], dt, 1,
                                      c["vp"].astype(np.float64), c["rec"])
    np.testing.assert_array_equal(rlin, rlin_o)
    np.testing.assert_allclose(cw.sum(axis=1), 1.0, atol=1e-6)
    assert np.all((cid >= -1) & (cid < len(rlin)))
    assert np.all((cid >= 0) == (cw != 0))
    p.close()


@pytest.mark.parametrize("nsrc", [256, 1024])
def test_inspector_power_of_two_corner_count(tb, nsrc):
    """8 * nsrc corners fill the sort exactly (no sentinel tail)."""
    import torch
    c, dt, _ = setup("ragged_so8")
    g = wl.rng(77)
    ext = np.array([(c["shape"][d] - 1) * c["h"][d] for d in range(3)])
    src = g.uniform(0.05, 0.95, size=(nsrc, 3)) * ext
    wav = np.repeat(wl.ricker(55.0, dt, 8)[None, :], nsrc, axis=0)
    p = tb.Propagator(c["shape"], c["h"], c["so"], nbl=c["nbl"])
    p.set_model(torch.from_numpy(c["vp"]).cuda(), dt=dt)
    p.set_sources(src, wav)
    lin, _ = p.source_points()
    lin_o, _ = oracle.inspect_points(c["shape"], c["h"], c["so"], dt, 8,
                                     c["vp"].astype(np.float64), src, wav)
    np.testing.assert_array_equal(lin, lin_o)
    p.close()


def test_empty_geometry_and_zero_steps(tb):
    import torch
    c, dt, wav = setup("ragged_so12")
    p = tb.Propagator(c["shape"], c["h"], c["so"], nbl=c["nbl"])
    p.set_model(torch.from_numpy(c["vp"]).cuda(), dt=dt)
    p.set_sources(np.zeros((0, 3)), np.zeros((0, 5), np.float32))
    p.set_receivers(c["rec"])
    tr = p.forward(9, schedule="blocked")
    assert float(tr.abs().max()) == 0.0 and float(p.field(0).abs().max()) == 0.0
    p.forward(0, schedule="onestep")
    p.close()


def test_error_paths(tb):
    import torch
    c, dt, wav = setup("ragged_so12")
    vp = torch.from_numpy(c["vp"]).cuda()
    p = tb.Propagator(c["shape"], c["h"], c["so"], nbl=c["nbl"], check_nan=True)
    with pytest.raises(tb.TBError) as e:
        p.forward(5)
    assert e.value.status == tb._tb.TB_ESTATE
    with pytest.raises(tb.TBError) as e:
        p.set_model(vp, dt=1.5 * oracle.cfl_dt_max(c["so"], c["h"], float(c["vp"].max())))
    assert e.value.status == tb._tb.TB_EUNSTABLE
    bad = vp.clone()
    bad[3, 4, 5] = -1.0
    with pytest.raises(tb.TBError) as e:
        p.set_model(bad, dt=dt)
    assert e.value.status == tb._tb.TB_EINVAL
    p.set_model(vp, dt=dt)
    with pytest.raises(tb.TBError) as e:
        p.set_sources(np.array([[-5.0, 10.0, 10.0]]), wav[:1])
    assert e.value.status == tb._tb.TB_EINVAL
    p.set_sources(c["src"], wav)
    p.set_receivers(c["rec"])
    with pytest.raises(tb.TBError) as e:
        p.forward(c["nt"] + 1)
    assert e.value.status == tb._tb.TB_EINVAL
    # non-finite wavelet -> non-finite traces -> TB_EDIVERGED (host-made failure)
    w2 = wav.copy()
    w2[0, 3] = np.nan
    p.set_sources(c["src"], w2)
    with pytest.raises(tb.TBError) as e:
        p.forward(c["nt"], schedule="blocked")
    assert e.value.status == tb._tb.TB_EDIVERGED
    # the handle stays usable
    p.set_sources(c["src"], wav)
    tr = p.forward(c["nt"], schedule="blocked")
    assert torch.isfinite(tr).all()
    p.close()


def test_bounded_wait_times_out_and_context_survives(tb):
    import torch
    st = tb.tb_selftest_wait(0.2)
    assert st == tb._tb.TB_ETIMEOUT
    x = torch.ones(1000, device="cuda")
    assert float(x.sum()) == 1000.0
    test_onestep_matches_oracle(tb, "ragged_so12")


# ---------------------------------------------------------------------------
# Full size (512^3, space order 8): the launch configuration bench.py times
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def big(tb):
    w = wl.acoustic_512_so8()
    return w


def _big_run(tb, w, nt, schedule, time_tile=3):
    import torch
    p = tb.Propagator(w.shape, w.spacing, w.so, nbl=w.nbl, time_tile=time_tile)
    p.set_model(torch.from_numpy(w.vp).cuda())
    dt = p.dt
    p.set_sources(w.src_xyz, w.wavelets(dt)[:, :nt])
    p.set_receivers(w.rec_xyz)
    tr = p.forward(nt, schedule=schedule)
    torch.cuda.synchronize()
    return p, dt, tr


def test_full_size_short_run_matches_oracle(tb, big):
    """512^3 so8, 24 steps (the source wavelet delayed so that the field is
    well away from zero), in the benchmark's launch configuration (blocked
    T = 3, bands pipelined across time tiles over every co-resident CTA):
    whole wavefield and all 65,536 traces vs oracle."""
    import torch
    nt = 24
    p, dt, _ = _big_run(tb, big, nt, "blocked", time_tile=3)
    wav = wl.ricker(big.f0, dt, nt, t0=6 * dt)[None, :]
    p.set_sources(big.src_xyz, wav)
    tr = p.forward(nt, schedule="blocked").cpu().numpy()
    u = p.field(0).cpu().numpy()
    p.close()
    torch.cuda.empty_cache()
    tr_o, u_o, _ = oracle.acoustic_forward(big.shape, big.spacing, big.so, dt, nt,
                                           big.vp.astype(np.float64), nbl=big.nbl,
                                           src_xyz=big.src_xyz, src_wav=wav, rec_xyz=big.rec_xyz)
    print(f"512^3 so8 {nt} steps: rel-L2 field {rel(u, u_o):.3e}, traces {rel(tr, tr_o):.3e}")
    assert rel(u, u_o) <= TOL, rel(u, u_o)
    assert rel(tr, tr_o) <= TOL, rel(tr, tr_o)


@pytest.mark.parametrize("time_tile", [3, 4])
def test_full_size_blocked_equals_onestep_all_steps(tb, big, time_tile):
    """512^3 so8, the full 1000 steps: the blocked schedule bitwise equal to
    the one-step kernel (a property that holds at any size); T = 3 is the
    benchmark's configuration (pipelined bands at the full CTA count)."""
    import torch
    p, _, tr_b = _big_run(tb, big, big.nt, "blocked", time_tile=time_tile)
    u_b = p.field(0)
    tr_1 = p.forward(big.nt, schedule="onestep")
    u_1 = p.field(0)
    assert torch.equal(tr_b, tr_1)
    assert torch.equal(u_b, u_1)
    assert float(tr_1.abs().max()) > 0
    p.close()


def test_fp32_error_growth_1000_steps(tb):
    """The 512^3 recipe at 128^3 for 1000 steps against the FP64 oracle."""
    w = wl.acoustic_512_so8(shape=(128, 128, 128), nt=1000, nbl=10)
    c = dict(shape=w.shape, h=w.spacing, so=w.so, nt=w.nt, nbl=w.nbl, vp=w.vp, src=w.src_xyz,
             rec=w.rec_xyz, f0=w.f0)
    dt = 0.8 * oracle.cfl_dt_max(c["so"], c["h"], float(c["vp"].max()))
    wav = w.wavelets(dt)
    tr_o, u_o, _ = oracle.acoustic_forward(c["shape"], c["h"], c["so"], dt, c["nt"],
                                           c["vp"].astype(np.float64), nbl=c["nbl"],
                                           src_xyz=c["src"], src_wav=wav, rec_xyz=c["rec"])
    tr, u, _ = gpu_run(tb, c, dt, wav, "blocked", time_tile=4)
    print(f"128^3 so8 1000 steps: rel-L2 field {rel(u, u_o):.3e}, traces {rel(tr, tr_o):.3e}")
    assert rel(u, u_o) <= TOL, rel(u, u_o)
    assert rel(tr, tr_o) <= TOL, rel(tr, tr_o)


def test_measured_peaks_in_run(tb):
    """The library's own copy and FMA kernels measure plausible peaks."""
    hbm, fp32 = tb.tb_measure_peaks()
    print(f"copy {hbm:.0f} GB/s, packed FP32 FMA {fp32:.1f} TFLOP/s")
    assert 1000.0 < hbm < 10000.0
    assert 10.0 < fp32 < 200.0
