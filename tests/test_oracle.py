"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these compare the oracle with itself: each check is a closed form,
an invariant, an independent brute force, or an equivalence the paper states
(Sec. II: the grid-aligned, fused and temporally blocked forms compute the
same result as Listing 1).
"""
from __future__ import annotations

import math
import os
from fractions import Fraction as F

import numpy as np
import pytest

import oracle
from paper_2010_10248_gb300 import workloads as wl
from tests import _brute

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fd_weights.txt")


def _golden():
    out = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        kind, so, *cs = line.split()
        out[(kind, int(so))] = [F(c) for c in cs]
    return out


# --------------------------------------------------------------------------
# FD weights (Sec. III, space order 4/8/12)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("so", [4, 8, 12])
def test_golden_weights_satisfy_moment_conditions(so):
    """The stored rationals are exact: Taylor moment conditions hold in Q."""
    g = _golden()
    r = so // 2
    c = g[("d2", so)]
    for k in range(r + 1):
        lhs = (c[0] if k == 0 else 0) + 2 * sum(c[i] * F(i) ** (2 * k) for i in range(1, r + 1))
        assert lhs == (2 if k == 1 else 0)
    c = g[("d1", so)]
    for k in range(r):
        assert 2 * sum(c[i] * F(i) ** (2 * k + 1) for i in range(1, r + 1)) == (1 if k == 0 else 0)
    c = g[("stag", so)]
    for k in range(r):
        assert 2 * sum(c[i] * F(2 * i - 1, 2) ** (2 * k + 1) for i in range(1, r + 1)) == (
            1 if k == 0 else 0)


@pytest.mark.parametrize("so", [4, 8, 12])
def test_fornberg_matches_closed_rationals(oracle_lib, so):
    g = _golden()
    for kind, fn in (("d2", oracle.fd_weights_d2), ("d1", oracle.fd_weights_d1),
                     ("stag", oracle.fd_weights_stag)):
        got = fn(so)
        want = np.array([float(x) for x in g[(kind, so)]])
        np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-15, err_msg=kind)


@pytest.mark.parametrize("so", [4, 8, 12])
def test_dispersion_symbol_order(oracle_lib, so):
    """sigma(theta) = -(c0 + 2 sum c_i cos(i theta)) = theta^2 + O(theta^(so+2))."""
    c = oracle.fd_weights_d2(so)
    r = so // 2

    def sig(th):
        return -(c[0] + 2 * sum(c[i] * math.cos(i * th) for i in range(1, r + 1)))

    e1 = abs(sig(0.8) - 0.64)
    e2 = abs(sig(0.4) - 0.16)
    rate = math.log2(e1 / e2)
    assert rate > so + 2 - 0.5, rate


# --------------------------------------------------------------------------
# CFL time step (Sec. IV-B) and sponge (reading of Sec. IV-B)
# --------------------------------------------------------------------------
def test_cfl_closed_form(oracle_lib):
    # so4: S = |c0 + 2(-c1 + c2)| = 16/3 exactly, so dt_max = 2h / (v sqrt(16)) = h / (2v)
    assert oracle.cfl_dt_max(4, (10.0, 10.0, 10.0), 1500.0) == pytest.approx(1.0 / 300.0, rel=1e-14)
    g = _golden()
    for so in (8, 12):
        c = g[("d2", so)]
        S = abs(c[0] + 2 * sum(c[i] * (-1) ** i for i in range(1, so // 2 + 1)))
        want = 2 * 10.0 / (4500.0 * math.sqrt(3 * float(S)))
        assert oracle.cfl_dt_max(so, (10.0, 10.0, 10.0), 4500.0) == pytest.approx(want, rel=1e-13)
    # unequal spacing: sum of 1/h^2
    got = oracle.cfl_dt_max(4, (10.0, 20.0, 5.0), 2000.0)
    want = 2.0 / (2000.0 * math.sqrt(16.0 / 3.0 * (1 / 100 + 1 / 400 + 1 / 25)))
    assert got == pytest.approx(want, rel=1e-14)


def test_cfl_limit_is_sharp(oracle_lib):
    """Just above dt_max the leapfrog grows without bound; just below it stays bounded."""
    shape, h, v = (12, 12, 12), (10.0, 10.0, 10.0), 1500.0
    dtm = oracle.cfl_dt_max(4, h, v)
    k = [math.pi * (1 - 1 / 12) / h[0]] * 3  # near-Nyquist periodic mode
    x = [np.arange(n) * h[d] for d, n in enumerate(shape)]
    X, Y, Z = np.meshgrid(*x, indexing="ij")
    mode = np.cos(np.pi * (X / h[0] + Y / h[1] + Z / h[2]))  # checkerboard: highest symbol
    vp = np.full(shape, v)
    for fac, bounded in ((0.98, True), (1.02, False)):
        _, u, _ = oracle.acoustic_forward(shape, h, 4, fac * dtm, 400, vp, u_init=mode,
                                          uprev_init=mode, periodic=True)
        assert (np.abs(u).max() < 10.0) == bounded, (fac, np.abs(u).max())
    del k


def test_sponge_profile_special_values(oracle_lib):
    n, nbl, h, vmax = 50, 10, 10.0, 3000.0
    e = oracle.damping_axis(n, nbl, h, vmax)
    emax = 3 * vmax * math.log(1e3) / (2 * nbl * h)
    assert e[0] == pytest.approx(emax, rel=1e-15)
    assert e[n - 1] == pytest.approx(emax, rel=1e-15)
    assert e[nbl - 1] == pytest.approx(emax / nbl ** 2, rel=1e-14)
    assert np.all(e[nbl:n - nbl] == 0.0)
    np.testing.assert_array_equal(e, e[::-1])
    assert np.all(np.diff(e[:nbl + 1]) < 0)
    assert np.all(oracle.damping_axis(n, 0, h, vmax) == 0.0)


# --------------------------------------------------------------------------
# Eq. 1 stencil + leapfrog: closed-form discrete eigenmode on a periodic box
# --------------------------------------------------------------------------
@pytest.mark.parametrize("so", [4, 8, 12])
def test_eigenmode_closed_form(oracle_lib, so):
    shape, h, v = (16, 14, 18), (10.0, 12.0, 8.0), 1800.0
    c = oracle.fd_weights_d2(so)
    r = so // 2
    j = (1, 2, 3)
    k = [2 * math.pi * j[d] / (shape[d] * h[d]) for d in range(3)]
    dt = 0.5 * oracle.cfl_dt_max(so, h, v)

    def sig(th):
        return -(c[0] + 2 * sum(c[i] * math.cos(i * th) for i in range(1, r + 1)))

    rhs = v * v * sum(sig(k[d] * h[d]) / h[d] ** 2 for d in range(3))
    omega = math.acos(1 - 0.5 * dt * dt * rhs) / dt
    x = [np.arange(n) * h[d] for d, n in enumerate(shape)]
    X, Y, Z = np.meshgrid(*x, indexing="ij")
    mode = np.cos(k[0] * X + k[1] * Y + k[2] * Z)
    nt = 60
    _, u, up = oracle.acoustic_forward(shape, h, so, dt, nt, np.full(shape, v), u_init=mode,
                                       uprev_init=math.cos(omega * dt) * mode, periodic=True)
    np.testing.assert_allclose(u, math.cos(nt * omega * dt) * mode, atol=1e-11)
    np.testing.assert_allclose(up, math.cos((nt - 1) * omega * dt) * mode, atol=1e-11)


# --------------------------------------------------------------------------
# Independent brute force, point by point (Listing 1, tiny grids)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("so,shape", [(4, (7, 8, 9)), (8, (10, 11, 12))])
def test_brute_force_tiny_grid(oracle_lib, so, shape):
    h = (10.0, 9.0, 11.0)
    nt, nbl = 7, 2
    vp = wl.layered_vp(shape, 11, nlayers=3, nblobs=2).astype(np.float64)
    dt = 0.7 * oracle.cfl_dt_max(so, h, vp.max())
    src = np.array([[31.7, 40.2, 52.9], [3 * h[0], 4 * h[1], 5 * h[2]]])  # 2nd on a node
    wav = np.stack([np.sin(0.9 * np.arange(nt) + 0.3), np.cos(0.5 * np.arange(nt))])
    rec = np.array([[22.1, 31.0, 44.4], [(shape[0] - 1) * h[0], 12.5, 7.0], [40.0, 45.0, 55.0]])
    tr, u, up = oracle.acoustic_forward(shape, h, so, dt, nt, vp, nbl=nbl, src_xyz=src,
                                        src_wav=wav, rec_xyz=rec)
    btr, bu, bup = _brute.forward(shape, h, so, dt, nt, vp.tolist(), nbl, src.tolist(),
                                  wav.tolist(), rec.tolist())
    scale = np.abs(u).max()
    assert scale > 0
    np.testing.assert_allclose(u, np.array(bu), atol=1e-12 * scale, rtol=0)
    np.testing.assert_allclose(up, np.array(bup), atol=1e-12 * scale, rtol=0)
    np.testing.assert_allclose(tr, np.array(btr), atol=1e-12 * scale, rtol=0)


# --------------------------------------------------------------------------
# Trilinear injection / interpolation (Sec. I, Fig. 3)
# --------------------------------------------------------------------------
def test_inspector_partition_of_unity_and_nodes(oracle_lib):
    shape, h = (12, 13, 14), (10.0, 10.0, 10.0)
    vp = np.full(shape, 2000.0)
    dt, nt = 1e-3, 5
    q = np.arange(1, nt + 1, dtype=np.float64)
    m = 1 / 2000.0 ** 2
    # generic off-grid point: eight points, weights sum to one
    lin, dc = oracle.inspect_points(shape, h, 4, dt, nt, vp, [[31.3, 47.9, 88.2]], q[None, :])
    assert len(lin) == 8 and np.all(np.diff(lin) > 0)
    np.testing.assert_allclose(dc.sum(axis=1) * m / dt ** 2, q, rtol=1e-14)
    # a point exactly on a node is one affected point carrying the full amplitude
    lin, dc = oracle.inspect_points(shape, h, 4, dt, nt, vp, [[30.0, 40.0, 50.0]], q[None, :])
    assert list(lin) == [(3 * 13 + 4) * 14 + 5]
    np.testing.assert_allclose(dc[:, 0] * m / dt ** 2, q, rtol=1e-15)
    # upper edge: base index clamps to n-2, weight 1 on the last node
    lin, _ = oracle.inspect_points(shape, h, 4, dt, nt, vp, [[110.0, 120.0, 130.0]], q[None, :])
    assert list(lin) == [(11 * 13 + 12) * 14 + 13]
    # two sources sharing corners: unique IDs, contributions summed
    lin, dc = oracle.inspect_points(shape, h, 4, dt, nt, vp, [[31.3, 47.9, 88.2], [35.0, 41.0, 81.0]],
                                    np.stack([q, 2 * q]))
    assert len(lin) == 8
    np.testing.assert_allclose(dc.sum(axis=1) * m / dt ** 2, 3 * q, rtol=1e-14)
    with pytest.raises(oracle.OracleError):
        oracle.inspect_points(shape, h, 4, dt, nt, vp, [[-1.0, 5.0, 5.0]], q[None, :])


def test_interpolation_reproduces_affine_fields(oracle_lib):
    shape, h, so = (20, 18, 22), (10.0, 11.0, 9.0), 4
    x = [np.arange(n) * h[d] for d, n in enumerate(shape)]
    X, Y, Z = np.meshgrid(*x, indexing="ij")
    aff = lambda X, Y, Z: 0.3 * X - 1.7 * Y + 0.9 * Z + 5.0  # noqa: E731
    u0 = aff(X, Y, Z)
    rec = np.array([[55.5, 66.6, 77.7], [81.2, 90.9, 100.1], [60.0, 70.4, 95.3]])
    tr, _, _ = oracle.acoustic_forward(shape, h, so, 1e-3, 1, np.full(shape, 1500.0),
                                       rec_xyz=rec, u_init=u0, uprev_init=u0)
    np.testing.assert_allclose(tr[0], aff(rec[:, 0], rec[:, 1], rec[:, 2]), rtol=1e-13)


# --------------------------------------------------------------------------
# Sec. II equivalences: Listing 1 == Listing 5 == Listing 6; Fig. 4b differs
# --------------------------------------------------------------------------
def _mixed_case(so=8, shape=(26, 30, 34), nt=40):
    h = (10.0, 10.0, 10.0)
    vp = wl.layered_vp(shape, 5, nlayers=4, nblobs=3).astype(np.float64)
    dt = 0.8 * oracle.cfl_dt_max(so, h, vp.max())
    src = np.array([[75.3, 118.1, 161.7], [78.0, 121.0, 158.2], [120.0, 150.0, 200.0]])
    wav = np.stack([wl.ricker(40.0, dt, nt), 0.5 * wl.ricker(35.0, dt, nt), wl.ricker(50.0, dt, nt)])
    rec = np.array([[30.5, 40.5, 50.5], [250.0, 100.2, 300.9], [140.1, 140.2, 140.3],
                    [5.5, 290.0, 330.0], [200.0, 200.0, 200.0]])
    return dict(shape=shape, spacing=h, so=so, dt=dt, nt=nt, vp=vp, nbl=4, src_xyz=src,
                src_wav=wav, rec_xyz=rec)


def test_decomposed_equals_direct(oracle_lib):
    c = _mixed_case()
    tr, u, up = oracle.acoustic_forward(**c)
    tr2, u2, up2 = oracle.acoustic_decomposed(**c)
    s = np.abs(u).max()
    assert s > 0 and np.abs(tr).max() > 0
    np.testing.assert_allclose(u2, u, atol=1e-14 * s, rtol=0)
    np.testing.assert_allclose(up2, up, atol=1e-14 * s, rtol=0)
    np.testing.assert_allclose(tr2, tr, atol=1e-14 * np.abs(tr).max(), rtol=0)


@pytest.mark.parametrize("tt,tile,block", [(5, (8, 12), (4, 4)), (3, (16, 16), (8, 8)),
                                           (7, (5, 9), (2, 3)), (40, (64, 64), (8, 8))])
def test_wtb_is_bitwise_equal_to_unblocked(oracle_lib, tt, tile, block):
    c = _mixed_case()
    tr, u, up = oracle.acoustic_decomposed(**c)
    tr2, u2, up2 = oracle.acoustic_wtb(**c, tt=tt, tile=tile, block=block)
    np.testing.assert_array_equal(u2, u)
    np.testing.assert_array_equal(up2, up)
    np.testing.assert_array_equal(tr2, tr)


def test_naive_wtb_violates_dependences(oracle_lib):
    """Fig. 4b: off-grid injection inside a skewed tile reaches corners whose
    stencil update for that step has not run yet; the result is wrong."""
    c = _mixed_case()
    del c["rec_xyz"]
    # source whose corners straddle a block and a tile boundary (x = 7|8, y = 11|12)
    c["src_xyz"] = np.array([[75.3, 118.1, 161.7]])
    c["src_wav"] = c["src_wav"][:1]
    _, u, _ = oracle.acoustic_forward(**c)
    un, _ = oracle.acoustic_wtb_naive(**c, tt=5, tile=(8, 12), block=(4, 4))
    rel = np.linalg.norm(un - u) / np.linalg.norm(u)
    assert rel > 1e-2, rel


# --------------------------------------------------------------------------
# Invariants of the undamped scheme
# --------------------------------------------------------------------------
def test_energy_conserved_after_source_stops(oracle_lib):
    shape, h, so = (24, 20, 28), (10.0, 10.0, 10.0), 8
    vp = wl.layered_vp(shape, 3, nlayers=4, nblobs=3).astype(np.float64)
    dt = 0.8 * oracle.cfl_dt_max(so, h, vp.max())
    f0 = 40.0
    nmax = 170
    w = wl.ricker(f0, dt, nmax)
    w[np.arange(nmax) * dt > 2.0 / f0] = 0.0
    src = [[111.1, 95.5, 140.2]]
    E = []
    for nt in (90, 130, 170):
        _, u, up = oracle.acoustic_forward(shape, h, so, dt, nt, vp, src_xyz=src,
                                           src_wav=w[None, :nt])
        E.append(oracle.energy(shape, h, so, dt, vp, u, up))
    assert E[0] > 0
    assert abs(E[1] - E[0]) / E[0] < 1e-10 and abs(E[2] - E[0]) / E[0] < 1e-10, E
    # while the source is active the energy does change
    _, u, up = oracle.acoustic_forward(shape, h, so, dt, 30, vp, src_xyz=src, src_wav=w[None, :30])
    assert abs(oracle.energy(shape, h, so, dt, vp, u, up) - E[0]) / E[0] > 1e-3


def test_reciprocity(oracle_lib):
    shape, h, so, nt = (20, 22, 24), (10.0, 10.0, 10.0), 8, 90
    vp = wl.layered_vp(shape, 9, nlayers=4, nblobs=3).astype(np.float64)
    dt = 0.8 * oracle.cfl_dt_max(so, h, vp.max())
    w = wl.ricker(45.0, dt, nt)[None, :]
    a = np.array([[63.3, 81.7, 95.1]])
    b = np.array([[131.9, 120.4, 160.6]])
    tab, _, _ = oracle.acoustic_forward(shape, h, so, dt, nt, vp, src_xyz=a, src_wav=w, rec_xyz=b)
    tba, _, _ = oracle.acoustic_forward(shape, h, so, dt, nt, vp, src_xyz=b, src_wav=w, rec_xyz=a)
    s = np.abs(tab).max()
    assert s > 0
    np.testing.assert_allclose(tab, tba, atol=1e-11 * s, rtol=0)


# --------------------------------------------------------------------------
# Whole solve against the analytic 3D Green's function
# --------------------------------------------------------------------------
def _green_run(refine):
    """so8 (the 512^3 case's order), CFL 0.8, Ricker 10 Hz delayed to 1.5/f0 so
    that the wavelet starts smoothly.  Homogeneous, undamped, zero halo; the
    window closes before the first boundary reflection reaches a receiver."""
    v, f0, so, t0 = 1500.0, 10.0, 8, 0.15
    hc = 12.5 / refine
    n = 64 * refine
    shape, h = (n, n, n), (hc, hc, hc)
    dt = 0.8 * oracle.cfl_dt_max(so, h, v)
    nt = int(0.41 / dt)
    src = np.array([[400.0, 400.0, 400.0]])
    rec = np.array([[550.0, 403.1, 397.2], [400.0, 550.0, 401.9]])
    w = wl.ricker(f0, dt, nt, t0=t0)
    tr, _, _ = oracle.acoustic_forward(shape, h, so, dt, nt, np.full(shape, v), src_xyz=src,
                                       src_wav=w[None, :], rec_xyz=rec)
    dist = np.linalg.norm(rec - src, axis=1)
    t = (np.arange(nt) + 1) * dt  # trace[n] samples u^{n+1}
    # u(r, t) = h^3 q(t - r/c) / (4 pi r): the unit-weight grid source carries h^3 q
    exact = np.stack([hc ** 3 * _ricker_at(t - d / v, f0, t0) / (4 * np.pi * d) for d in dist],
                     axis=1)
    err = np.linalg.norm(tr - exact) / np.linalg.norm(exact)
    return err, tr, exact, dt, dist


def _ricker_at(t, f0, t0):
    tau = t - t0
    a = (np.pi * f0 * tau) ** 2
    return (1 - 2 * a) * np.exp(-a)


@pytest.mark.slow
def test_greens_function_convergence(oracle_lib):
    e1, tr, ex, dt, dist = _green_run(1)
    e2, _, _, _, _ = _green_run(2)
    rate = math.log2(e1 / e2)
    assert e1 < 0.03 and e2 < 0.006, (e1, e2)
    assert rate > 1.9, (e1, e2, rate)
    # time alignment: the peak arrives at t0 + r/c within one step
    k = int(np.argmax(tr[:, 0]))
    t_peak = (k + 1) * dt
    assert abs(t_peak - (0.15 + dist[0] / 1500.0)) <= dt
