"""Pins of the TTI (Sec. III-B, Eq. 2) and elastic (Eq. 3) oracles against
what the mathematics fixes: reductions to an independently written scheme,
closed-form discrete eigenmodes, discrete energy conservation and closed
stability limits.  CPU only."""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from tests import _brute as B

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def smooth_field(shape, seed, lo, hi):
    rng = np.random.default_rng(seed)
    f = rng.standard_normal(shape)
    for ax in range(3):  # a few box-filter passes: smooth, then rescale to [lo, hi]
        for _ in range(3):
            f = (np.roll(f, 1, ax) + f + np.roll(f, -1, ax)) / 3.0
    f = (f - f.min()) / (f.max() - f.min())
    return lo + (hi - lo) * f


def ricker(f0, dt, nt, t0=None):
    t0 = 1.0 / f0 if t0 is None else t0
    t = np.arange(nt) * dt - t0
    a = (math.pi * f0 * t) ** 2
    return (1 - 2 * a) * np.exp(-a)


# ----------------------------------------------------------------------- TTI
def frame(theta, phi):
    ct, st, cf, sf = math.cos(theta), math.sin(theta), math.cos(phi), math.sin(phi)
    return (np.array([ct * cf, ct * sf, -st]), np.array([-sf, cf, 0.0]),
            np.array([st * cf, st * sf, ct]))


def test_tti_frame_of_eq2_is_orthonormal():
    for th, ph in [(0.3, 1.1), (0.0, 0.0), (0.7, -0.4)]:
        M = np.stack(frame(th, ph))
        np.testing.assert_allclose(M @ M.T, np.eye(3), atol=1e-15)


@pytest.mark.parametrize("so", [4, 8])
def test_tti_without_anisotropy_is_the_acoustic_scheme(so):
    """eps = delta = 0: p and r obey one equation whose operator is
    H_h + H_z = sum_d Dc_d Dc_d for ANY tilt and azimuth (the frame of Eq. 2
    is orthonormal).  Checked against an independent numpy leapfrog of the
    acoustic equation with that Laplacian (closed rational weights), with
    damping, an off-grid source and receivers."""
    shape, h = (10, 11, 12), (10.0, 12.0, 9.0)
    vp = smooth_field(shape, 1, 1500.0, 2500.0)
    theta = smooth_field(shape, 2, 0.0, 0.8)
    phi = smooth_field(shape, 3, -0.5, 0.9)
    eta = smooth_field(shape, 4, 0.0, 30.0)
    zero = np.zeros(shape)
    dt = 0.5 * oracle.tti_dt_max(so, h, vp.max(), 0.0)
    nt = 25
    src = [(44.3, 61.7, 50.2)]
    wav = [ricker(40.0, dt, nt, t0=6 * dt)]
    rec = [(20.5, 33.3, 71.0), (71.0, 12.0, 18.4)]
    tr, st = oracle.tti_forward(shape, h, so, dt, nt, vp, zero, zero, theta, phi, eta=eta,
                                src_xyz=src, src_wav=wav, rec_xyz=rec)
    np.testing.assert_array_equal(st[0], st[2])  # p == r
    np.testing.assert_array_equal(st[1], st[3])

    def lap(u):
        return sum(B.dcentred(B.dcentred(u, d, so, h[d]), d, so, h[d]) for d in range(3))

    def src_term(n):
        return B.point_field(shape, h, src, [wav[0][n]]) * dt * dt * vp ** 2

    tr_b, u_b = B.acoustic_2nd_order(shape, h, dt, nt, vp, eta, lap, src, wav, rec, src_term)
    assert np.abs(st[0]).max() > 1e-6
    np.testing.assert_allclose(st[0], u_b, rtol=0, atol=1e-12 * np.abs(u_b).max())
    np.testing.assert_allclose(tr, tr_b, rtol=0, atol=1e-12 * np.abs(tr_b).max())


@pytest.mark.parametrize("so", [4, 8])
def test_tti_periodic_eigenmode(so):
    """Constant tilted medium on a periodic box: a plane wave cos(k.x) times an
    eigenvector of the 2x2 symbol matrix
        [[(1+2 eps) A, sqrt(1+2 delta) B], [sqrt(1+2 delta) A, B]],
        A = (xbar.s)^2 + (ybar.s)^2,  B = (zbar.s)^2,  s_d = (2/h) sum a_i sin(i k_d h)
    is an exact solution of the leapfrog with (2/dt^2)(1 - cos w dt) m = lambda."""
    shape, h = (16, 16, 16), (10.0, 10.0, 10.0)
    vp, eps, delta, th, ph = 2000.0, 0.25, 0.1, 0.5, 0.8
    j = (1, 2, 3)
    k = [2 * math.pi * j[d] / (shape[d] * h[d]) for d in range(3)]
    s = np.array([2.0 / h[d] * sum(float(c) * math.sin(i * k[d] * h[d])
                                   for i, c in enumerate(B.D1[so], start=1)) for d in range(3)])
    xb, yb, zb = frame(th, ph)
    A = (xb @ s) ** 2 + (yb @ s) ** 2
    Bz = (zb @ s) ** 2
    M2 = np.array([[(1 + 2 * eps) * A, math.sqrt(1 + 2 * delta) * Bz],
                   [math.sqrt(1 + 2 * delta) * A, Bz]])
    lam, vec = np.linalg.eig(M2)
    dt = 0.6 * oracle.tti_dt_max(so, h, vp, eps)
    m = 1.0 / vp ** 2
    X = np.meshgrid(*[np.arange(shape[d]) * h[d] for d in range(3)], indexing="ij")
    mode = np.cos(k[0] * X[0] + k[1] * X[1] + k[2] * X[2])
    nt = 40
    for i in range(2):
        w = math.acos(1.0 - 0.5 * dt * dt * lam[i].real / m) / dt
        al, be = vec[:, i].real
        init = np.stack([al * mode, math.cos(w * dt) * al * mode,
                         be * mode, math.cos(w * dt) * be * mode])
        _, st = oracle.tti_forward(shape, h, so, dt, nt, vp, eps, delta, th, ph, init=init,
                                   periodic=True)
        c = math.cos(nt * w * dt)
        np.testing.assert_allclose(st[0], c * al * mode, rtol=0, atol=1e-10)
        np.testing.assert_allclose(st[2], c * be * mode, rtol=0, atol=1e-10)


def test_tti_energy_conserved_heterogeneous():
    """Undamped, eps > delta, all parameters varying: the discrete energy
    D^T m C^-1 D / dt^2 - u^{n+1}.H u^n is constant once the source stops
    (needs H_h, H_z symmetric: Dc^T = -Dc and the flux form)."""
    shape, h, so = (14, 12, 13), (10.0, 10.0, 10.0), 8
    vp = smooth_field(shape, 11, 1500.0, 3000.0)
    eps = smooth_field(shape, 12, 0.1, 0.3)
    delta = smooth_field(shape, 13, 0.0, 0.08)
    theta = smooth_field(shape, 14, 0.0, 0.8)
    phi = smooth_field(shape, 15, 0.0, 0.8)
    dt = 0.8 * oracle.tti_dt_max(so, h, vp.max(), eps.max())
    f0 = 30.0
    nstop = int(2.0 / f0 / dt) + 2
    src = [(61.3, 52.2, 58.9)]
    es = []
    for nt in (nstop + 10, nstop + 25, nstop + 40):
        wav = ricker(f0, dt, nt)
        wav[nstop:] = 0.0
        _, a = oracle.tti_forward(shape, h, so, dt, nt, vp, eps, delta, theta, phi,
                                  src_xyz=src, src_wav=[wav])
        _, b = oracle.tti_forward(shape, h, so, dt, nt + 1, vp, eps, delta, theta, phi,
                                  src_xyz=src, src_wav=[np.append(wav, 0.0)])
        es.append(oracle.tti_energy(shape, h, so, dt, vp, eps, delta, theta, phi,
                                    b[0], a[0], b[2], a[2]))
    assert es[0] > 0
    assert abs(es[1] - es[0]) < 1e-10 * es[0] and abs(es[2] - es[0]) < 1e-10 * es[0]


def test_tti_rejects_eps_below_delta():
    shape = (10, 10, 10)
    with pytest.raises(oracle.OracleError):
        oracle.tti_forward(shape, (10.0,) * 3, 4, 1e-3, 2, 2000.0, 0.05, 0.1, 0.0, 0.0)


def test_tti_dt_max_closed_form_so4():
    """so4 centred first derivative: s(t) = 2 sum a_i sin(i t) =
    (4/3) sin t - (1/6) sin 2t peaks where s'(t) = 0, i.e. 2 cos^2 t -
    4 cos t - 1 = 0, cos t = 1 - sqrt(6)/2 (the root in [-1, 1])."""
    ct = 1.0 - math.sqrt(6.0) / 2.0
    st = math.sqrt(1 - ct * ct)
    S1 = 4.0 / 3.0 * st - 1.0 / 6.0 * 2 * st * ct
    h = (10.0, 20.0, 15.0)
    want = 2.0 / (3000.0 * math.sqrt(1.2) * S1 * math.sqrt(sum(1 / x ** 2 for x in h)))
    assert oracle.tti_dt_max(4, h, 3000.0, 0.1) == pytest.approx(want, rel=1e-9)


# ------------------------------------------------------------------- elastic
def test_elastic_dt_max_closed_form():
    """Staggered symbol 2 sum c_k sin((k-1/2) t) peaks at t = pi for so4:
    S = 2 (9/8 + 1/24) = 7/3."""
    h = (10.0, 12.0, 8.0)
    want = 2.0 / (3000.0 * 7.0 / 3.0 * math.sqrt(sum(1 / x ** 2 for x in h)))
    assert oracle.elastic_dt_max(4, h, 3000.0) == pytest.approx(want, rel=1e-12)


@pytest.mark.parametrize("so", [4, 8])
def test_elastic_p_and_s_eigenmodes(so):
    """Periodic constant medium.  P wave along axis 2 and S wave along axis 0
    (polarised along axis 2) are exact solutions of the staggered leapfrog
    with (2/dt) sin(w dt/2) = v s, s = (2/h) sum c_k sin((k - 1/2) kappa h),
    v = vp resp. vs; the normal stresses of the P wave keep the ratio
    lam / (lam + 2 mu)."""
    n, h = 16, 10.0
    shape = (n, n, n)
    vp, vs, rho = 3000.0, 1700.0, 2.0
    lam, mu, b = rho * (vp ** 2 - 2 * vs ** 2), rho * vs ** 2, 1.0 / rho
    dt = 0.7 * oracle.elastic_dt_max(so, (h,) * 3, vp)
    nt = 35
    kap = 2 * math.pi * 3 / (n * h)
    s = 2.0 / h * sum(float(c) * math.sin((k - 0.5) * kap * h)
                      for k, c in enumerate(B.STAG[so], start=1))
    i = np.arange(n)
    ones = np.ones(shape)
    # P along axis 2
    z_node = (i * h)[None, None, :] * ones
    z_half = ((i + 0.5) * h)[None, None, :] * ones
    T = 1.0
    init = np.zeros((9,) + shape)
    init[5] = T * np.cos(kap * z_node)
    init[3] = init[4] = lam / (lam + 2 * mu) * init[5]
    init[2] = dt * b * s * T / 2 * np.sin(kap * z_half)
    _, st = oracle.elastic_forward(shape, (h,) * 3, so, dt, nt, vp, vs, rho, init=init,
                                   periodic=True)
    w = 2.0 / dt * math.asin(dt * vp * s / 2.0)
    c = math.cos(nt * w * dt)
    np.testing.assert_allclose(st[5], c * T * np.cos(kap * z_node), atol=1e-10)
    np.testing.assert_allclose(st[3], c * lam / (lam + 2 * mu) * T * np.cos(kap * z_node),
                               atol=1e-10)
    np.testing.assert_allclose(st[6:], 0.0, atol=1e-12)
    # S along axis 0, polarised along axis 2 (vz, txz)
    x_node = (i * h)[:, None, None] * ones
    x_half = ((i + 0.5) * h)[:, None, None] * ones
    init = np.zeros((9,) + shape)
    init[7] = T * np.sin(kap * x_half)
    init[2] = -dt * b * s * T / 2 * np.cos(kap * x_node)
    _, st = oracle.elastic_forward(shape, (h,) * 3, so, dt, nt, vp, vs, rho, init=init,
                                   periodic=True)
    w = 2.0 / dt * math.asin(dt * vs * s / 2.0)
    np.testing.assert_allclose(st[7], math.cos(nt * w * dt) * T * np.sin(kap * x_half),
                               atol=1e-10)
    np.testing.assert_allclose(st[3:6], 0.0, atol=1e-12)


def test_elastic_energy_conserved_heterogeneous():
    """Undamped heterogeneous medium: E^n = 1/2 v^{n+1/2}.W v^{n-1/2} +
    1/2 tau^n : S tau^n is constant after the source stops (needs the
    node/half-node derivative pair to be exact negative transposes and the
    shear terms on the right edges)."""
    shape, h, so = (13, 12, 14), (10.0, 10.0, 10.0), 8
    vp = smooth_field(shape, 21, 2000.0, 3500.0)
    vs = vp / smooth_field(shape, 22, 1.6, 2.0)
    rho = smooth_field(shape, 23, 1.0, 2.5)
    dt = 0.8 * oracle.elastic_dt_max(so, h, vp.max())
    f0 = 30.0
    nstop = int(2.0 / f0 / dt) + 2
    src = [(61.3, 52.2, 58.9)]
    es = []
    for nt in (nstop + 10, nstop + 25, nstop + 40):
        wav = ricker(f0, dt, nt)
        wav[nstop:] = 0.0
        _, a = oracle.elastic_forward(shape, h, so, dt, nt, vp, vs, rho, src_xyz=src,
                                      src_wav=[wav])
        _, bb = oracle.elastic_forward(shape, h, so, dt, nt + 1, vp, vs, rho, src_xyz=src,
                                       src_wav=[np.append(wav, 0.0)])
        es.append(oracle.elastic_energy(shape, h, so, dt, vp, vs, rho, bb[:3], a[:3], a[3:]))
    assert es[0] > 0
    assert abs(es[1] - es[0]) < 1e-10 * es[0] and abs(es[2] - es[0]) < 1e-10 * es[0]


@pytest.mark.parametrize("so", [4, 8])
def test_elastic_without_shear_is_the_staggered_acoustic_scheme(so):
    """vs = 0, constant density: the three normal stresses stay equal and obey
    tau^{n+1} = 2 tau^n - tau^{n-1} + dt^2 vp^2 sum_d Dm_d Dp_d tau^n
    + dt (s^n - s^{n-1}) (eliminating v from the first-order system).  Checked
    against an independent numpy leapfrog of that second-order form, with
    heterogeneous vp, an off-grid source and receivers."""
    shape, h = (11, 10, 12), (10.0, 11.0, 9.0)
    vp = smooth_field(shape, 31, 1800.0, 3000.0)
    zero = np.zeros(shape)
    rho = 1.7
    dt = 0.6 * oracle.elastic_dt_max(so, h, vp.max())
    nt = 30
    src = [(47.1, 52.9, 40.3)]
    wav = ricker(40.0, dt, nt, t0=6 * dt)
    rec = [(20.5, 33.3, 71.0), (71.0, 12.0, 18.4)]
    tr, st = oracle.elastic_forward(shape, h, so, dt, nt, vp, zero, rho, src_xyz=src,
                                    src_wav=[wav], rec_xyz=rec)
    np.testing.assert_array_equal(st[3], st[4])
    np.testing.assert_array_equal(st[3], st[5])

    def lap(u):
        return sum(B.dstag_minus(B.dstag_plus(u, d, so, h[d]), d, so, h[d]) for d in range(3))

    def src_term(n):
        prev = wav[n - 1] if n > 0 else 0.0
        return B.point_field(shape, h, src, [dt * (wav[n] - prev)])

    tr_b, u_b = B.acoustic_2nd_order(shape, h, dt, nt, vp, zero, lap, src, [wav], rec, src_term)
    assert np.abs(u_b).max() > 1e-6
    np.testing.assert_allclose(st[5], u_b, rtol=0, atol=1e-11 * np.abs(u_b).max())
    np.testing.assert_allclose(tr, tr_b, rtol=0, atol=1e-11 * np.abs(tr_b).max())


def test_elastic_material_averaging_restated():
    """R18's averaging, restated in numpy and compared array by array with the
    oracle's: b = 1/rho at a half-node is the mean of its two nodes, mu at an
    edge centre the harmonic mean of its four nodes (0 when one is 0), and a
    neighbour beyond the last node takes the last node's value (Sec. III-C,
    Eq. 3 on the Virieux grid).  Every edge and corner of the grid is in the
    comparison, so a change to the edge rule fails here."""
    shape = (7, 6, 9)
    g = np.random.Generator(np.random.PCG64(20101018))
    vp = g.uniform(2000.0, 3000.0, shape)
    vs = vp / g.uniform(1.6, 2.2, shape)
    vs[g.uniform(size=shape) < 0.15] = 0.0          # fluid points: mu = 0
    vs[-1, :, 2] = 0.0                              # on the upper x face
    rho = g.uniform(1000.0, 2500.0, shape)
    got = oracle.elastic_materials(shape, (10.0, 11.0, 12.0), 4, vp, vs, rho)

    def nb(a, d):   # value at index + 1 along axis d, the last node repeated
        return np.concatenate([np.take(a, np.arange(1, a.shape[d]), axis=d),
                               np.take(a, [a.shape[d] - 1], axis=d)], axis=d)

    mu = rho * vs ** 2
    lam = rho * (vp ** 2 - 2.0 * vs ** 2)
    b = 1.0 / rho

    def harm(a, b_, c, d):
        with np.errstate(divide="ignore"):
            h = 4.0 / (1.0 / a + 1.0 / b_ + 1.0 / c + 1.0 / d)
        return np.where((a > 0) & (b_ > 0) & (c > 0) & (d > 0), h, 0.0)

    want = {
        "lam": lam, "mu": mu,
        "bx": 0.5 * (b + nb(b, 0)), "by": 0.5 * (b + nb(b, 1)), "bz": 0.5 * (b + nb(b, 2)),
        "mxy": harm(mu, nb(mu, 0), nb(mu, 1), nb(nb(mu, 0), 1)),
        "mxz": harm(mu, nb(mu, 0), nb(mu, 2), nb(nb(mu, 0), 2)),
        "myz": harm(mu, nb(mu, 1), nb(mu, 2), nb(nb(mu, 1), 2)),
    }
    for k, v in want.items():
        np.testing.assert_allclose(got[k], v, rtol=1e-14, atol=0.0, err_msg=k)
    # the edge rule is visible: the last x-face's bx is that node's own 1/rho
    np.testing.assert_allclose(got["bx"][-1], b[-1], rtol=1e-15)
