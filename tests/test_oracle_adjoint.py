"""Pins of the oracle's adjoint and velocity gradient: the adjoint
dot-product test against the (pinned) forward map, and central finite
differences of <d(vp), r>.  CPU only."""
from __future__ import annotations

import numpy as np

import oracle
from tests.test_oracle_physics import ricker, smooth_field


def setup(shape=(14, 15, 16), so=8, nt=40, seed=3):
    h = (10.0, 11.0, 9.0)
    vp = smooth_field(shape, seed, 1800.0, 2600.0)
    eta = smooth_field(shape, seed + 1, 0.0, 40.0)  # damping everywhere, held fixed
    g = np.random.default_rng(seed + 2)
    ext = np.array([(shape[d] - 1) * h[d] for d in range(3)])
    src = g.uniform(0.3, 0.7, size=(2, 3)) * ext
    rec = g.uniform(0.05, 0.95, size=(9, 3)) * ext
    rec[0] = ext            # the upper corner (clamped base)
    dt = 0.7 * oracle.cfl_dt_max(so, h, vp.max())
    return h, so, nt, vp, eta, src, rec, dt, g


def test_adjoint_dot_product():
    """<F q, r> = <q, F^T r> for random wavelets q and adjoint traces r."""
    h, so, nt, vp, eta, src, rec, dt, g = setup()
    q = g.standard_normal((2, nt))
    r = g.standard_normal((nt, len(rec)))
    d, _, _ = oracle.acoustic_forward(vp.shape, h, so, dt, nt, vp, eta=eta, src_xyz=src, src_wav=q,
                                      rec_xyz=rec)
    gsrc, _ = oracle.acoustic_adjoint(vp.shape, h, so, dt, nt, vp, r, eta=eta, src_xyz=src,
                                      src_wav=q, rec_xyz=rec)
    lhs = float(np.sum(d * r))
    rhs = float(np.sum(q * gsrc))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1e-300)


def test_velocity_gradient_against_central_differences():
    """d<d(vp), r>/dvp . dv equals the central difference of <d(vp), r> (dt
    and damping fixed); O(e^2) truncation, e = 1e-3 relative."""
    h, so, nt, vp, eta, src, rec, dt, g = setup(nt=50)
    q = ricker(40.0, dt, nt, t0=6 * dt)[None, :].repeat(2, axis=0)
    r = g.standard_normal((nt, len(rec)))
    _, gvp = oracle.acoustic_adjoint(vp.shape, h, so, dt, nt, vp, r, eta=eta, src_xyz=src, src_wav=q,
                                     rec_xyz=rec)
    dv = smooth_field(vp.shape, 17, -1.0, 1.0) * vp
    e = 1e-3

    def J(v):
        d, _, _ = oracle.acoustic_forward(vp.shape, h, so, dt, nt, v, eta=eta, src_xyz=src,
                                          src_wav=q, rec_xyz=rec)
        return float(np.sum(d * r))

    fd = (J(vp + e * dv) - J(vp - e * dv)) / (2 * e)
    an = float(np.sum(gvp * dv))
    assert abs(fd - an) <= 1e-6 * abs(an)
    # the source term of the gradient matters: a point perturbation at a
    # source corner changes <d, r> as the gradient says
    c = tuple(np.floor(src[0] / np.array(h)).astype(int))
    dv2 = np.zeros(vp.shape)
    dv2[c] = vp[c]
    fd2 = (J(vp + e * dv2) - J(vp - e * dv2)) / (2 * e)
    assert abs(fd2 - float(np.sum(gvp * dv2))) <= 1e-5 * abs(fd2)
