"""FP64 CPU oracle for the temporally blocked wave propagator (arXiv 2010.10248).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA path (``paper_2010_10248_gb300``)
and imports nothing from it.

The arithmetic lives in ``tb_oracle.c`` (plain C, FP64, compiled with
``-ffp-contract=off`` so that every schedule of the same point update rounds
identically).  This module only compiles it with gcc and marshals numpy
arrays through ctypes.

Functions and what they follow in the paper:

* ``acoustic_forward``    Eq. 1 (Sec. III-A) with Listing 1's direct off-grid
                          injection / interpolation.  The oracle proper.
* ``acoustic_decomposed`` Listing 5 (fused, reduced injection loop).
* ``acoustic_wtb``        Listing 6 (wave-front temporal blocking).
* ``acoustic_wtb_naive``  Fig. 4b (dependence-violating injection; negative test).
* ``inspect_points``      Sec. II-A.1-2 (SM / SID) and Listing 3 (src_dcmp).
* ``tti_forward``         Sec. III-B: the pseudo-acoustic TTI system built on
                          Eq. 2's rotated derivatives (two fields p, r).
* ``elastic_forward``     Eq. 3 (Sec. III-C): isotropic elastic velocity-stress
                          on the staggered grid, explosive source.
* ``acoustic_adjoint``    the exact discrete adjoint of ``acoustic_forward``'s
                          map from wavelets to traces, and the adjoint-state
                          gradient of <traces, residual> with respect to vp.
* ``fd_weights_*``, ``cfl_dt_max``, ``tti_dt_max``, ``elastic_dt_max``,
  ``damping_axis``, ``energy``, ``tti_energy``, ``elastic_energy`` helpers.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tb_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libtb_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile tb_oracle.c into oracle/_build/libtb_oracle.so (gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
           "-Wall", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class Grid(C.Structure):
    _fields_ = [("n", C.c_int64 * 3), ("h", C.c_double * 3), ("so", C.c_int),
                ("nbl", C.c_int), ("periodic", C.c_int), ("nthreads", C.c_int),
                ("dt", C.c_double), ("nt", C.c_int)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            dp = C.POINTER(C.c_double)
            gp = C.POINTER(Grid)
            L = _lib
            L.orc_fd_weights_d2.argtypes = [C.c_int, dp]
            L.orc_fd_weights_d1.argtypes = [C.c_int, dp]
            L.orc_fd_weights_stag.argtypes = [C.c_int, dp]
            L.orc_cfl_dt_max.argtypes = [C.c_int, dp, C.c_double]
            L.orc_cfl_dt_max.restype = C.c_double
            L.orc_damping_axis.argtypes = [C.c_int64, C.c_int, C.c_double, C.c_double, dp]
            L.orc_damping_axis.restype = None
            L.orc_acoustic_forward.argtypes = [gp, dp, dp, C.c_int, dp, dp, C.c_int, dp, dp,
                                               dp, dp, dp, dp]
            L.orc_acoustic_decomposed.argtypes = [gp, dp, dp, C.c_int, dp, dp, C.c_int, dp, dp,
                                                  dp, dp]
            L.orc_acoustic_wtb.argtypes = [gp, dp, dp, C.c_int, dp, dp, C.c_int, dp, dp, dp, dp,
                                           C.c_int, C.c_int, C.c_int, C.c_int, C.c_int]
            L.orc_acoustic_wtb_naive.argtypes = [gp, dp, dp, C.c_int, dp, dp, dp, dp,
                                                 C.c_int, C.c_int, C.c_int, C.c_int, C.c_int]
            L.orc_inspect_points.argtypes = [gp, dp, C.c_int, dp, dp, C.POINTER(C.c_int64),
                                             C.POINTER(C.c_int64), dp]
            L.orc_acoustic_energy.argtypes = [gp, dp, dp, dp]
            L.orc_acoustic_energy.restype = C.c_double
            L.orc_tti_dt_max.argtypes = [C.c_int, dp, C.c_double, C.c_double]
            L.orc_tti_dt_max.restype = C.c_double
            L.orc_tti_forward.argtypes = [gp, dp, dp, dp, dp, dp, dp, C.c_int, dp, dp, C.c_int,
                                          dp, dp, dp, dp]
            L.orc_tti_energy.argtypes = [gp, dp, dp, dp, dp, dp, dp, dp, dp, dp]
            L.orc_tti_energy.restype = C.c_double
            L.orc_elastic_dt_max.argtypes = [C.c_int, dp, C.c_double]
            L.orc_elastic_dt_max.restype = C.c_double
            L.orc_elastic_forward.argtypes = [gp, dp, dp, dp, dp, C.c_int, dp, dp, C.c_int, dp, dp,
                                              dp, dp]
            L.orc_elastic_energy.argtypes = [gp, dp, dp, dp, dp, dp, dp]
            L.orc_elastic_materials.argtypes = [gp, dp, dp, dp, dp]
            L.orc_elastic_energy.restype = C.c_double
            L.orc_acoustic_adjoint.argtypes = [gp, dp, dp, C.c_int, dp, dp, C.c_int, dp, dp, dp, dp]
        return _lib


def _dp(a):
    if a is None:
        return None
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a):
    if a is None:
        return None
    return np.ascontiguousarray(a, dtype=np.float64)


class OracleError(RuntimeError):
    pass


def _check(st, what):
    if st != 0:
        raise OracleError(f"{what} failed with status {st}")


def make_grid(shape, spacing, so, dt, nt, nbl=0, periodic=False, nthreads=0) -> Grid:
    g = Grid()
    for d in range(3):
        g.n[d] = int(shape[d])
        g.h[d] = float(spacing[d])
    g.so, g.nbl, g.periodic, g.nthreads = int(so), int(nbl), int(bool(periodic)), int(nthreads)
    g.dt, g.nt = float(dt), int(nt)
    return g


def fd_weights_d2(so):
    c = np.zeros(32)
    _check(_load().orc_fd_weights_d2(so, _dp(c)), "fd_weights_d2")
    return c[: so // 2 + 1].copy()


def fd_weights_d1(so):
    c = np.zeros(32)
    _check(_load().orc_fd_weights_d1(so, _dp(c)), "fd_weights_d1")
    return c[: so // 2 + 1].copy()


def fd_weights_stag(so):
    c = np.zeros(32)
    _check(_load().orc_fd_weights_stag(so, _dp(c)), "fd_weights_stag")
    return c[: so // 2 + 1].copy()


def cfl_dt_max(so, spacing, vmax):
    h = np.asarray(spacing, dtype=np.float64)
    return float(_load().orc_cfl_dt_max(so, _dp(h), float(vmax)))


def damping_axis(n, nbl, h, vmax):
    e = np.zeros(int(n))
    _load().orc_damping_axis(int(n), int(nbl), float(h), float(vmax), _dp(e))
    return e


def _geom(xyz):
    if xyz is None or len(xyz) == 0:
        return 0, None
    a = _f64(np.asarray(xyz).reshape(-1, 3))
    return a.shape[0], a


def acoustic_forward(shape, spacing, so, dt, nt, vp, *, nbl=0, eta=None, src_xyz=None,
                     src_wav=None, rec_xyz=None, u_init=None, uprev_init=None,
                     periodic=False, nthreads=0):
    """Eq. 1 with Listing 1's direct off-grid injection and interpolation.

    Returns (traces [nt, nrec], u^{nt}, u^{nt-1}) in FP64.
    """
    g = make_grid(shape, spacing, so, dt, nt, nbl, periodic, nthreads)
    vp = _f64(vp)
    nsrc, sx = _geom(src_xyz)
    nrec, rx = _geom(rec_xyz)
    sw = _f64(np.asarray(src_wav).reshape(nsrc, nt)) if nsrc else None
    traces = np.zeros((nt, max(nrec, 1)))
    u = np.zeros(tuple(shape))
    up = np.zeros(tuple(shape))
    st = _load().orc_acoustic_forward(C.byref(g), _dp(vp), _dp(_f64(eta)), nsrc, _dp(sx), _dp(sw),
                                      nrec, _dp(rx), _dp(traces), _dp(_f64(u_init)),
                                      _dp(_f64(uprev_init)), _dp(u), _dp(up))
    _check(st, "acoustic_forward")
    return traces[:, :nrec], u, up


def acoustic_decomposed(shape, spacing, so, dt, nt, vp, *, nbl=0, eta=None, src_xyz=None,
                        src_wav=None, rec_xyz=None, nthreads=0):
    """Listing 5 form (grid-aligned fused injection, reduced z2 loop)."""
    g = make_grid(shape, spacing, so, dt, nt, nbl, False, nthreads)
    vp = _f64(vp)
    nsrc, sx = _geom(src_xyz)
    nrec, rx = _geom(rec_xyz)
    sw = _f64(np.asarray(src_wav).reshape(nsrc, nt)) if nsrc else None
    traces = np.zeros((nt, max(nrec, 1)))
    u = np.zeros(tuple(shape))
    up = np.zeros(tuple(shape))
    st = _load().orc_acoustic_decomposed(C.byref(g), _dp(vp), _dp(_f64(eta)), nsrc, _dp(sx),
                                         _dp(sw), nrec, _dp(rx), _dp(traces), _dp(u), _dp(up))
    _check(st, "acoustic_decomposed")
    return traces[:, :nrec], u, up


def acoustic_wtb(shape, spacing, so, dt, nt, vp, *, tt, tile, block, nbl=0, eta=None,
                 src_xyz=None, src_wav=None, rec_xyz=None, nthreads=0):
    """Listing 6 form: wave-front temporal blocking (tt steps per time tile)."""
    g = make_grid(shape, spacing, so, dt, nt, nbl, False, nthreads)
    vp = _f64(vp)
    nsrc, sx = _geom(src_xyz)
    nrec, rx = _geom(rec_xyz)
    sw = _f64(np.asarray(src_wav).reshape(nsrc, nt)) if nsrc else None
    traces = np.zeros((nt, max(nrec, 1)))
    u = np.zeros(tuple(shape))
    up = np.zeros(tuple(shape))
    st = _load().orc_acoustic_wtb(C.byref(g), _dp(vp), _dp(_f64(eta)), nsrc, _dp(sx), _dp(sw),
                                  nrec, _dp(rx), _dp(traces), _dp(u), _dp(up), int(tt),
                                  int(tile[0]), int(tile[1]), int(block[0]), int(block[1]))
    _check(st, "acoustic_wtb")
    return traces[:, :nrec], u, up


def acoustic_wtb_naive(shape, spacing, so, dt, nt, vp, *, tt, tile, block, nbl=0, eta=None,
                       src_xyz=None, src_wav=None):
    """Fig. 4b: WTB with the off-grid injection at the source's home block."""
    g = make_grid(shape, spacing, so, dt, nt, nbl, False, 1)
    vp = _f64(vp)
    nsrc, sx = _geom(src_xyz)
    sw = _f64(np.asarray(src_wav).reshape(nsrc, nt)) if nsrc else None
    u = np.zeros(tuple(shape))
    up = np.zeros(tuple(shape))
    st = _load().orc_acoustic_wtb_naive(C.byref(g), _dp(vp), _dp(_f64(eta)), nsrc, _dp(sx),
                                        _dp(sw), _dp(u), _dp(up), int(tt), int(tile[0]),
                                        int(tile[1]), int(block[0]), int(block[1]))
    _check(st, "acoustic_wtb_naive")
    return u, up


def inspect_points(shape, spacing, so, dt, nt, vp, xyz, wav=None):
    """Affected points of a set of off-grid points (ascending linear index)
    and, if ``wav`` is given, the decomposition table src_dcmp [nt, npts]."""
    g = make_grid(shape, spacing, so, dt, nt)
    vp = _f64(vp)
    n, x = _geom(xyz)
    npts = C.c_int64(0)
    L = _load()
    _check(L.orc_inspect_points(C.byref(g), _dp(vp), n, _dp(x), None, C.byref(npts), None, None),
           "inspect_points")
    lin = np.zeros(max(npts.value, 1), dtype=np.int64)
    dcmp = np.zeros((nt, max(npts.value, 1))) if wav is not None else None
    w = _f64(np.asarray(wav).reshape(n, nt)) if wav is not None else None
    _check(L.orc_inspect_points(C.byref(g), _dp(vp), n, _dp(x), _dp(w), C.byref(npts),
                                lin.ctypes.data_as(C.POINTER(C.c_int64)), _dp(dcmp)),
           "inspect_points")
    lin = lin[: npts.value]
    if dcmp is not None:
        dcmp = dcmp[:, : npts.value]
    return lin, dcmp


def energy(shape, spacing, so, dt, vp, u_next, u_cur, periodic=False):
    """Discrete leapfrog energy E^{n+1/2} (undamped)."""
    g = make_grid(shape, spacing, so, dt, 1, 0, periodic, 0)
    return float(_load().orc_acoustic_energy(C.byref(g), _dp(_f64(vp)), _dp(_f64(u_next)),
                                             _dp(_f64(u_cur))))


ELASTIC_FIELDS = ("vx", "vy", "vz", "txx", "tyy", "tzz", "txy", "txz", "tyz")


def tti_dt_max(so, spacing, vmax, eps_max):
    h = np.asarray(spacing, dtype=np.float64)
    return float(_load().orc_tti_dt_max(so, _dp(h), float(vmax), float(eps_max)))


def elastic_dt_max(so, spacing, vpmax):
    h = np.asarray(spacing, dtype=np.float64)
    return float(_load().orc_elastic_dt_max(so, _dp(h), float(vpmax)))


def tti_forward(shape, spacing, so, dt, nt, vp, eps, delta, theta, phi, *, nbl=0, eta=None,
                src_xyz=None, src_wav=None, rec_xyz=None, init=None, periodic=False, nthreads=0):
    """Pseudo-acoustic TTI (Sec. III-B, Eq. 2), direct off-grid injection into
    p and r, receivers on p.  ``init``: None or [4, *shape] = p^0, p^-1, r^0,
    r^-1.  Returns (traces [nt, nrec], state [4, *shape] = p^nt, p^nt-1,
    r^nt, r^nt-1)."""
    g = make_grid(shape, spacing, so, dt, nt, nbl, periodic, nthreads)
    nsrc, sx = _geom(src_xyz)
    nrec, rx = _geom(rec_xyz)
    sw = _f64(np.asarray(src_wav).reshape(nsrc, nt)) if nsrc else None
    traces = np.zeros((nt, max(nrec, 1)))
    out = np.zeros((4,) + tuple(shape))
    args = [_f64(np.broadcast_to(a, tuple(shape))) for a in (vp, eps, delta, theta, phi)]
    st = _load().orc_tti_forward(C.byref(g), *[_dp(a) for a in args], _dp(_f64(eta)), nsrc,
                                 _dp(sx), _dp(sw), nrec, _dp(rx), _dp(traces),
                                 _dp(_f64(init)), _dp(out))
    _check(st, "tti_forward")
    return traces[:, :nrec], out


def tti_energy(shape, spacing, so, dt, vp, eps, delta, theta, phi, p_next, p_cur, r_next, r_cur,
               periodic=False):
    """Discrete energy of the undamped TTI leapfrog (eps > delta)."""
    g = make_grid(shape, spacing, so, dt, 1, 0, periodic, 0)
    args = [_f64(np.broadcast_to(a, tuple(shape))) for a in (vp, eps, delta, theta, phi)]
    return float(_load().orc_tti_energy(C.byref(g), *[_dp(a) for a in args],
                                        *[_dp(_f64(a)) for a in (p_next, p_cur, r_next, r_cur)]))


def elastic_forward(shape, spacing, so, dt, nt, vp, vs, rho, *, nbl=0, eta=None, src_xyz=None,
                    src_wav=None, rec_xyz=None, init=None, periodic=False, nthreads=0):
    """Isotropic elastic velocity-stress (Eq. 3) on the staggered grid,
    explosive off-grid source into txx, tyy, tzz, receivers on the mean
    normal stress.  ``init``: None or [9, *shape] in ELASTIC_FIELDS order
    (velocities at -1/2, stresses at 0).  Returns (traces [nt, nrec], state
    [9, *shape]: velocities at nt - 1/2, stresses at nt)."""
    g = make_grid(shape, spacing, so, dt, nt, nbl, periodic, nthreads)
    nsrc, sx = _geom(src_xyz)
    nrec, rx = _geom(rec_xyz)
    sw = _f64(np.asarray(src_wav).reshape(nsrc, nt)) if nsrc else None
    traces = np.zeros((nt, max(nrec, 1)))
    out = np.zeros((9,) + tuple(shape))
    args = [_f64(np.broadcast_to(a, tuple(shape))) for a in (vp, vs, rho)]
    st = _load().orc_elastic_forward(C.byref(g), *[_dp(a) for a in args], _dp(_f64(eta)), nsrc,
                                     _dp(sx), _dp(sw), nrec, _dp(rx), _dp(traces),
                                     _dp(_f64(init)), _dp(out))
    _check(st, "elastic_forward")
    return traces[:, :nrec], out


def elastic_materials(shape, spacing, so, vp, vs, rho):
    """The staggered scheme's material arrays (R18), as the oracle builds them:
    dict of bx, by, bz (buoyancy at half-nodes), lam, mu (nodes), mxy, mxz,
    myz (harmonic shear modulus at edge centres), each of shape ``shape``."""
    g = make_grid(shape, spacing, so, 1e-3, 1)
    args = [_f64(np.broadcast_to(a, tuple(shape))) for a in (vp, vs, rho)]
    out = np.zeros((8,) + tuple(shape))
    _check(_load().orc_elastic_materials(C.byref(g), *[_dp(a) for a in args], _dp(out)),
           "elastic_materials")
    return dict(zip(("bx", "by", "bz", "lam", "mu", "mxy", "mxz", "myz"), out))


def elastic_energy(shape, spacing, so, dt, vp, vs, rho, v_next, v_prev, tau, periodic=False):
    """Discrete energy E^n of the undamped staggered scheme from v^{n+1/2},
    v^{n-1/2} ([3, *shape]) and the stresses at n ([6, *shape])."""
    g = make_grid(shape, spacing, so, dt, 1, 0, periodic, 0)
    args = [_f64(np.broadcast_to(a, tuple(shape))) for a in (vp, vs, rho)]
    return float(_load().orc_elastic_energy(C.byref(g), *[_dp(a) for a in args],
                                            *[_dp(_f64(a)) for a in (v_next, v_prev, tau)]))


def acoustic_adjoint(shape, spacing, so, dt, nt, vp, resid, *, nbl=0, eta=None, src_xyz=None,
                     src_wav=None, rec_xyz=None, nthreads=0):
    """Adjoint of the forward map for adjoint traces ``resid`` [nt, nrec]:
    returns (grad_src [nsrc, nt] = d<d, r>/dq, grad_vp [shape] = d<d, r>/dvp)
    with dt and the damping held fixed."""
    g = make_grid(shape, spacing, so, dt, nt, nbl, False, nthreads)
    nsrc, sx = _geom(src_xyz)
    nrec, rx = _geom(rec_xyz)
    sw = _f64(np.asarray(src_wav).reshape(nsrc, nt)) if nsrc else None
    r = _f64(np.asarray(resid).reshape(nt, nrec))
    gsrc = np.zeros((max(nsrc, 1), nt))
    gvp = np.zeros(tuple(shape))
    st = _load().orc_acoustic_adjoint(C.byref(g), _dp(_f64(vp)), _dp(_f64(eta)), nsrc, _dp(sx), _dp(sw),
                                      nrec, _dp(rx), _dp(r), _dp(gsrc), _dp(gvp))
    _check(st, "acoustic_adjoint")
    return gsrc[:nsrc], gvp
