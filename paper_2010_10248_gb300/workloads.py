"""Seeded synthetic inputs shaped like the paper's workloads (Sec. IV-B).

This module holds input generators only: velocity models, off-grid source
and receiver coordinates, and the source time function.  It contains none of
the propagator's arithmetic (no stencil, no injection, no CFL, no damping),
so that the CUDA path and the FP64 oracle can both be fed from it without
sharing any of the method.

The paper evaluates synthetic 512^3 velocity models with grid spacing 10 m,
one spatially localised source wavelet, damping layers and zero initial
conditions (Sec. IV-B); it names no public dataset.  The recipes below stand
in for those models:

* ``constant``  homogeneous vp (the 64^3 so4 parity case);
* ``layered``   ``nlayers`` horizontal layers along axis 2 (depth), vp rising
                from ``vmin`` to ``vmax`` with depth, seeded interface depths,
                plus ``nblobs`` seeded Gaussian perturbations of +-5 % with
                sigma 20-60 cells (scaled with the grid), clipped to
                [vmin, vmax].

Coordinates are in metres with the origin at grid index 0 (axis order
x, y, z with z the contiguous depth axis).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 2010_10248


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def ricker(f0: float, dt: float, nt: int, t0: float | None = None) -> np.ndarray:
    """Ricker wavelet (amplitude 1) sampled at t_n = n dt, peak at t0 = 1/f0."""
    t0 = 1.0 / f0 if t0 is None else t0
    tau = np.arange(nt, dtype=np.float64) * dt - t0
    a = (math.pi * f0 * tau) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


def constant_vp(shape, v: float) -> np.ndarray:
    return np.full(tuple(shape), v, dtype=np.float32)


def _layers(n2, g, vmin, vmax, nlayers):
    # interface depths: sorted seeded fractions of the depth axis
    cuts = np.sort(g.uniform(0.05, 0.95, size=nlayers - 1)) * n2
    vel = np.linspace(vmin, vmax, nlayers)
    layer = np.searchsorted(cuts, np.arange(n2), side="right")
    return vel[layer].astype(np.float32)


def layered_profile(n2: int, seed: int, vmin: float = 1500.0, vmax: float = 4500.0, nlayers: int = 8) -> np.ndarray:
    """The depth profile of layered_vp without perturbations (the model is
    this profile along axis 2, the same at every (x, y))."""
    return _layers(int(n2), rng(seed), vmin, vmax, nlayers)


def layered_vp(shape, seed: int, vmin: float = 1500.0, vmax: float = 4500.0,
               nlayers: int = 8, nblobs: int = 16, blob_sigma=(20.0, 60.0),
               blob_amp: float = 0.05) -> np.ndarray:
    """Layered model along depth (axis 2) with smooth Gaussian perturbations."""
    n0, n1, n2 = (int(s) for s in shape)
    g = rng(seed)
    prof = _layers(n2, g, vmin, vmax, nlayers)
    vp = np.broadcast_to(prof[None, None, :], (n0, n1, n2)).copy()
    # sigma range is quoted for 512^3; scale it with the grid
    scale = min(n0, n1, n2) / 512.0
    for _ in range(nblobs):
        c = g.uniform(0, 1, size=3) * np.array([n0, n1, n2])
        sig = g.uniform(*blob_sigma) * scale
        amp = g.choice([-1.0, 1.0]) * blob_amp
        lo = [max(0, int(c[d] - 3 * sig)) for d in range(3)]
        hi = [min((n0, n1, n2)[d], int(c[d] + 3 * sig) + 1) for d in range(3)]
        if any(hi[d] <= lo[d] for d in range(3)):
            continue
        gx = np.exp(-0.5 * ((np.arange(lo[0], hi[0]) - c[0]) / sig) ** 2).astype(np.float32)
        gy = np.exp(-0.5 * ((np.arange(lo[1], hi[1]) - c[1]) / sig) ** 2).astype(np.float32)
        gz = np.exp(-0.5 * ((np.arange(lo[2], hi[2]) - c[2]) / sig) ** 2).astype(np.float32)
        box = vp[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]]
        box *= 1.0 + amp * (gx[:, None, None] * gy[None, :, None] * gz[None, None, :])
    np.clip(vp, vmin, vmax, out=vp)
    return vp


def offgrid_point(shape, spacing, seed: int, lo_frac=0.3, hi_frac=0.7) -> np.ndarray:
    """One seeded off-grid point inside the given fraction of the box."""
    g = rng(seed)
    ext = np.array([(shape[d] - 1) * spacing[d] for d in range(3)])
    return g.uniform(lo_frac, hi_frac, size=3) * ext


def receiver_line(shape, spacing, seed: int, nrec: int, margin_cells: float = 2.0) -> np.ndarray:
    """nrec receivers on a line along x at a seeded off-grid (y, z)."""
    g = rng(seed)
    ext = np.array([(shape[d] - 1) * spacing[d] for d in range(3)])
    y = g.uniform(0.3, 0.7) * ext[1]
    z = g.uniform(0.2, 0.5) * ext[2]
    x0 = margin_cells * spacing[0] + g.uniform(0.0, 1.0) * spacing[0]
    x1 = ext[0] - margin_cells * spacing[0]
    xs = np.linspace(x0, x1, nrec)
    return np.stack([xs, np.full(nrec, y), np.full(nrec, z)], axis=1)


def receiver_plane(shape, spacing, seed: int, nx: int, ny: int, depth_cells: float,
                   step_cells: float = 2.0) -> np.ndarray:
    """nx * ny receivers on a horizontal plane at an off-grid depth, spacing
    step_cells grid cells, with a seeded sub-cell offset."""
    g = rng(seed)
    off = g.uniform(0.05, 0.95, size=3)
    ext = np.array([(shape[d] - 1) * spacing[d] for d in range(3)])
    xs = (off[0] + step_cells * np.arange(nx)) * spacing[0]
    ys = (off[1] + step_cells * np.arange(ny)) * spacing[1]
    xs = xs[xs <= ext[0]]
    ys = ys[ys <= ext[1]]
    z = (depth_cells + off[2]) * spacing[2]
    X, Y = np.meshgrid(xs, ys, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), np.full(X.size, z)], axis=1)


def source_plane(shape, spacing, seed: int, n: int, depth_cells: float, margin_cells: float) -> np.ndarray:
    """n sources on a horizontal plane (fixed axis-2 depth): a square lattice
    over axes 0 and 1 inside the margin, each point with a seeded sub-cell
    offset (the sparse many-source case of Sec. V-C)."""
    g = rng(seed)
    k = max(1, int(math.ceil(math.sqrt(n))))
    lo0, hi0 = margin_cells, shape[0] - 2 - margin_cells
    lo1, hi1 = margin_cells, shape[1] - 2 - margin_cells
    X, Y = np.meshgrid(np.linspace(lo0, hi0, k), np.linspace(lo1, hi1, k), indexing="ij")
    off = g.uniform(0.05, 0.95, size=(k * k, 3))
    z = np.full(k * k, float(depth_cells))
    pts = np.stack([np.floor(X.ravel()), np.floor(Y.ravel()), z], axis=1) + off
    return pts[:n] * np.asarray(spacing, dtype=np.float64)


def source_cloud(shape, spacing, seed: int, n: int, margin_cells: float) -> np.ndarray:
    """n sources uniformly random in the box inside the margin (the dense
    many-source case of Sec. V-C)."""
    g = rng(seed)
    lo = np.full(3, float(margin_cells))
    hi = np.array([shape[d] - 1 - margin_cells for d in range(3)], dtype=np.float64)
    return g.uniform(lo, hi, size=(n, 3)) * np.asarray(spacing, dtype=np.float64)


@dataclass
class Workload:
    """One propagation problem: grid, model, geometry and wavelet recipe."""
    name: str
    shape: tuple
    spacing: tuple
    so: int
    nt: int
    nbl: int
    f0: float
    vp: np.ndarray
    src_xyz: np.ndarray
    rec_xyz: np.ndarray
    meta: dict = field(default_factory=dict)

    def wavelets(self, dt: float) -> np.ndarray:
        """[nsrc, nt] source time functions sampled with the step dt."""
        w = ricker(self.f0, dt, self.nt)
        return np.repeat(w[None, :], len(self.src_xyz), axis=0)


def acoustic_64_so4(seed: int = BASE_SEED + 0) -> Workload:
    """64^3, h = 10 m, so4, 100 steps, vp = 1.5 km/s, 10-cell sponge, one
    10 Hz Ricker at a seeded off-grid interior point, 64 receivers on an
    off-grid line along x."""
    shape, h = (64, 64, 64), (10.0, 10.0, 10.0)
    src = offgrid_point(shape, h, seed + 1)[None, :]
    rec = receiver_line(shape, h, seed + 2, 64)
    return Workload("acoustic 64^3 so4 100 steps", shape, h, 4, 100, 10, 10.0,
                    constant_vp(shape, 1500.0), src, rec)


def acoustic_512_so8(seed: int = BASE_SEED + 1, shape=(512, 512, 512), nt: int = 1000,
                     nbl: int = 40, so: int = 8) -> Workload:
    """512^3, h = 10 m, so8, 1000 steps, 40-cell sponge, seeded layered vp
    1.5-4.5 km/s with Gaussian perturbations, one 15 Hz Ricker near the top,
    256 x 256 receiver plane (spacing 2h) at a fixed off-grid depth.
    ``shape`` / ``nt`` / ``nbl`` may be reduced for parity runs that keep
    the same recipe; ``so`` selects another space order on the same model."""
    h = (10.0, 10.0, 10.0)
    g = rng(seed + 7)
    src = np.array([[(0.5 * (shape[0] - 1) + g.uniform(-0.5, 0.5)) * h[0],
                     (0.5 * (shape[1] - 1) + g.uniform(-0.5, 0.5)) * h[1],
                     (nbl + 10 + g.uniform(0.05, 0.95)) * h[2]]])
    # spacing 2h from a sub-cell offset < 1: n // 2 receivers fit in n - 1 cells
    # (256 x 256 = 65,536 at 512^3)
    nrx = min(256, shape[0] // 2)
    nry = min(256, shape[1] // 2)
    rec = receiver_plane(shape, h, seed + 3, nrx, nry, depth_cells=nbl + 20)
    vp = layered_vp(shape, seed + 4)
    return Workload(f"acoustic {shape[0]}x{shape[1]}x{shape[2]} so{so} {nt} steps", tuple(shape), h,
                    so, nt, nbl, 15.0, vp, src, rec)


def smooth_field(shape, seed: int, lo: float, hi: float, coarse: int = 6) -> np.ndarray:
    """Seeded smooth random field in [lo, hi]: uniform noise on a coarse
    (coarse x coarse x coarse) lattice, linearly interpolated to the grid."""
    g = rng(seed)
    c = g.uniform(0.0, 1.0, size=(coarse, coarse, coarse))
    out = c
    for ax, n in enumerate(shape):
        t = np.linspace(0.0, coarse - 1, int(n))
        i0 = np.clip(np.floor(t).astype(int), 0, coarse - 2)
        f = (t - i0).astype(np.float64)
        a = np.take(out, i0, axis=ax)
        b = np.take(out, i0 + 1, axis=ax)
        sh = [1, 1, 1]
        sh[ax] = int(n)
        out = a * (1.0 - f.reshape(sh)) + b * f.reshape(sh)
    return (lo + (hi - lo) * out).astype(np.float32)


def tti_384_so8(seed: int = BASE_SEED + 2, shape=(384, 384, 384), nt: int = 500,
                nbl: int = 30) -> Workload:
    """TTI 384^3, h = 20 m (the paper's TTI spacing), so8, 500 steps: layered
    vp, smooth seeded eps in [0, 0.3], delta in [0, 0.2] with delta <= eps,
    tilt and azimuth in [0, 45 deg]; one 10 Hz Ricker near the top; 128 x 128
    receiver plane.  meta["aux"] holds (eps, delta, theta, phi)."""
    h = (20.0, 20.0, 20.0)
    g = rng(seed + 7)
    src = np.array([[(0.5 * (shape[0] - 1) + g.uniform(-0.5, 0.5)) * h[0],
                     (0.5 * (shape[1] - 1) + g.uniform(-0.5, 0.5)) * h[1],
                     (nbl + 10 + g.uniform(0.05, 0.95)) * h[2]]])
    rec = receiver_plane(shape, h, seed + 3, min(128, (shape[0] - 1) // 2),
                         min(128, (shape[1] - 1) // 2), depth_cells=nbl + 20)
    vp = layered_vp(shape, seed + 4)
    eps = smooth_field(shape, seed + 5, 0.0, 0.3)
    delta = np.minimum(smooth_field(shape, seed + 6, 0.0, 0.2), eps)
    deg = math.pi / 180.0
    theta = smooth_field(shape, seed + 8, 0.0, 45.0 * deg)
    phi = smooth_field(shape, seed + 9, 0.0, 45.0 * deg)
    return Workload(f"tti {shape[0]}x{shape[1]}x{shape[2]} so8 {nt} steps", tuple(shape), h, 8, nt,
                    nbl, 10.0, vp, src, rec, meta={"aux": (eps, delta, theta, phi)})


def elastic_384_so8(seed: int = BASE_SEED + 3, shape=(384, 384, 384), nt: int = 500,
                    nbl: int = 30) -> Workload:
    """Isotropic elastic 384^3, h = 10 m, so8, 500 steps: layered vp,
    vs = vp / 1.7, layered density 1.0-2.5 (same interfaces as vp); one 15 Hz
    explosive Ricker near the top; 128 x 128 receiver plane.  meta["aux"]
    holds (vs, rho)."""
    h = (10.0, 10.0, 10.0)
    g = rng(seed + 7)
    src = np.array([[(0.5 * (shape[0] - 1) + g.uniform(-0.5, 0.5)) * h[0],
                     (0.5 * (shape[1] - 1) + g.uniform(-0.5, 0.5)) * h[1],
                     (nbl + 10 + g.uniform(0.05, 0.95)) * h[2]]])
    rec = receiver_plane(shape, h, seed + 3, min(128, (shape[0] - 1) // 2),
                         min(128, (shape[1] - 1) // 2), depth_cells=nbl + 20)
    vp = layered_vp(shape, seed + 4, nblobs=0)
    vs = (vp / 1.7).astype(np.float32)
    rho = (1.0 + (vp - 1500.0) / 3000.0 * 1.5).astype(np.float32)
    return Workload(f"elastic {shape[0]}x{shape[1]}x{shape[2]} so8 {nt} steps", tuple(shape), h, 8, nt,
                    nbl, 15.0, vp, src, rec, meta={"aux": (vs, rho)})
