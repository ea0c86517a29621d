"""Pure-Python brute force of the discretised Eq. 1 on tiny grids.

Written independently of oracle/tb_oracle.c: plain nested loops over Python
floats, the closed rational stencil weights (not Fornberg's recursion), an
explicit zero halo by bounds test, and Listing 1's off-grid injection and
trilinear interpolation written out corner by corner.  Used to pin the C
oracle point by point on grids of a few hundred to a few thousand points.
"""
from __future__ import annotations

import math
from fractions import Fraction as F

# Centred second-derivative weights (c0, c1, ..., cr), closed rationals.
D2 = {
    4: [F(-5, 2), F(4, 3), F(-1, 12)],
    8: [F(-205, 72), F(8, 5), F(-1, 5), F(8, 315), F(-1, 560)],
    12: [F(-5369, 1800), F(12, 7), F(-15, 56), F(10, 189), F(-1, 112), F(2, 1925),
         F(-1, 16632)],
}


def sponge(n, nbl, h, vmax):
    out = []
    for i in range(n):
        if nbl <= 0:
            out.append(0.0)
            continue
        if i < nbl:
            d = nbl - i
        elif i > n - 1 - nbl:
            d = i - (n - 1 - nbl)
        else:
            d = 0
        emax = 3.0 * vmax * math.log(1000.0) / (2.0 * nbl * h)
        out.append(emax * (d / nbl) ** 2)
    return out


def corners(pt, shape, h):
    """Eight (index, weight) pairs of the trilinear stencil of one point."""
    base, frac = [], []
    for d in range(3):
        t = pt[d] / h[d]
        i = int(math.floor(t))
        i = min(max(i, 0), shape[d] - 2)
        base.append(i)
        frac.append(t - i)
    out = []
    for bx in (0, 1):
        for by in (0, 1):
            for bz in (0, 1):
                w = ((frac[0] if bx else 1 - frac[0]) * (frac[1] if by else 1 - frac[1])
                     * (frac[2] if bz else 1 - frac[2]))
                out.append(((base[0] + bx, base[1] + by, base[2] + bz), w))
    return out


def forward(shape, h, so, dt, nt, vp, nbl, src, wav, rec):
    n0, n1, n2 = shape
    r = so // 2
    c = [float(x) for x in D2[so]]
    vmax = max(vp[x][y][z] for x in range(n0) for y in range(n1) for z in range(n2))
    ex = sponge(n0, nbl, h[0], vmax)
    ey = sponge(n1, nbl, h[1], vmax)
    ez = sponge(n2, nbl, h[2], vmax)

    def zeros():
        return [[[0.0] * n2 for _ in range(n1)] for _ in range(n0)]

    def get(u, x, y, z):
        if 0 <= x < n0 and 0 <= y < n1 and 0 <= z < n2:
            return u[x][y][z]
        return 0.0

    up, uc = zeros(), zeros()
    traces = [[0.0] * len(rec) for _ in range(nt)]
    for n in range(nt):
        un = zeros()
        for x in range(n0):
            for y in range(n1):
                for z in range(n2):
                    sx = c[0] * uc[x][y][z]
                    sy = c[0] * uc[x][y][z]
                    sz = c[0] * uc[x][y][z]
                    for i in range(1, r + 1):
                        sx += c[i] * (get(uc, x + i, y, z) + get(uc, x - i, y, z))
                        sy += c[i] * (get(uc, x, y + i, z) + get(uc, x, y - i, z))
                        sz += c[i] * (get(uc, x, y, z + i) + get(uc, x, y, z - i))
                    lap = sx / h[0] ** 2 + sy / h[1] ** 2 + sz / h[2] ** 2
                    m = 1.0 / vp[x][y][z] ** 2
                    a = (ex[x] + ey[y] + ez[z]) * dt / 2.0
                    un[x][y][z] = (dt * dt * lap + m * (2.0 * uc[x][y][z] - up[x][y][z])
                                   + a * up[x][y][z]) / (m + a)
        for s, pt in enumerate(src):
            for (ix, iy, iz), w in corners(pt, shape, h):
                if w != 0.0:
                    un[ix][iy][iz] += w * wav[s][n] * dt * dt * vp[ix][iy][iz] ** 2
        for k, pt in enumerate(rec):
            acc = 0.0
            for (ix, iy, iz), w in corners(pt, shape, h):
                if w != 0.0:
                    acc += w * un[ix][iy][iz]
            traces[n][k] = acc
        up, uc = uc, un
    return traces, uc, up


# Centred first-derivative weights (c1..cr; antisymmetric) and staggered
# first-derivative weights (c1..cr for nodes at +-(i - 1/2)), closed rationals.
D1 = {
    4: [F(2, 3), F(-1, 12)],
    8: [F(4, 5), F(-1, 5), F(4, 105), F(-1, 280)],
    12: [F(6, 7), F(-15, 56), F(5, 63), F(-1, 56), F(1, 385), F(-1, 5544)],
}
STAG = {
    4: [F(9, 8), F(-1, 24)],
    8: [F(1225, 1024), F(-245, 3072), F(49, 5120), F(-5, 7168)],
}


def _shift(u, axis, off):
    """u[i + off] along `axis` with zeros outside the array (numpy)."""
    import numpy as np
    out = np.zeros_like(u)
    n = u.shape[axis]
    src = [slice(None)] * u.ndim
    dst = [slice(None)] * u.ndim
    if off >= 0:
        src[axis] = slice(off, n)
        dst[axis] = slice(0, n - off)
    else:
        src[axis] = slice(0, n + off)
        dst[axis] = slice(-off, n)
    out[tuple(dst)] = u[tuple(src)]
    return out


def dcentred(u, axis, so, h):
    """Centred first derivative (zero outside the array)."""
    acc = 0.0
    for i, c in enumerate(D1[so], start=1):
        acc = acc + float(c) * (_shift(u, axis, i) - _shift(u, axis, -i))
    return acc / h


def dstag_plus(u, axis, so, h):
    """Node -> half-node staggered derivative: sum c_k (u[i+k] - u[i-k+1]) / h."""
    acc = 0.0
    for k, c in enumerate(STAG[so], start=1):
        acc = acc + float(c) * (_shift(u, axis, k) - _shift(u, axis, -(k - 1)))
    return acc / h


def dstag_minus(u, axis, so, h):
    """Half-node -> node staggered derivative: sum c_k (u[i+k-1] - u[i-k]) / h."""
    acc = 0.0
    for k, c in enumerate(STAG[so], start=1):
        acc = acc + float(c) * (_shift(u, axis, k - 1) - _shift(u, axis, -k))
    return acc / h


def point_field(shape, h, pts, vals):
    """Trilinear spreading of one value per point onto the grid (numpy)."""
    import numpy as np
    f = np.zeros(shape)
    for pt, v in zip(pts, vals):
        for idx, w in corners(pt, shape, h):
            if w != 0.0:
                f[idx] += w * v
    return f


def sample(u, shape, h, pts):
    return [sum(w * u[idx] for idx, w in corners(pt, shape, h) if w != 0.0) for pt in pts]


def acoustic_2nd_order(shape, h, dt, nt, vp, eta, lap, src, wav, rec, src_term):
    """Leapfrog u^{n+1} = [dt^2 vp^2 ... ] with a caller's Laplacian (numpy).

    ``src_term(n)`` returns the field added to u^{n+1} after the update.
    Returns (traces [nt][nrec], u^nt)."""
    import numpy as np
    m = 1.0 / vp ** 2
    a = eta * dt / 2.0
    up = np.zeros(shape)
    uc = np.zeros(shape)
    tr = np.zeros((nt, len(rec)))
    for n in range(nt):
        un = (dt * dt * lap(uc) + m * (2.0 * uc - up) + a * up) / (m + a)
        un = un + src_term(n)
        tr[n] = sample(un, shape, h, rec)
        up, uc = uc, un
    return tr, uc
