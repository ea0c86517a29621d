"""The sweep kernel's source table layout (host logic, no GPU): for any set
of grid points, the lookup the fused steps make (column pair of the lane,
plane offset from the pair's first plane, below its span) finds each point's
own slot, slots are distinct, pairs without points are empty, and the table
row holds exactly the pairs' plane ranges (Sec. II-A, grid-aligned
injection)."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2010_10248_gb300 import _tb
from paper_2010_10248_gb300 import build as tbbuild


@pytest.fixture(scope="module")
def lib():
    return _tb.load(tbbuild.build())


def check_layout(lin, n0, n1, n2):
    ev, slot, nev = _tb.tb_source_event_layout(lin, n1, n2)
    npair = (n2 + 1) // 2
    x, y, z = lin // (n1 * n2), (lin // n2) % n1, lin % n2
    first = ev[:, 0] & 0xFFFF
    span = (ev[:, 0] >> 16) & 0xFFFF
    base = ev[:, 1]
    pair = y * npair + z // 2
    # the kernel's test: off = x - first < span, then the value at 2 (base + off) + c
    off = x - first[pair]
    assert np.all((off >= 0) & (off < span[pair]))
    np.testing.assert_array_equal(slot, 2 * (base[pair] + off) + (z & 1))
    assert len(np.unique(slot)) == len(lin)
    assert np.all((slot >= 0) & (slot < 2 * nev))
    # ranges: from the first to the last point of the pair; empty pairs are zero
    used = np.zeros(len(ev), bool)
    used[pair] = True
    assert np.all(ev[~used] == 0)
    for p in np.flatnonzero(used):
        xs = x[pair == p]
        assert first[p] == xs.min() and span[p] == xs.max() - xs.min() + 1
    assert nev == int(span[used].sum())
    # the ranges tile [0, nev) without overlap
    order = np.argsort(base[used])
    b, s = base[used][order], span[used][order]
    assert b[0] == 0 and np.all(b[1:] == (b + s)[:-1])
    return nev


def unique_points(x, y, z, n1, n2):
    return np.unique((x.astype(np.int64) * n1 + y) * n2 + z)


@pytest.mark.parametrize("seed", range(6))
def test_random_point_sets(lib, seed):
    g = np.random.default_rng(seed)
    n0, n1, n2 = (int(v) for v in g.integers(8, 90, size=3))
    kind = seed % 3
    m = int(g.integers(1, 400))
    if kind == 0:    # dense: anywhere
        x, y, z = g.integers(0, n0, m), g.integers(0, n1, m), g.integers(0, n2, m)
    elif kind == 1:  # a horizontal plane: one depth (axis 2)
        d = int(g.integers(0, n2))
        x, y, z = g.integers(0, n0, m), g.integers(0, n1, m), np.full(m, d)
    else:            # a few columns with points along axis 0 (gaps inside the ranges)
        cols = g.integers(0, n1 * n2, 5)
        c = cols[g.integers(0, 5, m)]
        x, y, z = g.integers(0, n0, m), c // n2, c % n2
    lin = unique_points(x, y, z, n1, n2)
    check_layout(lin, n0, n1, n2)


def test_odd_last_column_and_single_point(lib):
    n0, n1, n2 = 20, 7, 9   # the last column (z = 8) has no partner
    lin = unique_points(np.array([3, 4, 19]), np.array([6, 6, 0]), np.array([8, 8, 0]), n1, n2)
    assert check_layout(lin, n0, n1, n2) == 2 + 1
    assert check_layout(lin[:1], n0, n1, n2) == 1


def test_empty_and_bad_arguments(lib):
    ev, slot, nev = _tb.tb_source_event_layout(np.zeros(0, np.int64), 4, 6)
    assert nev == 0 and not ev.any() and len(slot) == 0
    with pytest.raises(_tb.TBError):
        _tb.tb_source_event_layout(np.array([-1]), 4, 6)
    with pytest.raises(_tb.TBError):  # a plane beyond 16 bits
        _tb.tb_source_event_layout(np.array([70000 * 4 * 6]), 4, 6)
