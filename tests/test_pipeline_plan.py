"""The pipelined blocked schedule (host logic, no GPU): every time tile's
rows owned exactly once, every pass's inputs finished by earlier launches,
no pass overwriting rows another pass of its launch still reads, launches
within their CTA budget.

The rules follow from the leapfrog recurrence (Eq. 1) with a stencil of
radius r: u^{n+T} at row y depends on u^n at rows y - T r .. y + T r and on
u^{n-1} at rows y - (T - 1) r .. y + (T - 1) r.  Time tile t reads the two
fields tile t - 1 wrote and writes into the two fields tile t - 1 read."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2010_10248_gb300 import _tb
from paper_2010_10248_gb300 import build as tbbuild

TY, TZ = 16, 64


@pytest.fixture(scope="module")
def lib():
    return _tb.load(tbbuild.build())


def check_plan(p, n1, n2, so, T, K, cap):
    r = so // 2
    halo, reach = (T - 1) * r, T * r
    ntz = -(-n2 // TZ)
    launch, tile, y0, y1, yb0, nty, cta0 = (p[:, i] for i in range(7))
    assert np.all(np.diff(launch) >= 0) and launch[0] == 0
    nl = int(launch.max()) + 1
    # CTAs per launch and the computed rows of each pass
    for L in range(nl):
        sel = launch == L
        assert (nty[sel] * ntz).sum() <= cap
        assert sorted(cta0[sel]) == list(np.cumsum(np.r_[0, nty[sel] * ntz])[:-1])
        assert len(set(tile[sel])) == sel.sum() <= 2
        if sel.sum() == 2:  # the later tile follows the earlier one
            a, b = np.flatnonzero(sel)
            assert tile[b] == tile[a] + 1 and y0[b] == 0 and y1[a] == n1
    assert np.all(yb0 == np.maximum(0, y0 - halo))
    assert np.all(yb0 + nty * TY >= np.minimum(n1, y1 + halo))
    assert np.all(yb0 + (nty - 1) * TY < np.minimum(n1, y1 + halo))
    # every row of every tile owned exactly once
    done = np.full((K, n1), -1)
    for i in range(len(p)):
        assert np.all(done[tile[i], y0[i]:y1[i]] == -1)
        done[tile[i], y0[i]:y1[i]] = launch[i]
    assert np.all(done >= 0)
    for i in range(len(p)):
        t, L = tile[i], launch[i]
        if t == 0:
            continue
        # inputs: rows y0 - T r .. y1 + T r of tile t - 1, finished before
        lo, hi = max(0, y0[i] - reach), min(n1, y1[i] + reach)
        assert np.all(done[t - 1, lo:hi] < L), (i, t, L)
        # outputs go into the fields tile t - 1 read: in the same launch its
        # pass reads rows from its first owned row - T r on
        for j in np.flatnonzero((launch == L) & (tile == t - 1)):
            assert y1[i] <= y0[j] - reach, (i, j)
    return nl


@pytest.mark.parametrize("n1,n2,so,T,cap,per_tile", [
    (512, 512, 8, 3, 152, 1.78),   # the benchmark: 19 x 8 CTAs, 288 owned rows per launch
    (512, 512, 4, 4, 152, 1.78),
    (512, 512, 12, 2, 152, 1.78),
    (384, 384, 8, 3, 152, 1.0),    # one launch covers a time tile
])
def test_benchmark_grids(lib, n1, n2, so, T, cap, per_tile):
    K = 50
    p = _tb.tb_plan_pipeline(n1, n2, so, T, K, cap)
    nl = check_plan(p, n1, n2, so, T, K, cap)
    assert nl / K == pytest.approx(per_tile, abs=0.02)


def test_random_grids(lib):
    g = np.random.default_rng(2010)
    checked = shared = 0
    while checked < 300:
        so = int(g.choice([4, 8, 12]))
        T = int(g.integers(2, 5 if so < 12 else 3))
        n1 = int(g.integers(so + 2, 700))
        n2 = int(g.integers(so + 2, 700))
        ntz = -(-n2 // TZ)
        cap = int(ntz * g.integers(1, 25))
        K = int(g.integers(1, 12))
        try:
            p = _tb.tb_plan_pipeline(n1, n2, so, T, K, cap)
        except _tb.TBError:
            # only when a launch cannot hold one band: its tile rows cover at
            # most (T - 1) r rows beyond a band's overlap
            assert (cap // ntz) * TY <= 2 * (T - 1) * (so // 2)
            continue
        check_plan(p, n1, n2, so, T, K, cap)
        shared += int(np.sum(np.bincount(p[:, 0]) == 2))
        checked += 1
    assert shared > 100  # launches holding two time tiles were exercised


def test_bad_arguments(lib):
    for args in [(64, 64, 6, 3, 4, 16), (64, 64, 8, 1, 4, 16), (0, 64, 8, 3, 4, 16), (64, 64, 8, 3, 4, 0),
                 (96, 70, 8, 3, 4, 2)]:
        with pytest.raises(_tb.TBError):
            _tb.tb_plan_pipeline(*args)
