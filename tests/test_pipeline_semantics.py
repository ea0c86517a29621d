"""The pipelined blocked schedule executed, in FP64 on the host (no GPU): the
passes that tb_plan_pipeline returns are run the way the sweep kernel runs
them (four wavefield buffers, time tile k reading the pair tile k - 1 wrote;
a pass reads its input rows plus the stencil reach, keeps its fused levels
zero outside its computed rows, and writes u^{n+T}, u^{n+T-1} for its owned
rows only), the two passes of a launch in either order and with reads of
the fields as the launch found them, since they run concurrently.  The result must equal plain one-step time stepping bit for
bit; with the next tile's first band started one launch early it must not.

The recurrence is Eq. 1 without sources and damping on an n0 x n1 grid
(axis 0 streamed, axis 1 banded), zero outside the grid."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2010_10248_gb300 import _tb
from paper_2010_10248_gb300 import build as tbbuild

TY = 16
C8 = np.array([-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0, -1.0 / 560.0])  # so8 second derivative


@pytest.fixture(scope="module")
def lib():
    return _tb.load(tbbuild.build())


def step(u, up, c2, lo, hi, r):
    """One step of rows [lo, hi) of axis 1 from u (zero outside the grid and
    wherever the caller left it zero); returns the new rows."""
    n0, n1 = u.shape
    z = np.zeros((n0 + 2 * r, n1 + 2 * r))
    z[r:r + n0, r:r + n1] = u
    uc = z[r:r + n0, r + lo:r + hi]
    lap = np.zeros_like(uc)
    for i in range(1, r + 1):
        lap += C8[i] * ((z[r + i:r + i + n0, r + lo:r + hi] - uc) + (z[r - i:r - i + n0, r + lo:r + hi] - uc))
        lap += C8[i] * ((z[r:r + n0, r + lo + i:r + hi + i] - uc) + (z[r:r + n0, r + lo - i:r + hi - i] - uc))
    return uc + (c2[:, lo:hi] * lap + (uc - up[:, lo:hi]))


def reference(u0, u1, c2, nsteps, r):
    n1 = u0.shape[1]
    prev, cur = u0.copy(), u1.copy()
    for _ in range(nsteps):
        nxt = np.zeros_like(cur)
        nxt[:, :] = step(cur, prev, c2, 0, n1, r)
        prev, cur = cur, nxt
    return prev, cur


def run_pass(fields, c2, tile, own0, own1, yb0, nty, T, r, n1, reads=None):
    """One pass of time tile `tile`: reads (u^n, u^{n-1}) from the pair tile
    `tile` - 1 wrote (from `reads` when given: the fields as they were when
    the launch started) and writes (u^{n+T}, u^{n+T-1}) into the other pair."""
    src = fields if reads is None else reads
    i_in = 0 if tile % 2 == 0 else 2
    i_out = 2 - i_in
    lo, hi = yb0, min(n1, yb0 + nty * TY)  # computed rows
    cur = np.zeros_like(fields[0])
    prev = np.zeros_like(fields[0])
    # level 0: the input fields over the computed rows and the box halo
    blo, bhi = max(0, lo - r), min(n1, hi + r)
    cur[:, blo:bhi] = src[i_in][:, blo:bhi]
    prev[:, blo:bhi] = src[i_in + 1][:, blo:bhi]
    levels = [prev, cur]
    for k in range(T):
        src_lo, src_hi = (blo, bhi) if k == 0 else (lo, hi)  # fused levels: zero outside the pass
        a = np.zeros_like(cur)
        a[:, src_lo:src_hi] = levels[-1][:, src_lo:src_hi]
        b = np.zeros_like(cur)
        b[:, lo:hi] = levels[-2][:, lo:hi]
        nxt = np.zeros_like(cur)
        nxt[:, lo:hi] = step(a, b, c2, lo, hi, r)
        levels.append(nxt)
    fields[i_out][:, own0:own1] = levels[-1][:, own0:own1]
    fields[i_out + 1][:, own0:own1] = levels[-2][:, own0:own1]


def execute(plan, u0, u1, c2, T, r, order):
    n1 = u0.shape[1]
    fields = [u1.copy(), u0.copy(), np.zeros_like(u0), np.zeros_like(u0)]  # (u^0, u^{-1}) in pair 0
    nl = int(plan[:, 0].max()) + 1
    for L in range(nl):
        rows = plan[plan[:, 0] == L]
        if order == "reversed":
            rows = rows[::-1]
        # "snapshot": every pass reads the fields as the launch found them (no
        # pass of a launch may depend on another's output); "plan" and
        # "reversed": live reads, the passes one after the other (no pass may
        # overwrite what the other one reads)
        reads = [f.copy() for f in fields] if order == "snapshot" else None
        for launch, tile, y0, y1, yb0, nty, _ in rows:
            run_pass(fields, c2, tile, y0, y1, yb0, nty, T, r, n1, reads)
    K = int(plan[:, 1].max()) + 1
    last = 0 if K % 2 == 0 else 2
    return fields[last + 1], fields[last]


def problem(n0, n1, seed):
    g = np.random.default_rng(seed)
    u0 = g.standard_normal((n0, n1)) * 1e-3
    u1 = u0 + g.standard_normal((n0, n1)) * 1e-4
    c2 = g.uniform(0.02, 0.12, (n0, n1))
    return u0, u1, c2


@pytest.mark.parametrize("n1,T,cap", [(96, 3, 5), (96, 2, 4), (130, 4, 8), (70, 3, 4)])
def test_pipelined_schedule_equals_stepping(lib, n1, T, cap):
    so, r, n0, K = 8, 4, 6, 7
    plan = _tb.tb_plan_pipeline(n1, 64, so, T, K, cap)
    assert np.any(np.bincount(plan[:, 0]) == 2)  # launches holding two time tiles
    u0, u1, c2 = problem(n0, n1, n1 + T)
    ref_prev, ref_cur = reference(u0, u1, c2, K * T, r)
    for order in ("plan", "reversed", "snapshot"):
        prev, cur = execute(plan, u0, u1, c2, T, r, order)
        np.testing.assert_array_equal(cur, ref_cur)
        np.testing.assert_array_equal(prev, ref_prev)


def test_starting_the_next_tile_one_launch_early_breaks_it(lib):
    """The planted mistake: every first band of a time tile runs one launch
    earlier, before the rows of the previous tile it depends on are done."""
    so, r, n0, n1, T, K, cap = 8, 4, 6, 96, 3, 7, 5
    plan = _tb.tb_plan_pipeline(n1, 64, so, T, K, cap).copy()
    two = np.flatnonzero(np.bincount(plan[:, 0]) == 2)
    early = np.isin(plan[:, 0], two) & (plan[:, 2] == 0)
    plan[early, 0] -= 1
    plan = plan[np.argsort(plan[:, 0], kind="stable")]
    u0, u1, c2 = problem(n0, n1, 1)
    _, ref_cur = reference(u0, u1, c2, K * T, r)
    _, cur = execute(plan, u0, u1, c2, T, r, "snapshot")
    assert not np.array_equal(cur, ref_cur)
