"""The TTI / elastic wavefront schedule (host logic, no GPU): replaying the
planner's launches over a model of every buffer the sub-updates read and
write must give each read the same writer as the one-step order, and no two
items of one launch may touch a value one of them writes.

Model (Eq. 2 and Eq. 3 as two sub-updates per step, Sec. II-B, Fig. 7b):
every sub-update reads the other sub-update's output within r planes along
axis 0 and its own fields on its own planes.  TTI: the flux pass reads p^n,
r^n and writes the fluxes F; the update pass reads F, p^n, p^{n-1}, r^n,
r^{n-1} and writes p^{n+1}, r^{n+1} over p^{n-1}, r^{n-1}.  Elastic: the
velocity pass reads the stresses and writes v in place; the stress pass
reads v and writes the stresses in place.  After each step's second pass
the sources are added to its output and the receivers read it."""
from __future__ import annotations

import itertools

import numpy as np
import pytest

from paper_2010_10248_gb300 import _tb
from paper_2010_10248_gb300 import build as tbbuild


@pytest.fixture(scope="module")
def lib():
    return _tb.load(tbbuild.build())


def accesses(physics, u, x0, x1, n0, r):
    """(reads, writes) of sub-update u on planes [x0, x1): sets of (buffer, plane)."""
    near = range(max(0, x0 - r), min(n0, x1 + r))
    own = range(x0, x1)
    if physics == "tti_fused":  # one sub-update per step, reaching 2r planes
        cur, prev = u % 2, (u + 1) % 2
        near2 = range(max(0, x0 - 2 * r), min(n0, x1 + 2 * r))
        reads = {(f"{b}{cur}", x) for b in "PR" for x in near2} | {(f"{b}{prev}", x) for b in "PR" for x in own}
        writes = {(f"{b}{prev}", x) for b in "PR" for x in own}
        return reads, writes
    k, second = divmod(u, 2)
    if physics == "tti":
        cur, prev = k % 2, (k + 1) % 2
        if not second:
            reads = {(f"{b}{cur}", x) for b in "PR" for x in near}
            writes = {("F", x) for x in own}
        else:
            reads = {("F", x) for x in near} | {(f"{b}{i}", x) for b in "PR" for i in (0, 1) for x in own}
            writes = {(f"{b}{prev}", x) for b in "PR" for x in own}
    else:
        if not second:
            reads = {("S", x) for x in near} | {("V", x) for x in own}
            writes = {("V", x) for x in own}
        else:
            reads = {("V", x) for x in near} | {("S", x) for x in own}
            writes = {("S", x) for x in own}
    return reads, writes


def post_accesses(physics, u, x0, x1):
    """injection (read-modify-write) and sampling of the step's output"""
    k = u if physics == "tti_fused" else u // 2
    bufs = [f"P{(k + 1) % 2}", f"R{(k + 1) % 2}"] if physics.startswith("tti") else ["S"]
    rw = {(b, x) for b in bufs for x in range(x0, x1)}
    return rw, rw


def run_onestep(physics, n0, r, U):
    seen, ver = {}, {}
    for u in range(U):
        ops = []
        for x in range(n0):  # the whole sub-update reads before anything of it is written
            ops.append(accesses(physics, u, x, x + 1, n0, r))
        for x, (rd, _) in enumerate(ops):
            seen[("op", u, x)] = {a: ver.get(a) for a in rd}
        for x, (_, wr) in enumerate(ops):
            for a in wr:
                ver[a] = ("op", u, a[1])
        if u % 2 or physics == "tti_fused":
            for x in range(n0):
                rd, wr = post_accesses(physics, u, x, x + 1)
                seen[("post", u, x)] = {a: ver.get(a) for a in rd}
                for a in wr:
                    ver[a] = ("post", u, a[1])
    return seen


def run_wave(physics, items, n0, r, U):
    seen, ver = {}, {}
    done = np.zeros((U, n0), dtype=int)
    for L, grp in itertools.groupby(items, key=lambda it: it[0]):
        grp = list(grp)
        acc = [accesses(physics, u, x0, x1, n0, r) for _, u, x0, x1 in grp]
        # items of one launch run concurrently: nothing one writes is touched by another
        for i, j in itertools.permutations(range(len(grp)), 2):
            assert not (acc[i][1] & (acc[j][0] | acc[j][1])), (L, grp[i], grp[j])
        # per plane: what the one-step op of that plane reads
        for (_, u, x0, x1) in grp:
            done[u, x0:x1] += 1
            for x in range(x0, x1):
                prd, _ = accesses(physics, u, x, x + 1, n0, r)
                seen[("op", u, x)] = {a: ver.get(a) for a in prd}
        for (_, u, x0, x1), (_, wr) in zip(grp, acc):
            for a in wr:
                ver[a] = ("op", u, a[1])
        posts = [(u, x0, x1) for _, u, x0, x1 in grp if u % 2 or physics == "tti_fused"]
        pacc = [post_accesses(physics, u, x0, x1) for u, x0, x1 in posts]
        for i, j in itertools.permutations(range(len(posts)), 2):
            assert not (pacc[i][1] & (pacc[j][0] | pacc[j][1]))
        for (u, x0, x1) in posts:
            for x in range(x0, x1):
                prd, _ = post_accesses(physics, u, x, x + 1)
                seen[("post", u, x)] = {a: ver.get(a) for a in prd}
        for (u, x0, x1), (_, wr) in zip(posts, pacc):
            for a in wr:
                ver[a] = ("post", u, a[1])
    assert np.all(done == 1)  # every plane of every sub-update exactly once
    return seen


@pytest.mark.parametrize("physics", ["tti", "elastic"])
@pytest.mark.parametrize("n0,r,slab,T", [(24, 2, 4, 2), (37, 4, 4, 2), (37, 4, 5, 3), (50, 4, 8, 4),
                                         (41, 6, 6, 2), (41, 6, 13, 3), (9, 4, 8, 2), (30, 2, 2, 8)])
def test_wavefront_replays_the_onestep_order(lib, physics, n0, r, slab, T):
    U = 2 * T
    items = [tuple(map(int, it)) for it in _tb.tb_plan_wavefront(n0, slab, U)]
    assert [it[0] for it in items] == sorted(it[0] for it in items)
    ns = -(-n0 // slab)
    assert max(it[0] for it in items) + 1 == ns + 2 * (U - 1)
    assert all(it[0] == (it[2] // slab) + 2 * it[1] for it in items)
    ref = run_onestep(physics, n0, r, U)
    got = run_wave(physics, items, n0, r, U)
    assert got.keys() == ref.keys()
    for key in ref:
        assert got[key] == ref[key], key


@pytest.mark.parametrize("n0,r,slab,T", [(37, 2, 4, 3), (50, 4, 8, 4), (41, 6, 12, 2), (61, 4, 9, 8), (7, 4, 8, 3)])
def test_fused_tti_wavefront_replays_the_onestep_order(lib, n0, r, slab, T):
    """The fused TTI step is one sub-update per step reading p, r within 2r
    planes: slabs of at least 2r planes keep the same rules."""
    items = [tuple(map(int, it)) for it in _tb.tb_plan_wavefront(n0, slab, T)]
    ref = run_onestep("tti_fused", n0, r, T)
    got = run_wave("tti_fused", items, n0, r, T)
    assert got == ref


def test_fused_tti_slabs_thinner_than_its_reach_would_race(lib):
    items = [tuple(map(int, it)) for it in _tb.tb_plan_wavefront(40, 6, 4)]  # r = 4 reaches 8 planes
    with pytest.raises(AssertionError):
        run_wave("tti_fused", items, 40, 4, 4)


def test_skew_one_would_race(lib):
    """The planted schedule with sub-update u of slab s in launch s + u puts a
    reader and the writer of its input in one launch."""
    n0, r, slab, U = 24, 4, 4, 4
    items = sorted((s + u, u, s * slab, min(n0, (s + 1) * slab)) for u in range(U) for s in range(-(-n0 // slab)))
    with pytest.raises(AssertionError):
        run_wave("elastic", items, n0, r, U)


def test_slab_thinner_than_the_stencil_would_read_stale_values(lib):
    """With slabs thinner than r an item reads planes two slabs away, whose
    sub-update runs in the same launch or later."""
    n0, r, U = 24, 4, 4
    items = [tuple(map(int, it)) for it in _tb.tb_plan_wavefront(n0, 2, U)]
    with pytest.raises(AssertionError):
        run_wave("tti", items, n0, r, U)


def test_bad_arguments(lib):
    for args in [(0, 4, 4), (16, 0, 4), (16, 4, 0)]:
        with pytest.raises(_tb.TBError):
            _tb.tb_plan_wavefront(*args)
