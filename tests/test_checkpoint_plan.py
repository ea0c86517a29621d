"""The binomial checkpoint schedule of the adjoint gradient (host only).

The schedule (tb_plan_checkpoints) reverses nt forward steps of the
second-order recurrence with S stored states X_n = (u^n, u^{n-1}).  Checked by
simulating it: every action finds its input state where it says, no more than
S slots are ever occupied, every forward step is reversed once in the order
nt-1 .. 0, and the number of forward steps is the minimum a brute-force
dynamic programme over all split points finds (Griewank's binomial bound).
A replay of the schedule on a scalar recurrence gives, at every reverse step,
the same three states as the stored trajectory.
"""
from __future__ import annotations

import sys
from functools import lru_cache

import pytest

from paper_2010_10248_gb300 import _tb

sys.setrecursionlimit(20000)
ZERO, WORK = -1, -2


@lru_cache(None)
def _min_advances(l, s):
    """Fewest advanced steps to reverse l steps with the first state held and
    s free slots, by trying every split point."""
    if l <= 1:
        return 0
    if s == 0:
        return l * (l - 1) // 2
    return min(m + _min_advances(l - m, s - 1) + _min_advances(m, s) for m in range(1, l))


def _simulate(nt, S, actions):
    held = {}          # slot -> step of the state it holds
    work = None
    reversed_steps = []
    fwd = 0
    for kind, a, b, src, dst in actions:
        have = 0 if src == ZERO else (work if src == WORK else held.get(src))
        assert have == a, (kind, a, b, src, dst, have)
        if kind == 0:
            assert b > a
            fwd += b - a
            if dst == WORK:
                work = b
            else:
                assert 0 <= dst < S and dst not in held, "slot in use"
                held[dst] = b
            assert len(held) <= S
        else:
            assert kind == 1 and a == b
            fwd += 1
            reversed_steps.append(a)
            # a slot is free once the steps above its state are reversed
            for k in [k for k, v in held.items() if v >= a]:
                if v_done(held[k], reversed_steps):
                    del held[k]
    assert reversed_steps == list(range(nt - 1, -1, -1))
    return fwd


def v_done(v, reversed_steps):
    return reversed_steps[-1] <= v


@pytest.mark.parametrize("nt,S", [(1, 1), (2, 1), (7, 1), (30, 0), (30, 2), (45, 3), (100, 4), (200, 6),
                                  (800, 32), (1500, 32), (64, 64), (10, 20)])
def test_schedule_valid_and_optimal(nt, S):
    acts, fsteps = _tb.tb_plan_checkpoints(nt, S)
    assert fsteps == _simulate(nt, S, acts.tolist())
    if nt <= 200:
        assert fsteps == nt + _min_advances(nt, S)


def test_closed_form_count_at_the_gradient_workload():
    # 800 steps, 32 states: t = 3 (C(36, 3) = 7140 >= 800 > C(35, 2) = 595),
    # 3 * 800 - C(36, 2) = 1770 advanced steps, plus one per reverse step
    _, fsteps = _tb.tb_plan_checkpoints(800, 32)
    assert fsteps == 1770 + 800


def test_replay_gives_the_stored_trajectory():
    """Run the schedule on u^{n+1} = f(u^n, u^{n-1}, n) (a nonlinear scalar
    stand-in for one forward step) and check the states handed to each
    reverse step against the trajectory computed straight through."""
    def f(u, up, n):
        return (1.7 * u - 0.8 * up + 0.01 * n * n) % 97.0

    nt, S = 57, 3
    traj = [0.0, 0.0]   # u^{-1}, u^0
    for n in range(nt):
        traj.append(f(traj[-1], traj[-2], n))
    u = lambda n: traj[n + 1]   # u^n
    acts, _ = _tb.tb_plan_checkpoints(nt, S)
    slots, work = {}, None
    for kind, a, b, src, dst in acts.tolist():
        x = (0.0, 0.0) if src == ZERO else (work if src == WORK else slots[src])
        if kind == 0:
            cur, prev = x
            for n in range(a, b):
                cur, prev = f(cur, prev, n), cur
            if dst == WORK:
                work = (cur, prev)
            else:
                slots[dst] = (cur, prev)
        else:
            nxt = f(x[0], x[1], a)
            assert (nxt, x[0], x[1]) == (u(a + 1), u(a), u(a - 1))


def test_bad_arguments():
    lib = _tb.load()
    assert lib.tb_plan_checkpoints(0, 4, None, 0, None) == -_tb.TB_EINVAL
    assert lib.tb_plan_checkpoints(10, -1, None, 0, None) == -_tb.TB_EINVAL
