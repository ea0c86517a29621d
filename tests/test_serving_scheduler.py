"""The shot server's scheduling (host logic, no GPU): shots are admitted in
arrival order, never beyond the slot count or the memory budget, every shot
completes once, and a shot larger than the budget is refused up front.  The
slots are host-only stand-ins that "run" for a given time."""
from __future__ import annotations

import time

import numpy as np
import pytest

from paper_2010_10248_gb300 import serving


class Monitor:
    def __init__(self):
        self.running = {}
        self.launch_order = []
        self.max_slots = 0
        self.max_bytes = 0


class FakeSlot:
    def __init__(self, mon: Monitor):
        self.mon = mon
        self.bytes = 0
        self.req = None
        self.end = 0.0
        self.start = 0.0

    def launch(self, req, t0):
        self._t0 = t0  # the server's start (perf_counter seconds)
        now = time.perf_counter() - t0
        assert req.arrival <= now + 1e-9  # never before the shot arrived
        self.req, self.start, self.end = req, now, now + req.tag["run_s"]
        self.mon.running[id(self)] = self.bytes
        self.mon.launch_order.append(req.tag["i"])
        self.mon.max_slots = max(self.mon.max_slots, len(self.mon.running))
        self.mon.max_bytes = max(self.mon.max_bytes, sum(self.mon.running.values()))

    def ready(self):
        return self.req is not None and time.perf_counter() >= self._t0 + self.end

    def finish(self, t0):
        del self.mon.running[id(self)]
        r = serving.ShotResult(self.req.tag, np.zeros((1, 1), np.float32), 1e-3, self.req.arrival, self.start,
                               time.perf_counter() - t0)
        self.req = None
        return r


def make_requests(n, seed):
    g = np.random.default_rng(seed)
    reqs, t = [], 0.0
    for i in range(n):
        t += float(g.exponential(0.006))
        shape = tuple(int(32 * g.integers(4, 17)) for _ in range(3))
        nrec = int(g.integers(100, 5000))
        reqs.append(serving.ShotRequest(shape, (10.0, 10.0, 10.0), 8, None, np.zeros((1, 3)), 15.0,
                                        np.zeros((nrec, 3)), nt=int(g.integers(300, 1500)), arrival=t,
                                        storage=int(g.integers(0, 2)),
                                        tag={"i": i, "run_s": float(g.uniform(0.005, 0.03))}))
    return reqs


def run_server(reqs, slots, budget):
    mon = Monitor()
    srv = serving.ShotServer(slots=slots, memory_budget=budget, poll_s=1e-4, slot_factory=lambda: FakeSlot(mon))
    return srv.run(reqs), mon, srv


@pytest.mark.parametrize("slots,budget_shots", [(4, 2.5), (8, 6.0), (3, 100.0)])
def test_admission_order_slots_and_budget(slots, budget_shots):
    reqs = make_requests(40, 7 + slots)
    sizes = [serving.footprint_bytes(r) for r in reqs]
    budget = int(max(sizes) * budget_shots)
    results, mon, srv = run_server(reqs, slots, budget)
    assert sorted(r.tag["i"] for r in results) == list(range(len(reqs)))   # every shot, once
    assert mon.launch_order == sorted(mon.launch_order)                   # arrival (FIFO) order
    assert mon.max_slots <= slots
    assert mon.max_bytes <= budget
    assert srv.stats["max_bytes"] <= budget and srv.stats["max_in_flight"] <= slots
    for r in results:
        assert r.start >= r.arrival - 1e-9 and r.done >= r.start
    if budget_shots >= 100.0:
        assert mon.max_slots == slots  # with memory to spare the slots are the limit


def test_oversized_shot_is_refused():
    reqs = make_requests(3, 1)
    budget = min(serving.footprint_bytes(r) for r in reqs) - 1
    with pytest.raises(ValueError):
        run_server(reqs, 2, budget)


def test_footprint_grows_with_the_problem():
    base = make_requests(1, 2)[0]
    big = serving.ShotRequest(tuple(2 * s for s in base.shape), base.spacing, 8, None, base.src_xyz, 15.0,
                              base.rec_xyz, nt=base.nt, storage=base.storage)
    half = serving.ShotRequest(base.shape, base.spacing, 8, None, base.src_xyz, 15.0, base.rec_xyz, nt=base.nt,
                               storage=1)
    full = serving.ShotRequest(base.shape, base.spacing, 8, None, base.src_xyz, 15.0, base.rec_xyz, nt=base.nt,
                               storage=0)
    assert serving.footprint_bytes(big) > 7 * serving.footprint_bytes(base) * 0.9
    assert serving.footprint_bytes(half) < serving.footprint_bytes(full)
