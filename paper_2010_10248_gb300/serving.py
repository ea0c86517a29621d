"""Shot serving with continuous batching on one GPU.

A request is one shot: its own grid, velocity model, sources, receivers and
step count.  The server keeps a fixed set of slots; each slot owns a CUDA
stream and a propagator handle (wavefields and model resident on the device
for the life of the shot).  Requests are admitted in arrival order whenever a
slot is free and the shot's device footprint fits in the memory budget;
admitted shots run concurrently on their streams, so the kernels of small
shots fill the GPU together while a large shot runs beside them or alone
(when its footprint leaves no room).  A slot frees as soon as its shot's
traces are on the host; the next waiting request enters at once, without
waiting for the other shots in flight.

Small FP32 shots (at most ``batch_points`` grid points) do not take a slot:
they join a batch lane (one per space order), where every time step of every
shot in the lane is one launch of the one-step sweep over all of them
(tb_batch_*).  The lane advances in chunks of ``batch_chunk`` steps; shots
join and leave at chunk boundaries while the others keep running
(continuous batching inside one launch).  Large shots run alone on a slot's
stream with the temporally blocked sweep.

Latency of a shot = time from its arrival to its traces being ready on the
host.  The kernels are deterministic, so a shot gives bit-identical traces
alone and in any mix.
"""
from __future__ import annotations

import heapq
import time
from dataclasses import dataclass, field

import numpy as np

from . import _tb


@dataclass
class ShotRequest:
    """One propagation problem.  Arrays are host numpy arrays."""
    shape: tuple
    spacing: tuple
    space_order: int
    vp: object              # [n0, n1, n2] float32: numpy array, CUDA tensor, or a
                            # callable returning one when the shot is admitted
    src_xyz: np.ndarray     # [nsrc, 3] float64 metres
    wavelet_f0: float       # Ricker peak frequency (sampled with the shot's dt)
    rec_xyz: np.ndarray     # [nrec, 3] float64 metres
    nt: int
    nbl: int = 0
    time_tile: int = 0      # 0: blocked sweep with the default tile; 1: one-step
    arrival: float = 0.0    # seconds after the start of the run
    tag: object = None
    storage: int = 0        # wavefield storage: 0 FP32, 1 FP16, 2 BF16 (one-step)


@dataclass
class ShotResult:
    tag: object
    traces: np.ndarray
    dt: float
    arrival: float
    start: float
    done: float

    @property
    def latency(self) -> float:
        return self.done - self.arrival


def footprint_bytes(req: ShotRequest) -> int:
    """Device bytes a shot holds while it runs: four FP32 wavefield buffers
    (or two 16-bit ones) and the c2 field (padded rows), sponge tables,
    inspector tables, the receiver staging rows and the trace buffer, plus the
    blocked sweep's halo ring."""
    n0, n1, n2 = (int(s) for s in req.shape)
    if req.storage in (1, 2):
        n2p = (n2 + 7) // 8 * 8
        fields = (2 * 2 + 4) * n0 * n1 * n2p
    else:
        n2p = (n2 + 3) // 4 * 4
        fields = 5 * 4 * n0 * n1 * n2p
    nrec = len(req.rec_xyz)
    tables = 64 * 8 * (len(req.src_xyz) + nrec) + 8 * n1 * n2
    rec_rows = 16 * 4 * 8 * nrec
    traces = 4 * req.nt * nrec
    ring = 4 * ((n1 + 15) // 16 + 2) * ((n2 + 63) // 64) * 3 * 10 * 8 * 72
    return fields + tables + rec_rows + traces + ring + (8 << 20)


def _pinned(torch, a, dtype):
    """A pinned host copy of a numpy array (the library's copies from it are
    asynchronous, unlike from pageable memory)."""
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).pin_memory()


def _setup(torch, req: ShotRequest, stream, time_tile):
    """Propagator with the shot's model and geometry set on `stream`; returns
    (propagator, dt, pinned inputs kept alive until the stream passes them)."""
    from . import Propagator
    p = Propagator(req.shape, req.spacing, req.space_order, nbl=req.nbl, time_tile=time_tile,
                   storage=req.storage)
    vp = req.vp() if callable(req.vp) else req.vp
    if not (hasattr(vp, "is_cuda") and vp.is_cuda):
        vp = _pinned(torch, vp, np.float32)
    src = _pinned(torch, req.src_xyz, np.float64)
    rec = _pinned(torch, req.rec_xyz, np.float64)
    _tb.tb_set_model(p.h, vp, None, None, 0.0, stream)
    dt = _tb.tb_get_dt(p.h)
    w = _ricker(req.wavelet_f0, dt, req.nt)
    wav = _pinned(torch, np.repeat(w[None, :], len(req.src_xyz), axis=0), np.float32)
    _tb.tb_set_sources(p.h, len(req.src_xyz), src, req.nt, wav, stream)
    _tb.tb_set_receivers(p.h, len(req.rec_xyz), rec, stream)
    return p, dt, (vp, src, rec, wav)


class _Slot:
    def __init__(self, torch):
        self.torch = torch
        self.stream = torch.cuda.Stream()
        self.done_event = None
        self.prop = None
        self.req = None
        self.start = 0.0
        self.host_traces = None
        self.bytes = 0

    def launch(self, req: ShotRequest, t0: float):
        torch = self.torch
        self.req = req
        self.start = time.perf_counter() - t0
        with torch.cuda.stream(self.stream):
            st = self.stream
            self.prop, dt, self.staged = _setup(torch, req, st, req.time_tile if req.storage == 0 else 1)
            p = self.prop
            dev_tr = torch.empty((req.nt, len(req.rec_xyz)), dtype=torch.float32, device="cuda")
            sched = _tb.TB_BLOCKED if (req.time_tile != 1 and req.storage == 0) else _tb.TB_ONESTEP
            _tb.tb_forward(p.h, req.nt, dev_tr, sched, st)
            self.host_traces = torch.empty(dev_tr.shape, dtype=torch.float32, pin_memory=True)
            self.host_traces.copy_(dev_tr, non_blocking=True)
            self.dev_tr = dev_tr
            self.dt = dt
            self.done_event = torch.cuda.Event()
            self.done_event.record(self.stream)

    def ready(self) -> bool:
        return self.done_event is not None and self.done_event.query()

    def finish(self, t0: float) -> ShotResult:
        r = ShotResult(self.req.tag, self.host_traces.numpy().copy(), self.dt, self.req.arrival,
                       self.start, time.perf_counter() - t0)
        self.prop.close()
        self.prop = None
        self.req = None
        self.done_event = None
        self.dev_tr = None
        self.staged = None
        return r


class _BatchLane:
    """Small FP32 shots of one space order advanced together (tb_batch): one
    launch per time step covers every shot in the lane; shots join and leave
    between chunks of `chunk` steps."""

    def __init__(self, torch, max_shots, chunk):
        self.torch = torch
        self.stream = torch.cuda.Stream()
        self.batch = _tb.Batch(max_shots)
        self.max_shots = max_shots
        self.chunk = chunk
        self.shots = {}          # handle -> [req, prop, dev traces, start, staged, bytes]
        self.out = []            # finished: [req, prop, host traces, event, start, dt, bytes]
        self.chunk_event = None
        self.stats = {"launch_chunks": 0, "max_shots": 0}

    def free(self):
        return self.max_shots - len(self.shots)

    def admit(self, req: ShotRequest, t0: float, nbytes: int):
        torch = self.torch
        start = time.perf_counter() - t0
        with torch.cuda.stream(self.stream):
            prop, dt, staged = _setup(torch, req, self.stream, 1)
            dev_tr = torch.empty((req.nt, len(req.rec_xyz)), dtype=torch.float32, device="cuda")
            self.batch.add(prop.h, req.nt, dev_tr, self.stream)
        self.shots[prop.h] = [req, prop, dev_tr, start, staged, nbytes, dt]
        self.stats["max_shots"] = max(self.stats["max_shots"], len(self.shots))

    def busy(self) -> bool:
        return bool(self.shots) or bool(self.out)

    def advance(self):
        """When the last chunk has finished: hand its finished shots' traces to
        the host (asynchronously) and enqueue the next chunk."""
        torch = self.torch
        if self.chunk_event is not None and not self.chunk_event.query():
            return
        self.chunk_event = None
        with torch.cuda.stream(self.stream):
            for hnd in self.batch.finished():
                req, prop, dev_tr, start, staged, nbytes, dt = self.shots.pop(hnd)
                host = torch.empty(dev_tr.shape, dtype=torch.float32, pin_memory=True)
                host.copy_(dev_tr, non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(self.stream)
                self.out.append([req, prop, host, ev, start, dt, nbytes, dev_tr])
            if self.batch.active():
                self.batch.step(self.chunk, self.stream)
                self.chunk_event = torch.cuda.Event()
                self.chunk_event.record(self.stream)
                self.stats["launch_chunks"] += 1

    def collect(self, t0: float):
        """Results whose traces are on the host, with their device bytes."""
        done = []
        for item in list(self.out):
            req, prop, host, ev, start, dt, nbytes, _ = item
            if ev.query():
                done.append((ShotResult(req.tag, host.numpy().copy(), dt, req.arrival, start,
                                        time.perf_counter() - t0), nbytes))
                prop.close()
                self.out.remove(item)
        return done


def _ricker(f0, dt, nt):
    t = np.arange(nt) * dt - 1.0 / f0
    a = (np.pi * f0 * t) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


class ShotServer:
    """Continuous-batching server: ``run(requests)`` processes a stream of
    requests (arrival times in ``ShotRequest.arrival``, seconds from the start)
    and returns their results in completion order."""

    def __init__(self, slots: int = 8, memory_budget: int | None = None, poll_s: float = 2e-4,
                 slot_factory=None, batch_points: int = 0, batch_max: int = 16, batch_chunk: int = 32):
        """``slot_factory`` (no arguments) makes the slots; by default a slot
        is a CUDA stream with a propagator.  Any object with ``bytes``,
        ``launch(req, t0)``, ``ready()`` and ``finish(t0)`` serves (the
        scheduling logic is tested with host-only slots).  ``batch_points``
        > 0: FP32 shots of at most that many grid points go to a batch lane
        of their space order (at most ``batch_max`` shots, advanced in chunks
        of ``batch_chunk`` steps) instead of a slot."""
        self.batch_points = int(batch_points)
        self.batch_max = int(batch_max)
        self.batch_chunk = int(batch_chunk)
        self.lanes = {}
        if slot_factory is None:
            import torch
            self._torch = torch
            self.slots = [_Slot(torch) for _ in range(slots)]
            if memory_budget is None:
                free, _ = torch.cuda.mem_get_info()
                memory_budget = int(free * 0.85)
        else:
            self.slots = [slot_factory() for _ in range(slots)]
            if memory_budget is None:
                raise ValueError("a memory budget is needed with a custom slot factory")
        self.budget = int(memory_budget)
        self.poll_s = poll_s
        self.stats = {"max_in_flight": 0, "max_bytes": 0}

    def run(self, requests):
        reqs = sorted(requests, key=lambda r: r.arrival)
        for r in reqs:
            if footprint_bytes(r) > self.budget:
                raise ValueError(f"shot {r.tag}: footprint {footprint_bytes(r)} exceeds the budget {self.budget}")
        pending = list(reqs)
        waiting = []      # arrived, not admitted (arrival order)
        results = []
        in_use = 0
        t0 = time.perf_counter()
        busy = []

        def lane_of(req):
            if self.batch_points <= 0 or req.storage != 0 or int(np.prod(req.shape)) > self.batch_points:
                return None
            if req.space_order not in self.lanes:
                self.lanes[req.space_order] = _BatchLane(self._torch, self.batch_max, self.batch_chunk)
            return self.lanes[req.space_order]

        def lanes_busy():
            return any(ln.busy() for ln in self.lanes.values())

        while pending or waiting or busy or lanes_busy():
            now = time.perf_counter() - t0
            while pending and pending[0].arrival <= now:
                waiting.append(pending.pop(0))
            # retire finished shots (frees their slot and memory at once)
            for s in list(busy):
                if s.ready():
                    in_use -= s.bytes
                    results.append(s.finish(t0))
                    busy.remove(s)
            for ln in self.lanes.values():
                for res, nbytes in ln.collect(t0):
                    in_use -= nbytes
                    results.append(res)
            # admit in arrival order while a slot (or lane place) is free and
            # the shot fits
            while waiting:
                need = footprint_bytes(waiting[0])
                if in_use + need > self.budget:
                    break
                lane = lane_of(waiting[0])
                if lane is not None:
                    if lane.free() <= 0:
                        break
                    req = waiting.pop(0)
                    in_use += need
                    lane.admit(req, t0, need)
                else:
                    free_slots = [s for s in self.slots if s not in busy]
                    if not free_slots:
                        break
                    req = waiting.pop(0)
                    slot = free_slots[0]
                    slot.bytes = need
                    in_use += need
                    slot.launch(req, t0)
                    busy.append(slot)
                inflight = len(busy) + sum(len(ln.shots) for ln in self.lanes.values())
                self.stats["max_in_flight"] = max(self.stats["max_in_flight"], inflight)
                self.stats["max_bytes"] = max(self.stats["max_bytes"], in_use)
            for ln in self.lanes.values():
                ln.advance()
            if busy or waiting or pending or lanes_busy():
                nxt = pending[0].arrival - (time.perf_counter() - t0) if pending and not waiting else 0
                active = busy or lanes_busy()
                time.sleep(min(self.poll_s, max(nxt, 0.0)) if active else max(min(nxt, 0.01), 0.0))
        self.stats["lanes"] = {so: ln.stats for so, ln in self.lanes.items()}
        return results


def percentile(values, q):
    v = np.sort(np.asarray(values, dtype=np.float64))
    if v.size == 0:
        return float("nan")
    return float(np.percentile(v, q))
