"""Benchmark: temporally blocked acoustic propagation, 512^3, space order 8.

One bench step is one whole shot through the C ABI: model setup (CFL step,
sponge, c2), the source and receiver inspectors, and tb_forward over 1000
time steps with the blocked schedule (receiver traces included).  The metric
is grid-point updates per second (N * nt / step time).  The one-step
spatially blocked kernel is timed in the same run for comparison.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the FP64 CPU oracle (the only other implementation of
this method; there is no reference code) on a bounded sample of the same
workload.  Under torchrun (N > 1) every rank runs an independent replica of
the shot on its own GPU (the path has no data exchange between shots).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GPts/s blocked vs spatial-blocked at rel-L2<=1e-4; shot p50/p99 latency"
UNIT = "GPts/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--size", type=int, default=512, help="cube edge (512 = the benchmark)")
    ap.add_argument("--nt", type=int, default=1000)
    ap.add_argument("--time-tile", type=int, default=3)  # the fastest fused depth at 512^3 so8
    ap.add_argument("--space-order", type=int, default=8, choices=[4, 8, 12],
                    help="the benchmark model at another space order (the headline is so8)")
    ap.add_argument("--no-onestep", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-steps", type=int, default=8)
    ap.add_argument("--serving", action="store_true",
                    help="Poisson stream of acoustic so8 shots of mixed sizes through the continuous-"
                         "batching server: p50/p99 shot latency and aggregate GPts/s")
    ap.add_argument("--shots", type=int, default=500)
    ap.add_argument("--storage", default="f32", choices=["f32", "f16", "bf16", "plain"],
                    help="f16 / bf16 / plain: the 512^3 acoustic shot with 16-bit (or plain FP32) wavefield "
                         "storage in the streaming one-step kernel")
    ap.add_argument("--slots", type=int, default=8)
    ap.add_argument("--adjoint", action="store_true",
                    help="vp gradient of the 256^3 so8 shot (800 steps, 32 checkpoints) instead")
    ap.add_argument("--many-sources", action="store_true",
                    help="blocked vs one-step with many sources on a plane and spread through the grid")
    ap.add_argument("--wave-tile", type=int, default=16, help="TTI / elastic: steps per wavefront")
    ap.add_argument("--slab", type=int, default=0, help="TTI / elastic: planes per wavefront slab (0: auto)")
    ap.add_argument("--tti-fused", action="store_true", help="TTI: both passes of a step in one kernel")
    ap.add_argument("--stream-l1", action="store_true", help="TTI / elastic: the L1 streaming kernels")
    ap.add_argument("--physics", default="acoustic", choices=["acoustic", "tti", "elastic"],
                    help="tti / elastic: the 384^3 so8 500-step TTI or elastic workload, one-step "
                         "schedule (the headline line is the acoustic one)")
    return ap.parse_args()


def max_over_ranks(ms, dist, device):
    """Step time of the slowest rank (the whole job ends when it ends)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(points_per_rank_step, steps, ms, world):
    """Whole-job GPts/s: every rank runs an independent replica, so the units
    of all ranks count, over the slowest rank's time."""
    return world * points_per_rank_step * steps / (ms * 1e-3) / 1e9


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("tb_sweep.cuh", "tb_async.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2010_10248_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs"), "measured"
    return 6800.0, "fallback"


def ncu_counters(kernel_key):
    """The committed ncu figures of a sweep kernel (DRAM bytes per full-size
    launch, warp instructions per point update), if they were taken on the
    current kernel source; else an empty dict."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return {}
    e = json.load(open(p)).get(kernel_key)
    if not e or e.get("source_hash") != kernel_source_hash():
        return {}
    return e


def fp32_peak_tflops(nsm):
    """FP32 FMA peak from unit counts and the maximum SM clock: 128 FP32
    lanes per SM, 2 flops per FMA."""
    mhz = 2070.0
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        mhz = float(json.load(open(p)).get("sm_max_mhz", mhz))
    return nsm * 128 * 2 * mhz * 1e6 / 1e12, mhz


def alg_flops(space_order):
    """Algorithmic flops per point and step of Eq. 1: per axis r pair sums
    and r multiply-adds (3 flops per pair), the centre and axis sums, and the
    leapfrog update with damping (~8)."""
    r = space_order // 2
    return 9 * r + 10


def cpu_oracle_rate(w, dt, steps_a, steps_b):
    """GPts/s of the FP64 oracle on the host, from the difference of two runs
    (removes its serial setup); returns (rate, seconds, threads)."""
    import oracle
    oracle.build()
    wav = w.wavelets(dt)
    vp64 = w.vp.astype(np.float64)
    N = int(np.prod(w.shape))
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    t = []
    for s in (steps_a, steps_b):
        t0 = time.perf_counter()
        oracle.acoustic_forward(w.shape, w.spacing, w.so, dt, s, vp64, nbl=w.nbl,
                                src_xyz=w.src_xyz, src_wav=wav[:, :s], rec_xyz=w.rec_xyz,
                                nthreads=threads)
        t.append(time.perf_counter() - t0)
    dtime = max(t[1] - t[0], 1e-9)
    return N * (steps_b - steps_a) / dtime / 1e9, t[0] + t[1], threads


def cpu_oracle_rate_physics(physics, mk, size, steps_a, steps_b):
    """GPts/s of the FP64 TTI or elastic oracle on the host, on the same
    recipe at a reduced cube edge (difference of two runs); returns (rate,
    seconds, threads, sample description)."""
    import oracle
    oracle.build()
    w = mk(shape=(size,) * 3, nt=steps_b)
    aux = [a.astype(np.float64) for a in w.meta["aux"]]
    vp64 = w.vp.astype(np.float64)
    if physics == "tti":
        dt = 0.8 * oracle.tti_dt_max(w.so, w.spacing, float(w.vp.max()), float(aux[0].max()))
    else:
        dt = 0.8 * oracle.elastic_dt_max(w.so, w.spacing, float(w.vp.max()))
    wav = w.wavelets(dt)
    t = []
    for s in (steps_a, steps_b):
        t0 = time.perf_counter()
        if physics == "tti":
            oracle.tti_forward(w.shape, w.spacing, w.so, dt, s, vp64, *aux, nbl=w.nbl, src_xyz=w.src_xyz,
                               src_wav=wav[:, :s], rec_xyz=w.rec_xyz)
        else:
            oracle.elastic_forward(w.shape, w.spacing, w.so, dt, s, vp64, *aux, nbl=w.nbl, src_xyz=w.src_xyz,
                                   src_wav=wav[:, :s], rec_xyz=w.rec_xyz)
        t.append(time.perf_counter() - t0)
    dtime = max(t[1] - t[0], 1e-9)
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    N = size ** 3
    sample = (f"{physics} {size}^3 so{w.so}, {steps_b - steps_a} steps (difference of a {steps_a}- and a "
              f"{steps_b}-step FP64 oracle run, {t[0] + t[1]:.1f} s total)")
    return N * (steps_b - steps_a) / dtime / 1e9, t[0] + t[1], threads, sample


def bench_config(w, args, ws):
    """The workload of the headline line (the same dict in both arms)."""
    return {"workload": w.name, "grid": list(w.shape), "space_order": w.so, "nt": w.nt,
            "time_tile": args.time_tile, "receivers": len(w.rec_xyz), "sources": len(w.src_xyz),
            "schedule": "blocked", "parallelism": f"replicas x{ws}",
            "l2": "inputs larger than L2 (512 MiB per field, 5 fields)",
            "step": "set_model + set_sources + set_receivers + forward(nt)"}


def oracle_full_runs():
    """Whole runs of the FP64 oracle (setup included) on one thread and on
    every host core: the 64^3 so4 100-step workload and the 512^3 recipe at
    128^3 so8 for 1000 steps.  Returns a list of dicts."""
    import oracle
    from paper_2010_10248_gb300 import workloads as wl
    oracle.build()
    cores = os.cpu_count() or 1
    rows = []
    for w in (wl.acoustic_64_so4(), wl.acoustic_512_so8(shape=(128, 128, 128), nt=1000, nbl=10)):
        dt = 0.8 * oracle.cfl_dt_max(w.so, w.spacing, float(w.vp.max()))
        wav = w.wavelets(dt)
        N = int(np.prod(w.shape))
        for nth in (1, cores):
            t0 = time.perf_counter()
            oracle.acoustic_forward(w.shape, w.spacing, w.so, dt, w.nt, w.vp.astype(np.float64),
                                    nbl=w.nbl, src_xyz=w.src_xyz, src_wav=wav, rec_xyz=w.rec_xyz,
                                    nthreads=nth)
            el = time.perf_counter() - t0
            rows.append({"workload": w.name, "threads": nth, "seconds": el,
                         "gpts": N * w.nt / el / 1e9, "run": "full (setup included)"})
    return rows


def run_reference(args):
    """The FP64 oracle on the host cores, on a bounded sample of the benchmark
    workload.  One bench step = a 2-step and a (2 + cpu_steps)-step oracle run;
    value = grid-point updates of the extra steps over the extra time (the
    same definition as the native line's cpu_baseline: setup excluded), and
    ms_per_step = the wall time of the two runs (what the step ran)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from paper_2010_10248_gb300 import workloads as wl
    import oracle
    w = wl.acoustic_512_so8(shape=(args.size,) * 3, nt=args.nt)
    dt = 0.8 * oracle.cfl_dt_max(w.so, w.spacing, float(w.vp.max()))
    table = [] if args.no_cpu else oracle_full_runs()
    rates, walls = [], []
    threads = 1
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        rate, _, threads = cpu_oracle_rate(w, dt, 2, 2 + args.cpu_steps)
        el = time.perf_counter() - t0
        if i >= args.warmup:
            rates.append(rate)
            walls.append(el)
    v = float(np.median(rates))
    sample = (f"{w.shape[0]}^3 so8 with all {len(w.rec_xyz)} receivers: per bench step a 2-step and a "
              f"{2 + args.cpu_steps}-step FP64 oracle run (Listing 1 form), rate = {args.cpu_steps} steps "
              f"x N over the difference of their times (setup excluded); ms_per_step is the wall time "
              f"of the two runs, not of the {w.nt}-step workload")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": float(np.mean(walls)) * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(w, args, ws),
            "sample_steps_per_bench_step": 4 + args.cpu_steps,
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "oracle_full_runs": table, "nproc": os.cpu_count()}
    print(json.dumps(line), flush=True)


def run_native(args):
    import torch
    import paper_2010_10248_gb300 as tb
    from paper_2010_10248_gb300 import build as tbbuild
    from paper_2010_10248_gb300 import workloads as wl

    ws, rank, local = dist_env()
    dist = None
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(local)
    if rank == 0:
        tbbuild.build()
    if dist:
        dist.barrier()
    tb.load()
    dev = torch.device("cuda", local)

    w = wl.acoustic_512_so8(shape=(args.size,) * 3, nt=args.nt, so=args.space_order)
    N = int(np.prod(w.shape))
    nt = w.nt
    vp_dev = torch.from_numpy(w.vp).to(dev)
    src_dev = torch.from_numpy(w.src_xyz).to(dev)
    rec_dev = torch.from_numpy(w.rec_xyz).to(dev)
    nrec = len(w.rec_xyz)

    prop = tb.Propagator(w.shape, w.spacing, w.so, nbl=w.nbl, time_tile=args.time_tile,
                         profile=True)
    stream = torch.cuda.current_stream()
    prop.set_model(vp_dev)
    dt = prop.dt
    wav_dev = torch.from_numpy(w.wavelets(dt).astype(np.float32)).to(dev)
    traces = torch.empty((nt, nrec), dtype=torch.float32, device=dev)

    def shot(schedule, traces_out=traces, vp=vp_dev, src=src_dev, wav=wav_dev, rec=rec_dev):
        h = prop.h
        tb.tb_set_model(h, vp, None, None, 0.0, stream)
        tb.tb_set_sources(h, len(w.src_xyz), src, nt, wav, stream)
        tb.tb_set_receivers(h, nrec, rec, stream)
        tb.tb_forward(h, nt, traces_out, tb.TB_BLOCKED if schedule == "blocked" else tb.TB_ONESTEP,
                      stream)

    def timed(schedule, k, warm, **kw):
        for _ in range(warm):
            shot(schedule, **kw)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        l0 = tb.tb_launch_count()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        kt_ms, kt_n = 0.0, 0
        e0.record(stream)
        for _ in range(k):
            shot(schedule, **kw)
            n, ms = prop.kernel_time(0)  # sweep launches of this shot (synchronises)
            kt_ms += ms
            kt_n += n
        e1.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        ms = e0.elapsed_time(e1) / k
        launches = tb.tb_launch_count() - l0
        ms = max_over_ranks(ms, dist, dev)
        return ms, kt_ms / max(kt_n, 1), kt_n // k, launches

    clocks = ClockSampler(local)
    clocks.start()
    ms_b, kms_b, kl_b, launches = timed("blocked", args.steps, args.warmup)
    clk = clocks.stop()
    tr_blocked = traces.clone()
    value = job_rate(N, nt, ms_b, ws)

    out = {}
    if not args.no_onestep:
        ms_1, kms_1, kl_1, _ = timed("onestep", args.steps, args.warmup)
        out["onestep"] = {"value": N * nt / (ms_1 * 1e-3) / 1e9, "ms_per_step": ms_1,
                          "kernel_ms_per_launch": kms_1, "launches_per_step": kl_1}
        out["blocked_equals_onestep"] = bool(torch.equal(tr_blocked, traces))

    # end to end through the C ABI with host buffers (pinned), copies inside
    e2e = None
    if not args.no_e2e:
        vp_h = torch.from_numpy(w.vp).pin_memory()
        src_h = torch.from_numpy(w.src_xyz).pin_memory()
        rec_h = torch.from_numpy(w.rec_xyz).pin_memory()
        wav_h = torch.from_numpy(w.wavelets(dt).astype(np.float32)).pin_memory()
        tr_h = torch.empty((nt, nrec), dtype=torch.float32).pin_memory()
        ms_e, _, _, _ = timed("blocked", max(1, args.steps // 2), 1, traces_out=tr_h, vp=vp_h,
                              src=src_h, wav=wav_h, rec=rec_h)
        h2d = vp_h.numel() * 4 + src_h.numel() * 8 + rec_h.numel() * 8 + wav_h.numel() * 4
        d2h = tr_h.numel() * 4
        e2e = {"value": ws * N * nt / (ms_e * 1e-3) / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "ms_per_step": ms_e}

    # roofline of the dominant kernel (the blocked sweep), against the lowest of
    # its algorithmic ceilings: HBM (20/T B per point-step: u^n, u^{n-1}, c2
    # read and u^{n+T}, u^{n+T-1} written once per sweep) and the FP32 pipe
    # (the algorithmic flops of Eq. 1 per point-step).  The binding one is the
    # reported bound; the other and the issue rate (ncu's instructions per
    # point update) are given beside it as the explanation.
    T = args.time_tile
    peak, peak_kind = measured_peaks()
    launches_per_shot = kl_b
    full_sweeps = nt // T
    points_per_launch = N * full_sweeps / max(launches_per_shot, 1)
    bytes_per_launch = 20.0 * points_per_launch
    achieved = bytes_per_launch / (kms_b * 1e-3) / 1e9
    key = f"sweep_R{w.so // 2}_T{T}"
    counters = ncu_counters(key)
    upd_per_s = points_per_launch * T / (kms_b * 1e-3)
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    fpk, mhz = fp32_peak_tflops(nsm)
    fl = alg_flops(w.so)
    flops_per_launch = fl * points_per_launch * T
    ceil_hbm = peak / (20.0 / T)            # GPts/s
    ceil_fp32 = fpk * 1e12 / fl / 1e9       # GPts/s
    fp32_part = {"achieved": upd_per_s * fl / 1e12, "peak": fpk, "unit": "TFLOP/s",
                 "frac": upd_per_s * fl / 1e12 / fpk, "ceiling_gpts": ceil_fp32,
                 "peak_source": f"derived: {nsm} SMs x 128 FP32 lanes x 2 flops x {mhz:.0f} MHz",
                 "flops_per_point_step": fl, "flops_per_launch": flops_per_launch}
    hbm_part = {"achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "ceiling_gpts": ceil_hbm, "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
                "bytes_per_point_step": 20.0 / T, "bytes_per_launch": bytes_per_launch}
    traffic = (counters.get("dram_bytes_per_launch_full_size")
               if counters.get("grid_edge") == args.size else None)
    if ceil_hbm <= ceil_fp32:
        roof = {"bound": "hbm", **{k: hbm_part[k] for k in ("achieved", "peak", "unit", "frac")},
                "traffic": traffic, "peak_source": hbm_part["peak_source"], "fp32": fp32_part}
    else:
        roof = {"bound": "alu", **{k: fp32_part[k] for k in ("achieved", "peak", "unit", "frac")},
                "traffic": traffic, "peak_source": fp32_part["peak_source"], "hbm": hbm_part}
    roof.update({"kernel": f"sweep_kernel<R={w.so // 2},T={T}>", "bytes_per_launch": bytes_per_launch,
                 "kernel_ms_per_launch": kms_b, "point_updates_per_s_in_kernel": upd_per_s / 1e9,
                 "ceilings_gpts": {"hbm": ceil_hbm, "fp32": ceil_fp32}})
    # the peaks measured in this run with the library's own kernels (float4
    # copy, packed-FP32 FMA chains), beside the measured ones
    try:
        hbm_run, fp_run = tb.tb_measure_peaks()
        roof["in_run"] = {"hbm_gbs": hbm_run, "fp32_tflops": fp_run,
                          "frac_hbm": achieved / hbm_run, "frac_fp32": upd_per_s * fl / 1e12 / fp_run}
    except Exception as e:  # reported, not required
        roof["in_run"] = {"error": str(e)}
    ipp = counters.get("warp_inst_per_point_update")
    if ipp:
        ipeak = nsm * 4 * mhz * 1e6
        roof["issue"] = {"warp_inst_per_point_update": ipp, "achieved": ipp * upd_per_s / 1e9,
                         "peak": ipeak / 1e9, "unit": "G warp-inst/s", "frac": ipp * upd_per_s / ipeak,
                         "source": counters.get("inst_measured_on")}
    if "onestep" in out:
        o = out["onestep"]
        bpl1 = 16.0 * N * nt / max(o["launches_per_step"], 1)
        roof["onestep_kernel"] = {"achieved": bpl1 / (o["kernel_ms_per_launch"] * 1e-3) / 1e9,
                                  "frac": bpl1 / (o["kernel_ms_per_launch"] * 1e-3) / 1e9 / peak,
                                  "bytes_per_launch": bpl1,
                                  "kernel_ms_per_launch": o["kernel_ms_per_launch"]}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        try:
            rate, secs, threads = cpu_oracle_rate(w, dt, 2, 2 + args.cpu_steps)
            cpu = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
                   "sample": f"{w.shape[0]}^3 so{w.so}, {args.cpu_steps} steps (difference of a 2- "
                             f"and a {2 + args.cpu_steps}-step FP64 oracle run, {secs:.1f} s total)"}
        except Exception as e:  # the baseline is reported, not required
            cpu = {"value": None, "unit": UNIT, "cores": None, "kind": "oracle",
                   "sample": f"failed: {e}"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_b, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": bench_config(w, args, ws),
                "e2e": e2e, "gpu_launches": int(launches), "clocks": clk, "roofline": roof,
                "cpu_baseline": cpu, **out}
        if out.get("onestep"):
            line["speedup_vs_onestep"] = value / (ws * out["onestep"]["value"])
        print(json.dumps(line), flush=True)
    prop.close()
    if dist:
        dist.destroy_process_group()


def run_physics(args):
    """TTI or elastic propagation of the 384^3 so8 workload (500 steps),
    temporally blocked (the wavefront of --wave-tile steps over slabs of
    --slab planes) and one step per launch: one JSON line with GPts/s of the
    blocked shot, the one-step shot beside it, and the HBM roofline."""
    import torch
    import paper_2010_10248_gb300 as tb
    from paper_2010_10248_gb300 import build as tbbuild
    from paper_2010_10248_gb300 import workloads as wl
    torch.cuda.set_device(0)
    tbbuild.build()
    tb.load()
    size = args.size if args.size != 512 else 384
    nt = args.nt if args.nt != 1000 else 500
    if args.physics == "tti":
        w = wl.tti_384_so8(shape=(size,) * 3, nt=nt)
        phys = tb.TB_TTI
        # fused minimum per point and step: p, r at three levels (4 reads,
        # 2 writes), m, eps, delta, theta, phi
        alg_bytes = 44.0
    else:
        w = wl.elastic_384_so8(shape=(size,) * 3, nt=nt)
        phys = tb.TB_ELASTIC
        # fused minimum: 9 fields read and written, b, lam, mu
        alg_bytes = 84.0
    N = int(np.prod(w.shape))
    T = args.wave_tile
    dev = torch.device("cuda", 0)
    vp = torch.from_numpy(w.vp).to(dev)
    aux = torch.from_numpy(np.stack(w.meta["aux"])).to(dev)
    prop = tb.Propagator(w.shape, w.spacing, w.so, physics=phys, nbl=w.nbl, profile=True, time_tile=T,
                         slab_planes=args.slab, tti_fused=args.tti_fused, stream_l1=args.stream_l1)
    st = torch.cuda.current_stream()
    prop.set_model(vp, aux=aux)
    dt = prop.dt
    wav = torch.from_numpy(w.wavelets(dt).astype(np.float32)).to(dev)
    src = torch.from_numpy(w.src_xyz).to(dev)
    rec = torch.from_numpy(w.rec_xyz).to(dev)
    traces = {k: torch.empty((nt, len(w.rec_xyz)), dtype=torch.float32, device=dev)
              for k in (tb.TB_BLOCKED, tb.TB_ONESTEP)}

    def shot(sched):
        tb.tb_set_model(prop.h, vp, aux, None, 0.0, st)
        tb.tb_set_sources(prop.h, len(w.src_xyz), src, nt, wav, st)
        tb.tb_set_receivers(prop.h, len(w.rec_xyz), rec, st)
        tb.tb_forward(prop.h, nt, traces[sched], sched, st)

    def measure(sched):
        for _ in range(args.warmup):
            shot(sched)
        torch.cuda.synchronize()
        clocks = ClockSampler(0)
        clocks.start()
        l0 = tb.tb_launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        kms, kn = 0.0, 0
        e0.record(st)
        for _ in range(args.steps):
            shot(sched)
            n, ms = prop.kernel_time(0)
            kms += ms
            kn += n
        e1.record(st)
        torch.cuda.synchronize()
        clk = clocks.stop()
        ms = e0.elapsed_time(e1) / args.steps
        return ms, kms / args.steps, kn // args.steps, int(tb.tb_launch_count() - l0), clk

    ms_b, kms_b, kn_b, launches_b, clk = measure(tb.TB_BLOCKED)
    ms_1, kms_1, kn_1, launches_1, clk_1 = measure(tb.TB_ONESTEP)
    value = N * nt / (ms_b * 1e-3) / 1e9
    v1 = N * nt / (ms_1 * 1e-3) / 1e9
    peak, peak_kind = measured_peaks()
    # the step's kernels of the one-step shot and the wavefront launches of
    # the blocked shot (CUDA events around each launch on the stream)
    achieved_b = alg_bytes * N * nt / (kms_b * 1e-3) / 1e9
    achieved_1 = alg_bytes * N * nt / (kms_1 * 1e-3) / 1e9
    finite = bool(torch.isfinite(traces[tb.TB_BLOCKED]).all().item())
    same = bool(torch.equal(traces[tb.TB_BLOCKED], traces[tb.TB_ONESTEP]))
    cpu = None
    if not args.no_cpu:
        try:
            mk = wl.tti_384_so8 if args.physics == "tti" else wl.elastic_384_so8
            rate, secs, threads, sample = cpu_oracle_rate_physics(args.physics, mk, 256, 2, 22)
            cpu = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample}
        except Exception as e:  # the baseline is reported, not required
            cpu = {"value": None, "unit": UNIT, "cores": None, "kind": "oracle", "sample": f"failed: {e}"}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_b, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "grid": list(w.shape), "space_order": w.so, "nt": nt,
                       "receivers": len(w.rec_xyz), "schedule": "blocked", "time_tile": T,
                       "slab_planes": args.slab or 32,
                       "passes": "fused (TTI)" if args.tti_fused else ("L1 streaming" if args.stream_l1
                                                                       else "TMA-staged"),
                       "l2": "inputs larger than L2",
                       "step": "set_model + set_sources + set_receivers + forward(nt)"},
            "gpu_launches": launches_b, "clocks": clk,
            "onestep": {"value": v1, "ms_per_step": ms_1, "kernel_ms": kms_1, "launches": launches_1,
                        "achieved_gbs": achieved_1, "frac": achieved_1 / peak, "clocks": clk_1},
            "blocked_over_onestep": value / v1, "blocked_equals_onestep": same,
            "roofline": {"bound": "hbm", "achieved": achieved_b, "peak": peak, "unit": "GB/s",
                         "frac": achieved_b / peak, "traffic": None, "peak_source": peak_kind,
                         "kernel": f"{args.physics} wavefront launches of one shot (T = {T})",
                         "bytes_per_point_step": alg_bytes, "kernel_ms_per_shot": kms_b,
                         "wavefront_launches_per_shot": kn_b},
            "cpu_baseline": cpu, "traces_finite": finite}
    print(json.dumps(line), flush=True)
    prop.close()


def serving_shots(n, seed):
    """The serving workload: grids uniform over multiples of 32 in [128, 512]
    per axis, 300-1500 steps, 1-4 off-grid sources, 1k-64k receivers
    (log-uniform), seeded layered vp, so8, 10 m spacing, FP32 or FP16
    wavefield storage (50/50)."""
    from paper_2010_10248_gb300 import serving
    from paper_2010_10248_gb300 import workloads as wl
    g = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(n):
        shape = tuple(int(32 * g.integers(4, 17)) for _ in range(3))
        h = (10.0, 10.0, 10.0)
        ext = np.array([(shape[d] - 1) * h[d] for d in range(3)])
        nbl = 20
        # the layered model, built on the device when the shot is admitted
        vp = _DeviceLayers(shape, wl.layered_profile(shape[2], seed + 1000 + i))
        nsrc = int(g.integers(1, 5))
        src = np.stack([g.uniform(0.3, 0.7, nsrc) * ext[0], g.uniform(0.3, 0.7, nsrc) * ext[1],
                        np.full(nsrc, (nbl + 5 + g.uniform(0.1, 0.9)) * h[2])], axis=1)
        nrec = int(np.exp(g.uniform(np.log(1000), np.log(64000))))
        rec = np.stack([g.uniform(0.02, 0.98, nrec) * ext[0], g.uniform(0.02, 0.98, nrec) * ext[1],
                        np.full(nrec, (nbl + 8 + g.uniform(0.1, 0.9)) * h[2])], axis=1)
        storage = int(g.integers(0, 2))  # FP32 or FP16 wavefield storage, 50/50
        out.append(serving.ShotRequest(shape, h, 8, vp, src, 15.0, rec, nt=int(g.integers(300, 1501)), nbl=nbl,
                                       time_tile=0, tag=i, storage=storage))
    return out


class _DeviceLayers:
    """A layered velocity model (a depth profile repeated over x, y) made on
    the device when called: 500 shots of up to 512^3 would not fit in host
    memory made up front."""

    def __init__(self, shape, profile):
        self.shape, self.profile = tuple(shape), profile

    def __call__(self):
        import torch
        return torch.from_numpy(self.profile).cuda()[None, None, :].expand(self.shape).contiguous()


def run_serving(args):
    import torch
    import paper_2010_10248_gb300 as tb
    from paper_2010_10248_gb300 import build as tbbuild
    from paper_2010_10248_gb300 import serving
    torch.cuda.set_device(0)
    tbbuild.build()
    tb.load()
    reqs = serving_shots(args.shots, 2010_10248 + 4)
    work = np.array([np.prod(r.shape) * r.nt for r in reqs], dtype=np.float64)
    # capacity: the first ncal shots run one at a time, each alone on the GPU
    # (blocked sweep for FP32 storage, one-step for FP16), after one untimed
    # shot that takes the first-use costs (module loading, memory pool growth)
    ncal = min(20, len(reqs))
    cal = serving.ShotServer(slots=1)
    cal.run([serving.ShotRequest(**{**reqs[2].__dict__, "tag": "warm"})])
    t0 = time.perf_counter()
    cal.run([serving.ShotRequest(**{**reqs[i].__dict__, "tag": f"cal{i}", "arrival": 0.0}) for i in range(ncal)])
    cap = work[:ncal].sum() / (time.perf_counter() - t0)  # point updates / s, one at a time
    rate = 0.8 * cap / work.mean()                         # shots / s at 80 % of that capacity
    g = np.random.Generator(np.random.PCG64(2010_10248 + 5))
    arr = np.cumsum(g.exponential(1.0 / rate, size=len(reqs)))
    for r, a in zip(reqs, arr):
        r.arrival = float(a - arr[0])
    srv = serving.ShotServer(slots=args.slots, batch_points=256 ** 3, batch_max=16, batch_chunk=32)
    clocks = ClockSampler(0)
    clocks.start()
    t0 = time.perf_counter()
    res = srv.run(reqs)
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    lat = [r.latency for r in res]
    value = work.sum() / wall / 1e9
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": len(reqs), "warmup": 2,
            "ms_per_step": wall / len(reqs) * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"serving: Poisson stream of {len(reqs)} acoustic so8 shots, grids 128^3-512^3 "
                                   "(multiples of 32), 300-1500 steps, 1-4 sources, 1k-64k receivers",
                       "arrival_rate_per_s": rate, "slots": args.slots,
                       "schedule": ("FP32 shots of at most 256^3 points: batch lane (one launch per step for "
                                    "all shots in it, chunks of 32 steps); larger FP32 shots: blocked sweep "
                                    "alone on a slot; FP16 shots: one-step sweep on a slot"),
                       "precision": "FP32 arithmetic; FP32 or FP16 wavefield storage per shot (50/50)",
                       "fp16_shots": int(sum(1 for r in reqs if r.storage == 1)),
                       "batched_shots": int(sum(1 for r in reqs if r.storage == 0 and np.prod(r.shape) <= 256 ** 3)),
                       "calibration_shots": ncal},
            "latency_s": {"p50": serving.percentile(lat, 50), "p99": serving.percentile(lat, 99),
                          "mean": float(np.mean(lat)), "max": float(np.max(lat))},
            "capacity_alone_gpts": cap / 1e9, "value_over_capacity": value / (cap / 1e9),
            "lanes": srv.stats.get("lanes"), "max_in_flight": srv.stats["max_in_flight"],
            "max_bytes_in_flight": srv.stats["max_bytes"], "clocks": clk}
    print(json.dumps(line), flush=True)


def run_storage(args):
    """The acoustic benchmark shot with 16-bit wavefield storage (the one-step
    sweep) or scaled plain-FP32 storage (the streaming kernel), FP32
    arithmetic."""
    import torch
    import paper_2010_10248_gb300 as tb
    from paper_2010_10248_gb300 import build as tbbuild
    from paper_2010_10248_gb300 import workloads as wl
    torch.cuda.set_device(0)
    tbbuild.build()
    tb.load()
    stor = {"f16": tb.TB_F16, "bf16": tb.TB_BF16, "plain": tb.TB_F32_PLAIN}[args.storage]
    w = wl.acoustic_512_so8(shape=(args.size,) * 3, nt=args.nt)
    N, nt = int(np.prod(w.shape)), w.nt
    dev = torch.device("cuda", 0)
    prop = tb.Propagator(w.shape, w.spacing, w.so, nbl=w.nbl, storage=stor, profile=True)
    st = torch.cuda.current_stream()
    vp = torch.from_numpy(w.vp).to(dev)
    prop.set_model(vp)
    dt = prop.dt
    wav = torch.from_numpy(w.wavelets(dt).astype(np.float32)).to(dev)
    src = torch.from_numpy(w.src_xyz).to(dev)
    rec = torch.from_numpy(w.rec_xyz).to(dev)
    traces = torch.empty((nt, len(w.rec_xyz)), dtype=torch.float32, device=dev)

    def shot():
        tb.tb_set_model(prop.h, vp, None, None, 0.0, st)
        tb.tb_set_sources(prop.h, len(w.src_xyz), src, nt, wav, st)
        tb.tb_set_receivers(prop.h, len(w.rec_xyz), rec, st)
        tb.tb_forward(prop.h, nt, traces, tb.TB_ONESTEP, st)

    for _ in range(args.warmup):
        shot()
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    kms, kn = 0.0, 0
    l0 = tb.tb_launch_count()
    e0.record(st)
    for _ in range(args.steps):
        shot()
        n, ms = prop.kernel_time(0)
        kms += ms
        kn += n
    e1.record(st)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    step_ms = kms / max(kn, 1)
    bpp = 4.0 + (3 * 2.0 if stor != tb.TB_F32_PLAIN else 3 * 4.0)  # c2 + u^n, u^{n-1}, u^{n+1}
    peak, peak_kind = measured_peaks()
    achieved = bpp * N / (step_ms * 1e-3) / 1e9
    cpu = None
    if not args.no_cpu:
        try:
            rate, secs, threads = cpu_oracle_rate(w, dt, 2, 2 + args.cpu_steps)
            cpu = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
                   "sample": f"{w.shape[0]}^3 so{w.so}, {args.cpu_steps} steps (difference of a 2- "
                             f"and a {2 + args.cpu_steps}-step FP64 oracle run, {secs:.1f} s total)"}
        except Exception as e:  # the baseline is reported, not required
            cpu = {"value": None, "unit": UNIT, "cores": None, "kind": "oracle", "sample": f"failed: {e}"}
    line = {"metric": METRIC, "value": N * nt / (ms * 1e-3) / 1e9, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": {"f16": "f16-storage/f32-math",
                                                              "bf16": "bf16-storage/f32-math",
                                                              "plain": "f32"}[args.storage],
            "data": "synthetic",
            "config": {"workload": w.name, "grid": list(w.shape), "space_order": w.so, "nt": nt,
                       "schedule": "onestep (" + ("streaming kernel" if args.storage == "plain" else "TMA sweep") + ")",
                       "storage": args.storage,
                       "step": "set_model + set_sources + set_receivers + forward(nt)"},
            "gpu_launches": int(tb.tb_launch_count() - l0), "clocks": clk,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "peak_source": peak_kind,
                         "bytes_per_point_step": bpp, "kernel_ms_per_step": step_ms},
            "cpu_baseline": cpu}
    print(json.dumps(line), flush=True)
    prop.close()


def run_many_sources(args):
    """The 512^3 so8 benchmark grid with many sources (Sec. V-C): sources on a
    horizontal plane (sparse) and uniformly spread through the grid (dense),
    1 .. 32768 of them.  Per case: set_sources (inspector, decomposition,
    event table) timed on the host, then the blocked (T = 3) and the one-step
    schedule timed with CUDA events; the line's value is the blocked rate of
    the densest case."""
    import torch
    import paper_2010_10248_gb300 as tb
    from paper_2010_10248_gb300 import build as tbbuild
    from paper_2010_10248_gb300 import workloads as wl
    torch.cuda.set_device(0)
    tbbuild.build()
    tb.load()
    nt = args.nt if args.nt != 1000 else 300
    w = wl.acoustic_512_so8(shape=(args.size,) * 3, nt=nt)
    N = int(np.prod(w.shape))
    dev = torch.device("cuda", 0)
    T = args.time_tile
    prop = tb.Propagator(w.shape, w.spacing, w.so, nbl=w.nbl, time_tile=T, profile=True)
    st = torch.cuda.current_stream()
    prop.set_model(torch.from_numpy(w.vp).to(dev))
    dt = prop.dt
    prop.set_receivers(w.rec_xyz)
    traces = torch.empty((nt, len(w.rec_xyz)), dtype=torch.float32, device=dev)
    base_ws = None
    cases = []
    clocks = ClockSampler(0)
    clocks.start()
    l0 = tb.tb_launch_count()
    for layout in ("plane", "dense"):
        for n in (1, 64, 1024, 8192, 32768):
            if layout == "plane":
                src = wl.source_plane(w.shape, w.spacing, 101, n, depth_cells=w.nbl + 10, margin_cells=w.nbl)
            else:
                src = wl.source_cloud(w.shape, w.spacing, 102, n, margin_cells=w.nbl)
            wav = np.repeat(wl.ricker(w.f0, dt, nt)[None, :], n, axis=0).astype(np.float32)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            prop.set_sources(src, wav)
            torch.cuda.synchronize()
            set_s = time.perf_counter() - t0
            ws = tb.tb_workspace_bytes(prop.h)
            if base_ws is None:
                base_ws = ws
            rates = {}
            for sched in ("blocked", "onestep"):
                prop.forward(nt, traces, schedule=sched)
                ts = []
                for _ in range(max(1, args.steps // 2)):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(st)
                    prop.forward(nt, traces, schedule=sched)
                    e1.record(st)
                    torch.cuda.synchronize()
                    ts.append(e0.elapsed_time(e1))
                kn, kms = prop.kernel_time(0)
                rates[sched] = N * nt / (min(ts) * 1e-3) / 1e9
                rates[sched + "_kernel_ms_per_launch"] = kms / max(kn, 1)
            cases.append({"layout": layout, "sources": n, "grid_points": int(tb.tb_get_source_points(prop.h)),
                          "blocked": rates["blocked"], "onestep": rates["onestep"],
                          "speedup": rates["blocked"] / rates["onestep"], "set_sources_s": set_s,
                          "source_table_bytes": int(ws - base_ws)})
    clk = clocks.stop()
    worst = cases[-1]
    fl = alg_flops(w.so)
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    fpk, mhz = fp32_peak_tflops(nsm)
    hpk, hkind = measured_peaks()
    line = {"metric": METRIC, "value": worst["blocked"], "unit": UNIT, "n_gpus": 1,
            "steps": max(1, args.steps // 2), "warmup": 1, "ms_per_step": N * nt / (worst["blocked"] * 1e9) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"{w.name}, many sources (plane / dense, 1..32768)", "grid": list(w.shape),
                       "space_order": w.so, "nt": nt, "time_tile": T, "receivers": len(w.rec_xyz),
                       "value_case": "dense, 32768 sources, blocked",
                       "step": "forward(nt) (set_sources timed separately per case)"},
            "gpu_launches": int(tb.tb_launch_count() - l0), "clocks": clk,
            "roofline": {"bound": "hbm", "achieved": worst["blocked"] * 20.0 / T, "peak": hpk, "unit": "GB/s",
                         "frac": worst["blocked"] * 20.0 / T / hpk, "traffic": None,
                         "peak_source": f"{hkind} (MEASURED_PEAKS.json hbm_gbs)",
                         "note": ("end-to-end forward rate x 20/T algorithmic bytes per point-step (the "
                                  "source table rows add little); the HBM ceiling "
                                  f"{hpk / (20.0 / T):.0f} GPts/s is below the FP32 one "
                                  f"{fpk * 1e3 / fl:.0f} GPts/s"),
                         "fp32": {"achieved": worst["blocked"] * fl / 1e3, "peak": fpk, "unit": "TFLOP/s",
                                  "frac": worst["blocked"] * fl / 1e3 / fpk}},
            "cpu_baseline": None, "cases": cases}
    print(json.dumps(line), flush=True)
    prop.close()


def run_adjoint(args):
    """vp gradient of the acoustic shot at 256^3 so8 (the 512^3 recipe), 800
    steps, 32 checkpoints: one step = tb_adjoint_gradient (forward with
    checkpoints, then per segment the recomputation and the adjoint steps with
    the imaging condition) for the residual traces - traces of a model with a
    +3 % Gaussian anomaly.  GPts/s = grid points x steps / gradient time."""
    import torch
    import paper_2010_10248_gb300 as tb
    from paper_2010_10248_gb300 import build as tbbuild
    from paper_2010_10248_gb300 import workloads as wl
    torch.cuda.set_device(0)
    tbbuild.build()
    tb.load()
    size = args.size if args.size != 512 else 256
    nt = args.nt if args.nt != 1000 else 800
    nsnap = 32
    w = wl.acoustic_512_so8(shape=(size,) * 3, nt=nt)
    N = size ** 3
    dev = torch.device("cuda", 0)
    p = tb.Propagator(w.shape, w.spacing, w.so, nbl=w.nbl)
    vp = torch.from_numpy(w.vp).to(dev)
    p.set_model(vp)
    dt = p.dt
    ax = [torch.arange(n, device=dev, dtype=torch.float32) - n / 2 for n in w.shape]
    blob = torch.exp(-(ax[0][:, None, None] ** 2 + ax[1][None, :, None] ** 2 + ax[2][None, None, :] ** 2)
                     / (2 * (size / 10) ** 2))

    def geometry(model):
        p.set_model(model, dt=dt)
        p.set_sources(w.src_xyz, w.wavelets(dt))
        p.set_receivers(w.rec_xyz)

    geometry((vp * (1 + 0.03 * blob)).contiguous())
    d_obs = p.forward(nt, schedule="onestep").clone()
    geometry(vp)
    resid = (p.forward(nt, schedule="onestep") - d_obs).contiguous()
    st = torch.cuda.current_stream()
    # the forward alone, for the cost of a gradient in forward runs
    for _ in range(2):
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(st)
        p.forward(nt, schedule="onestep")
        f1.record(st)
        torch.cuda.synchronize()
    fwd_ms = f0.elapsed_time(f1)
    peak, peak_kind = measured_peaks()
    sched = {}
    grads = {}
    clocks = ClockSampler(0)
    clocks.start()
    l0 = tb.tb_launch_count()
    for mode in ("segments", "binomial"):
        gvp = torch.empty_like(vp)

        def step():
            p.adjoint_gradient(nt, resid, grad_vp=gvp, n_snapshots=nsnap, checkpointing=mode)

        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(args.steps):
            step()
        e1.record(st)
        torch.cuda.synchronize()
        ms_m = e0.elapsed_time(e1) / args.steps
        fsteps, scratch = p.adjoint_stats()
        # algorithmic bytes per point and step of the gradient: the forward
        # one-step sweeps (16 B each, fsteps of them for nt steps), the adjoint
        # sweep on mu = D lam (16) and the imaging condition (mu, u^k, u^{k-1},
        # u^{k-2}: 16, + FP64 sum 16)
        bpp_m = 16.0 * fsteps / nt + 16.0 + 32.0
        sched[mode] = {"value": N * nt / (ms_m * 1e-3) / 1e9, "ms_per_gradient": ms_m,
                       "gradient_in_forward_runs": ms_m / fwd_ms, "forward_steps": fsteps,
                       "forward_steps_per_nt": fsteps / nt, "scratch_bytes": scratch,
                       "scratch_fields": scratch / (4.0 * N), "bytes_per_point_step": bpp_m,
                       "hbm_frac": bpp_m * N * nt / (ms_m * 1e-3) / 1e9 / peak}
        grads[mode] = gvp
    clk = clocks.stop()
    launches = tb.tb_launch_count() - l0
    gvp = grads["binomial"]
    ms = sched["binomial"]["ms_per_gradient"]
    value = sched["binomial"]["value"]
    bpp = sched["binomial"]["bytes_per_point_step"]
    achieved = bpp * N * nt / (ms * 1e-3) / 1e9
    same = bool(torch.equal(grads["binomial"], grads["segments"]))
    finite = bool(torch.isfinite(gvp).all().item()) and float(gvp.abs().max()) > 0
    cpu = None
    if not args.no_cpu:
        try:
            import oracle
            oracle.build()
            ws = wl.acoustic_512_so8(shape=(192,) * 3, nt=44, nbl=10)
            dts = 0.8 * oracle.cfl_dt_max(ws.so, ws.spacing, float(ws.vp.max()))
            wav = ws.wavelets(dts)
            t = []
            for k in (4, 44):
                r = np.random.default_rng(1).standard_normal((k, len(ws.rec_xyz)))
                t0 = time.perf_counter()
                oracle.acoustic_adjoint(ws.shape, ws.spacing, ws.so, dts, k, ws.vp.astype(np.float64), r,
                                        nbl=ws.nbl, src_xyz=ws.src_xyz, src_wav=wav[:, :k], rec_xyz=ws.rec_xyz)
                t.append(time.perf_counter() - t0)
            threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
            cpu = {"value": 192 ** 3 * 40 / max(t[1] - t[0], 1e-9) / 1e9, "unit": UNIT, "cores": threads,
                   "kind": "oracle",
                   "sample": f"192^3 so8 gradient, 40 steps (difference of a 4- and a 44-step FP64 oracle "
                             f"adjoint run, {t[0] + t[1]:.1f} s total)"}
        except Exception as e:  # the baseline is reported, not required
            cpu = {"value": None, "unit": UNIT, "cores": None, "kind": "oracle", "sample": f"failed: {e}"}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"vp gradient, acoustic {size}^3 so8 {nt} steps", "grid": list(w.shape),
                       "space_order": w.so, "nt": nt, "snapshots": nsnap, "receivers": len(w.rec_xyz),
                       "checkpointing": "binomial (value); segments beside it",
                       "step": "tb_adjoint_gradient_ckpt (forward states from the checkpoints + adjoint)"},
            "gpu_launches": int(launches), "clocks": clk,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "peak_source": peak_kind,
                         "kernel": "gradient step (all kernels of one time step)", "bytes_per_point_step": bpp},
            "forward_ms": fwd_ms, "gradient_in_forward_runs": ms / fwd_ms, "schedules": sched,
            "binomial_equals_segments": same, "cpu_baseline": cpu, "gradient_finite": finite}
    print(json.dumps(line), flush=True)
    p.close()


def main():
    args = parse()
    if args.impl == "native" and args.storage != "f32":
        run_storage(args)
        return
    if args.impl == "native" and args.serving:
        run_serving(args)
        return
    if args.impl == "native" and args.physics != "acoustic":
        run_physics(args)
        return
    if args.impl == "native" and args.adjoint:
        run_adjoint(args)
        return
    if args.impl == "native" and args.many_sources:
        run_many_sources(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
