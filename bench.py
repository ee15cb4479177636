#!/usr/bin/env python
"""Benchmark of the RQA hot path on B300.

Primary line: recurrence cells/s (n^2 / step time) and the fraction of the
FP32 ALU issue roofline of the fused tile kernel, on a 1,048,576-point AR(1)
series (phi = 0.95, z-scored; m = 3, tau = 1, L2, eps = 0.5, Theiler 1,
minimum line lengths 2).  A step is one complete RQA computation through the
C ABI (embed -> fused tile kernel -> boundary merges -> line-of-identity join
-> histograms to the host -> measures) on a series already resident in HBM;
L2 is flushed (a 512 MiB write) before every timed step.

Also reported on the same line: end-to-end cells/s through the C ABI with
host buffers (copies inside the timed region), the FP64-everywhere GPU path
on the same series, cross recurrence of two 524,288-point series, line
detection over a 32,768 x 32,768 precomputed bit matrix, an 8,192 x 8,192
recurrence-plot window, the paper's own sine workload end to end (Sect. 8.2,
with the paper's runtimes as context), the batched workload (4,096 uneven
series, one graph per call) against sequential single-series calls, the
served workload (Poisson arrivals, p50 / p99 latency), the clocks seen during
the timed region, and the FP64 CPU oracle timed on a bounded sample on the
host's cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

WORKLOAD = "ar1_n1m"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
SM_MAX_FALLBACK = 2032.0
FP32_LANES_PER_SM = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-cross", action="store_true")
    ap.add_argument("--no-sine", action="store_true")
    ap.add_argument("--no-matrix", action="store_true")
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--no-saturation", action="store_true",
                    help="skip the served-rate sweep (the server vs one sequential worker)")
    ap.add_argument("--batch-count", type=int, default=4096)
    ap.add_argument("--N", type=int, default=0,
                    help="series length override (default: the 1,048,576-point workload)")
    ap.add_argument("--cpu-stride", type=int, default=0,
                    help="oracle sample: every k-th column and diagonal (0: pick ~15 s)")
    return ap.parse_args()


# ------------------------------------------------------------------ helpers
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(seconds: float, dist, device) -> float:
    """The job's time: the maximum of a per-rank time over all ranks (the
    rank itself when not distributed)."""
    if dist is None:
        return seconds
    import torch
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank_step: float, world: int, steps: int, seconds: float) -> float:
    """Units all ranks processed per second of the job's time (every rank
    runs the same workload: weak scaling, replicas)."""
    return world * units_per_rank_step * steps / seconds


def measured_peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f), "measured"
    except Exception:
        return {"sm_max_mhz": SM_MAX_FALLBACK}, "fallback"


class ClockSampler:
    """nvidia-smi sampling (200 ms) during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def tile_traffic(n):
    """DRAM bytes per tile-kernel launch from the committed ncu summary, or
    None if the kernel source changed since the counters were taken or the
    workload differs."""
    import hashlib
    prof = os.path.join(ROOT, "profiles", "tile_kernel_traffic.json")
    src = os.path.join(ROOT, "paper_2402_16853_b300", "csrc", "rqa_tile.cuh")
    try:
        rec = json.load(open(prof))
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except Exception:
        return None
    if rec.get("kernel_source_sha256_16") != sha or rec.get("scaled_to_n_vec") != n:
        return None
    return rec.get("tile_kernel_dram_bytes_per_launch")


def cpu_baseline(series, params, stride: int, target_s: float = 15.0):
    """The FP64 oracle as it stands, on the host's cores, over every
    stride-th column and diagonal of the same workload."""
    import oracle
    st = oracle.Settings(**params)
    n = len(series) - (params["m"] - 1) * params["tau"]
    cores = os.cpu_count() or 1
    if stride <= 0:
        # calibrate on a small sample, then size the run to ~target_s
        probe = max(1, int(2 * n * n // (cores * 5e7)))   # ~0.1-1 s of work
        t0 = time.perf_counter()
        *_, visited = oracle.histograms_streaming(series, st, threads=cores, stride=probe)
        dt = time.perf_counter() - t0
        rate = visited / max(dt, 1e-6)
        stride = max(1, int(2 * n * n / (rate * target_s)))
    t0 = time.perf_counter()
    *_, visited = oracle.histograms_streaming(series, st, threads=cores, stride=stride)
    dt = time.perf_counter() - t0
    cells_per_s = (visited / 2.0) / dt   # a cell costs one column and one diagonal visit
    return {"value": cells_per_s, "unit": "cells/s", "cores": cores, "kind": "oracle",
            "sample": f"every {stride}-th column and diagonal of the {n}-vector matrix "
                      f"({visited} cell visits in {dt:.1f} s; rate = visits/2/s)",
            "seconds": dt}


# ------------------------------------------------------------- reference arm
def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    s, params = synth.workload(WORKLOAD)
    n = len(s) - (params["m"] - 1) * params["tau"]
    stride = args.cpu_stride
    vals = []
    cb = None
    # W + K bounded samples, each ~5 s of CPU work
    for k in range(max(1, args.warmup) + max(1, args.steps)):
        cb = cpu_baseline(s, params, stride, target_s=5.0)
        stride = int(cb["sample"].split("every ")[1].split("-th")[0])
        if k >= max(1, args.warmup):
            vals.append(cb["value"])
    v = float(np.median(vals))
    step_s = n * n / v
    line = {"impl": "reference", "metric": "recurrence cells/s", "value": v,
            "extrapolated": True,
            "extrapolation": "value = cells/s of bounded samples (every k-th column and "
                             "diagonal); ms_per_step = n^2 / value, the whole matrix at "
                             "that rate, not a timed full run",
            "unit": "cells/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": step_s * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "N": len(s), **params},
            "cpu_baseline": {**cb, "value": v},
            "e2e": {"value": v, "unit": "cells/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ----------------------------------------------------------------- our arm
def run_mine(args):
    import torch
    import paper_2402_16853_b300 as gp

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    peaks, peak_kind = measured_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_max = float(peaks.get("sm_max_mhz", SM_MAX_FALLBACK))

    s, params = synth.workload(WORKLOAD)
    if args.N:
        s = synth.ar1(args.N, 1003, 0.95)
    N = len(s)
    n = N - (params["m"] - 1) * params["tau"]
    st = gp.Settings(**params)
    t_s = torch.tensor(s, dtype=torch.float64, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    r = gp.RQA(st)

    def barrier():
        torch.cuda.synchronize(dev)
        if dist is not None:
            dist.barrier()

    for _ in range(args.warmup):
        flush.fill_(1)
        r.run(t_s)
    stats0 = r.stats()
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    kernel_ms = []
    launches = 0
    ev0.record(stream)
    for _ in range(args.steps):
        flush.fill_(1)
        r.run(t_s)
        stt = r.stats()
        kernel_ms.append(stt["kernel_ms"])
        launches += stt["launches"] + 1   # + the L2 flush fill
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    elapsed = max_over_ranks(ev0.elapsed_time(ev1) / 1e3, dist, dev)
    barrier()
    meas = r.measures()
    stt = r.stats()
    cells = float(n) * n
    value = whole_job_rate(cells, world, args.steps, elapsed)
    pairs = stt["pairs"]
    ops_per_pair = 2 * params["m"] + 1
    k_ms = float(np.mean(kernel_ms))
    achieved = pairs * ops_per_pair / (k_ms / 1e3) / 1e12
    peak_theory = sms * FP32_LANES_PER_SM * sm_max * 1e6 / 1e12
    # measured FP32 issue throughput of the distance loop's operations; the
    # roofline divides by the larger of theory and measurement
    try:
        probes = {k: v / 1e12 for k, v in gp.probe_alu().items()}
    except gp.RQAError:
        probes = {}
    peak = max([peak_theory] + list(probes.values()))
    traffic = tile_traffic(n)

    # ---- end to end through the C ABI with host buffers
    host = torch.tensor(s, dtype=torch.float64).pin_memory().numpy()
    r.run(host)
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    e2e_steps = max(1, min(args.steps, 3))
    for _ in range(e2e_steps):
        flush.fill_(1)
        r.run(host)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    e2e_s = e0.elapsed_time(e1) / 1e3
    st_e2e = r.stats()
    e2e = {"value": world * cells * e2e_steps / e2e_s, "unit": "cells/s",
           "h2d_bytes_per_step": int(st_e2e["h2d_bytes"]),
           "d2h_bytes_per_step": int(st_e2e["d2h_bytes"])}

    extra = {}
    # ---- FP64-everywhere GPU path on the same series
    if not args.no_fp64:
        r64 = gp.RQA(gp.Settings(**params, precision=gp.PREC_FP64))
        r64.run(t_s)
        barrier()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        r64.run(t_s)
        a1.record(stream)
        torch.cuda.synchronize(dev)
        t64 = a0.elapsed_time(a1) / 1e3
        m64 = r64.measures()
        same = all((meas[k] == m64[k]) or (isinstance(meas[k], float) and math.isnan(meas[k])
                                            and math.isnan(m64[k])) for k in meas)
        extra["fp64_path"] = {"value": cells / t64, "unit": "cells/s",
                              "kernel_ms": r64.stats()["kernel_ms"],
                              "speedup_fp32_recheck": (cells / (elapsed / args.steps)) /
                                                      (cells / t64),
                              "measures_identical": bool(same)}
        del r64

    # ---- the two smaller single-series workloads (context lines)
    extra["logistic_n2000"] = bench_single(gp, "logistic_n2000", dev, barrier, flush, peak, 50)
    extra["lorenz_n100k"] = bench_single(gp, "lorenz_n100k", dev, barrier, flush, peak, 10)

    # ---- cross recurrence of two AR(1) series (context line)
    if not args.no_cross:
        extra["cross"] = bench_cross(gp, params, dev, barrier, flush, peak)

    # ---- line detection over a precomputed bit matrix, and the plot (context)
    if not args.no_matrix:
        extra["matrix_input"] = bench_matrix(gp, dev, barrier, flush)
        extra["plot"] = bench_plot(gp, s, params)

    # ---- the paper's own timing workload (context line)
    if not args.no_sine:
        extra["paper_sine"] = bench_sine(gp, dev, barrier)

    # ---- batched workload vs sequential single-series calls
    if not args.no_batch:
        extra["batched"] = bench_batch(gp, args, dev, barrier)

    # ---- served workload
    if not args.no_serve:
        extra["served"] = bench_serve(gp, args)

    line = {
        "metric": "recurrence cells/s", "value": value, "unit": "cells/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": elapsed / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": N, "n_vec": n, **params,
                   "series": "AR(1) phi=0.95, N(0,1) noise, z-scored, seed 1003",
                   "l2": "flushed before every timed step (512 MiB write)",
                   "parallelism": f"replicas{world}" if world > 1 else "single GPU"},
        "pairs_per_s": world * pairs * args.steps / elapsed,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TOP/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "tile_kernel<3,L2,4,fp32>", "kernel_ms": k_ms,
                     "ops_per_pair": ops_per_pair, "pairs_per_launch": pairs,
                     "peak_basis": f"max of {sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x "
                                   f"{sm_max:.0f} MHz ({peak_kind} sm_max_mhz) = "
                                   f"{peak_theory:.2f} TOP/s and the measured probes",
                     "peak_probes_tops": probes,
                     "frac_of_theory_at_run_clock": (
                         achieved / (peak_theory * clk["sm_mhz"] / sm_max)
                         if clk.get("sm_mhz") else None)},
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk,
        "rechecks_per_step": int(stt["rechecks"]), "recheck_band_rel": stt["band"],
        "exact": bool(stt["exact"]),
        "measures": {k: meas[k] for k in ("rr", "det", "l", "l_max", "lam", "tt", "v_max")},
        **extra,
    }
    if rank == 0 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(s, params, args.cpu_stride)
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


def bench_single(gp, name, dev, barrier, flush, peak, steps):
    """One of the smaller single-series workloads on a device-resident series:
    cells/s per step (L2 flushed before each), and the tile kernel's share of
    the ALU roofline as for the primary line."""
    import torch
    s, p = synth.workload(name)
    t = torch.tensor(s, dtype=torch.float64, device=dev)
    r = gp.RQA(gp.Settings(**p))
    for _ in range(3):
        r.run(t)
    barrier()
    stream = torch.cuda.current_stream(dev)
    # each step timed alone, the L2 flush before its start event: at these
    # sizes the 512 MiB fill would otherwise be a quarter of a step
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    kms = []
    for e0, e1 in evs:
        flush.fill_(1)
        e0.record(stream)
        r.run(t)
        e1.record(stream)
        kms.append(r.stats()["kernel_ms"])
    torch.cuda.synchronize(dev)
    sec = sum(e0.elapsed_time(e1) for e0, e1 in evs) / 1e3 / steps
    st = r.stats()
    n = st["n_vec"]
    k_ms = float(np.median(kms))
    ops = st["pairs"] * (2 * p["m"] + 1)
    return {"workload": f"{name}: N = {len(s)}, m = {p['m']}, tau = {p['tau']}, "
                        f"norm {p['norm']}, eps = {p['eps']}, w = {p['theiler']}",
            "value": float(n) * n / sec, "unit": "cells/s", "ms_per_step": sec * 1e3,
            "steps": steps, "kernel_ms": k_ms, "roofline_frac": ops / (k_ms / 1e3) / 1e12 / peak,
            "band_rows": int(st["band_rows"]), "strip_width": int(st["strip_width"]),
            "l2": "flushed before every timed step (512 MiB write, outside the step's events)"}


def bench_cross(gp, params, dev, barrier, flush, peak, N=524_288, steps=2):
    """Cross recurrence (Sect. 3.3) of two independent AR(1) series of N
    points each with the primary line's parameters: n1 x n2 cells per step."""
    import torch
    x = torch.tensor(synth.ar1(N, 1003, 0.95), dtype=torch.float64, device=dev)
    y = torch.tensor(synth.ar1(N, 1007, 0.95), dtype=torch.float64, device=dev)
    r = gp.RQA(gp.Settings(**params))
    flush.fill_(1)
    r.run_cross(x, y)
    barrier()
    stream = torch.cuda.current_stream(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    kms = []
    e0.record(stream)
    for _ in range(steps):
        flush.fill_(1)
        r.run_cross(x, y)
        kms.append(r.stats()["kernel_ms"])
    e1.record(stream)
    torch.cuda.synchronize(dev)
    t = e0.elapsed_time(e1) / 1e3 / steps
    st = r.stats()
    cells = float(st["n_vec"]) * st["n_cols"]
    k_ms = float(np.mean(kms))
    ops = st["pairs"] * (2 * params["m"] + 1)
    achieved = ops / (k_ms / 1e3) / 1e12
    return {"workload": f"AR(1) x AR(1), N = {N} each (seeds 1003, 1007), same parameters",
            "value": cells / t, "unit": "cells/s", "ms_per_step": t * 1e3, "steps": steps,
            "kernel_ms": k_ms, "roofline_frac": achieved / peak,
            "kernel": f"tile_kernel<{params['m']},L2,4,fp32,cross>",
            "rechecks": int(st["rechecks"]), "rr": r.measures()["rr"]}


def bench_matrix(gp, dev, barrier, flush, rows=32768, cols=32768, steps=3):
    """rqa_run_matrix_device on a random bit matrix (each bit the AND of
    three random bits: density 1/8, seed 5) with a black band of columns
    5,024 .. 5,311 across strips: rows x cols cells per step."""
    import torch
    rng = np.random.default_rng(5)
    wpr = (cols + 31) // 32
    words = rng.integers(0, 1 << 32, size=(rows, wpr), dtype=np.uint32)
    for _ in range(2):
        words &= rng.integers(0, 1 << 32, size=(rows, wpr), dtype=np.uint32)
    words[:, 157:166] = 0xFFFFFFFF
    t = torch.from_numpy(words.view(np.int32)).to(dev)
    r = gp.RQA(gp.Settings(m=1, tau=1, eps=1.0, norm=0, theiler=0))
    r.run_matrix(t, cols=cols)
    barrier()
    stream = torch.cuda.current_stream(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    kms = []
    e0.record(stream)
    for _ in range(steps):
        flush.fill_(1)
        r.run_matrix(t, cols=cols)
        kms.append(r.stats()["kernel_ms"])
    e1.record(stream)
    torch.cuda.synchronize(dev)
    sec = e0.elapsed_time(e1) / 1e3 / steps
    return {"workload": f"{rows} x {cols} random bit matrix (density 1/8) on the device",
            "value": float(rows) * cols / sec, "unit": "cells/s", "ms_per_step": sec * 1e3,
            "kernel_ms": float(np.mean(kms)), "matrix_bytes": int(words.nbytes),
            "rr": r.measures()["rr"]}


def bench_plot(gp, s, params, rows=8192, cols=8192):
    """rqa_recurrence_plot: an 8,192 x 8,192 window of the primary series'
    matrix, bit-packed, to host memory (one call, wall clock)."""
    st = gp.Settings(**params)
    gp.recurrence_plot(st, s, i0=0, j0=0, rows=64, cols=64)
    t0 = time.perf_counter()
    gp.recurrence_plot(st, s, i0=500_000, j0=500_000, rows=rows, cols=cols, packed=True)
    sec = time.perf_counter() - t0
    return {"workload": f"{rows} x {cols} window of the primary series' matrix",
            "value": float(rows) * cols / sec, "unit": "cells/s", "seconds": sec}


def bench_sine(gp, dev, barrier, steps=2):
    """The paper's runtime experiment (Sect. 8.2): sin over 1,000,001 points,
    m = 2, tau = 2, radius 1, no Theiler window, timed end to end from a host
    series (copies, all kernels, histograms back, measures), as the paper
    times total runtime.  The paper's figures are context on other hardware."""
    s, p = synth.workload("sine_paper")
    r = gp.RQA(gp.Settings(**p))
    r.run(s)
    barrier()
    t0 = time.perf_counter()
    for _ in range(steps):
        meas = r.run(s)
    t = (time.perf_counter() - t0) / steps
    n = meas["n_vec"]
    return {"workload": "sin(linspace(0, 1000 pi, 1000001)), m=2, tau=2, eps=1, L2, w=0",
            "seconds_per_run": t, "value": float(n) * n / t, "unit": "cells/s",
            "l_max": meas["l_max"], "det": meas["det"],
            "paper_seconds_context": {"4x GK104 (2x GTX 690)": 68.94, "1x GK104": 204.81,
                                      "i7-3820 OpenCL": 1667.58,
                                      "CRP 1.13z, 1 thread": 28480.09}}


def bench_batch(gp, args, dev, barrier):
    import torch
    specs = synth.batch_specs(args.batch_count)
    series, eps = synth.make_series(specs, seed=2004)
    settings = [gp.Settings(m=sp.m, tau=sp.tau, eps=e, norm=sp.norm, theiler=sp.theiler,
                            l_min=sp.l_min, v_min=sp.v_min, w_min=sp.w_min)
                for sp, e in zip(specs, eps)]
    tuned = gp.tuning_table_loaded()
    b = gp.Batch()
    res, status, rc = b.run(settings, series)   # captures the graph
    assert rc == 0, status
    b.run(settings, series)
    calls = 5   # the median call: the host half of a call varies with the box's load
    barrier()
    tb = []
    for _ in range(calls):
        t0 = time.perf_counter()
        res2, st2, rc2 = b.run(settings, series)
        tb.append(time.perf_counter() - t0)
    t_batch = float(np.median(tb))
    bst = b.stats()
    untuned = None
    if tuned:  # the same batch with the size rule only (tuning table cleared)
        gp.autotune_clear()
        b.run(settings, series)
        tu = []
        for _ in range(calls):
            t0 = time.perf_counter()
            b.run(settings, series)
            tu.append(time.perf_counter() - t0)
        untuned = len(series) / float(np.median(tu))
        gp.load_tuning_table(gp.rqa.TUNING_TABLE)
    # sequential single-series calls of the same kernels on one prebuilt
    # handle (rqa_set_settings between series), its buffers already grown to
    # the largest series, so only the per-series launch work is timed
    rr = gp.RQA(settings[0])
    big = max(range(len(series)), key=lambda q: len(series[q]))
    rr.set_settings(settings[big])
    rr.run(series[big])
    t0 = time.perf_counter()
    seq = []
    for stg, s in zip(settings, series):
        rr.set_settings(stg)
        seq.append(rr.run(s))
    t_seq = time.perf_counter() - t0
    rr.close()
    same = all(a == bb or (isinstance(a, float) and math.isnan(a) and math.isnan(bb))
               for m1, m2 in zip(res2, seq) for a, bb in zip(m1.values(), m2.values()))
    cells = float(sum((len(s) - (sp.m - 1) * sp.tau) ** 2 for s, sp in zip(series, specs)))
    return {"series": len(series), "series_per_s": len(series) / t_batch,
            "cells_per_s": cells / t_batch, "ms_per_batch": t_batch * 1e3,
            "kernel_ms": bst["kernel_ms"], "device_ms": bst["total_ms"],
            "sequential_series_per_s": len(series) / t_seq,
            "speedup_vs_sequential": t_seq / t_batch, "identical_to_sequential": bool(same),
            "sequential_baseline": "rqa_run per series on one prebuilt handle "
                                   "(rqa_set_settings between series)",
            "tuned": tuned, "untuned_series_per_s": untuned,
            "speedup_tuned_vs_untuned": (len(series) / t_batch) / untuned if untuned else None,
            "graph": "captured once, replayed",
            "timing": f"median of {calls} calls (ms per call: "
                      + ", ".join(f"{1e3 * t:.1f}" for t in tb) + ")",
            "cpu_oracle": batch_oracle_sample(specs, series, eps) if not args.no_cpu else None}


def batch_oracle_sample(specs, series, eps, every=64):
    """The FP64 oracle on every 64th series of the batch, one series after
    another on all host cores (streaming mode): series/s and cells/s."""
    import oracle
    cores = os.cpu_count() or 1
    idx = list(range(0, len(series), every))
    cells = 0.0
    t0 = time.perf_counter()
    for q in idx:
        sp = specs[q]
        st = oracle.Settings(m=sp.m, tau=sp.tau, eps=eps[q], norm=sp.norm, theiler=sp.theiler,
                             l_min=sp.l_min, v_min=sp.v_min, w_min=sp.w_min)
        oracle.rqa(series[q], st, mode="streaming", threads=cores)
        n = len(series[q]) - (sp.m - 1) * sp.tau
        cells += float(n) * n
    dt = time.perf_counter() - t0
    return {"series_per_s": len(idx) / dt, "cells_per_s": cells / dt, "cores": cores,
            "kind": "oracle", "sample": f"every {every}-th series of the batch "
                                         f"({len(idx)} series, {dt:.1f} s)"}


def serve_stream_run(gp, arrivals, settings, series, cells_per_req, seconds,
                     workers=None, epoch_cells=None, drain_s=120.0):
    """Replay a Poisson request stream against a fresh server (optionally with
    RQA_SERVE_WORKERS / RQA_SERVE_EPOCH_CELLS overrides) and measure each
    request from submission to completion.  Requests still pending drain_s
    after the last arrival count as not served."""
    env = {}
    if workers is not None:
        env["RQA_SERVE_WORKERS"] = str(workers)
    if epoch_cells is not None:
        env["RQA_SERVE_EPOCH_CELLS"] = repr(float(epoch_cells))
    old = {k: os.environ.get(k) for k in env}
    os.environ.update(env)
    try:
        srv = gp.Server(40 << 30, max_slots=4096)
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    t = srv.submit(settings[0], series[0])   # warm the engines
    srv.wait(t)
    srv.release(t)
    k_all = len(series)
    done_at = [None] * k_all
    tickets = [None] * k_all
    submit_at = [None] * k_all
    stop = threading.Event()
    t0 = time.perf_counter()

    def poller():
        pending = set()
        q = 0
        while q < k_all or pending:
            while q < k_all and tickets[q] is not None:
                pending.add(q)
                q += 1
            fin = []
            for k in pending:
                rc, _ = srv.poll(tickets[k])
                if rc != gp.rqa.RQA_PENDING:
                    done_at[k] = time.perf_counter()
                    fin.append(k)
            for k in fin:
                pending.discard(k)
                srv.release(tickets[k])
            if stop.is_set() and q >= k_all:
                break
            if not fin:
                time.sleep(0.0005)

    th = threading.Thread(target=poller)
    th.start()
    for k, (a, stg, s) in enumerate(zip(arrivals, settings, series)):
        now = time.perf_counter() - t0
        if a > now:
            time.sleep(a - now)
        submit_at[k] = time.perf_counter()
        tickets[k] = srv.submit(stg, s)
    deadline = time.perf_counter() + drain_s
    while th.is_alive() and time.perf_counter() < deadline:
        th.join(timeout=0.5)
    stop.set()
    th.join()
    srv.close()   # waits for epochs in flight, drops what is still queued
    done = [q for q in range(k_all) if done_at[q] is not None]
    lat = np.array([done_at[q] - submit_at[q] for q in done])
    t_end = max(done_at[q] for q in done)
    wall = t_end - t0
    return {"requests": k_all, "completed": len(done),
            "offered_rate_per_s": k_all / seconds,
            "series_per_s": len(done) / wall,
            "cells_per_s": float(sum(cells_per_req[q] for q in done)) / wall,
            "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "max_ms": float(lat.max() * 1e3)}


def bench_serve(gp, args):
    """cfg5: Poisson arrivals at 200 req/s for --serve-seconds (60 s by
    default, about 12,000 requests), lengths log-uniform in [1,000, 200,000],
    memory admission under a 40 GB budget.  Then a rate sweep (8 s per rate)
    against the same server and against one worker that runs one request per
    launch epoch (sequential plain launches): the highest offered rate each
    sustains with p99 under 100 ms and every request served."""
    def stream(rate, seconds, seed):
        arrivals, specs, series, eps = synth.serve_stream(rate=rate, duration=seconds, seed=seed)
        settings = [gp.Settings(m=sp.m, tau=sp.tau, eps=e, norm=sp.norm, theiler=sp.theiler,
                                l_min=sp.l_min, v_min=sp.v_min, w_min=sp.w_min)
                    for sp, e in zip(specs, eps)]
        cells = [float(len(s) - (sp.m - 1) * sp.tau) ** 2 for s, sp in zip(series, specs)]
        return arrivals, settings, series, cells

    arrivals, settings, series, cells = stream(200.0, args.serve_seconds, 1005)
    out = serve_stream_run(gp, arrivals, settings, series, cells, args.serve_seconds)
    out.update({"budget_bytes": 40 << 30, "seconds_of_arrivals": args.serve_seconds,
                "workers": 4})
    if not args.no_saturation:
        sweep = []
        for rate in (200.0, 300.0, 400.0, 500.0, 600.0):
            arr, stg, ser, cl = stream(rate, 8.0, 3005)
            row = {"offered_rate_per_s": rate}
            for name, w, ec in (("continuous_4_workers", None, None),
                                ("sequential_1_worker", 1, 1.0)):
                r = serve_stream_run(gp, arr, stg, ser, cl, 8.0, workers=w, epoch_cells=ec,
                                     drain_s=30.0)
                row[name] = {k: r[k] for k in ("completed", "requests", "series_per_s",
                                               "p50_ms", "p99_ms")}
            sweep.append(row)

        def sustained(name):
            ok = [row["offered_rate_per_s"] for row in sweep
                  if row[name]["completed"] == row[name]["requests"]
                  and row[name]["p99_ms"] < 100.0]
            return max(ok) if ok else None
        out["rate_sweep_8s"] = sweep
        out["sustained_rate_p99_under_100ms"] = {"continuous_4_workers":
                                                 sustained("continuous_4_workers"),
                                                 "sequential_1_worker":
                                                 sustained("sequential_1_worker")}
    return out


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_mine(args)


if __name__ == "__main__":
    main()
