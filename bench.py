#!/usr/bin/env python
"""Benchmark of the Lomb-Scargle NUFFT hot path on one or more GB300s.

Workload (default): the large single series -- N_d = 1,000,000 times over a
10-year baseline with seasonal gaps, N_f = 12,000,000 frequencies
(f0 = 1/3650, df = 1/18250), FP32 spread/FFT at eps = 1e-6 (relative l2
error <= 1e-5 against the FP64 oracle).  A step is one periodogram: every
kernel of the path (preprocess, bin sort, pass A, pass B) over one series.

Prints one JSON line (rank 0).  ``value`` = periodograms/s with the inputs
resident in HBM (device time of K steps, CUDA events, L2 flushed between
steps outside the timed events); ``e2e`` = the same metric through the
C-ABI with pinned host buffers (copies in and out inside the timed region);
``roofline`` = the dominant kernel's algorithmic bytes over its live
event-timed duration against the measured HBM copy bandwidth;
``cpu_baseline`` = the FP64 oracle timed on this host's cores on a bounded
sample of the same workload.

``--impl reference`` times the oracle as the reference arm (host cores only).
Multi-GPU (torchrun): every rank computes its own periodograms (independent
series, no collective on the data path); value = all ranks' periodograms
divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import functools
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("periodograms/s and p50/p99 latency at rel err <=1e-5; "
          "spread+FFT HBM GB/s vs peak")
UNIT = "periodograms/s"
FALLBACK_HBM_GBS = 6800.0


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--workload", default="single_large",
                    choices=["single_large", "single_medium", "single_small", "uniform_batch",
                             "ragged_batch", "serving"])
    ap.add_argument("--batch-scale", type=float, default=1.0,
                    help="fraction of the batch workloads' series (4096 uniform, 10,000 ragged)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64-path", action="store_true")
    ap.add_argument("--no-fft-reference", action="store_true")
    ap.add_argument("--upsampling", type=float, default=0.0,
                    help="fine-grid upsampling: 0 (plan chooses), 2.0 or 1.5")
    ap.add_argument("--batch-mode", default="graph", choices=["graph", "prepared", "direct"],
                    help="batch workloads: replay a recorded graph of a prepared batch, run the "
                         "prepared batch, or call ls_execute_batch(_shared) each step")
    ap.add_argument("--serving-copy-limit", type=int, default=None,
                    help="serving with host results: batches with at most this many output "
                         "bytes are copied out per request, larger ones handed out as views")
    ap.add_argument("--serving-results", default="host", choices=["host", "device"],
                    help="serving: deliver results as host arrays or device tensor views")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target CPU time of the oracle baseline sample")
    ap.add_argument("--no-extras", action="store_true",
                    help="single_large: skip the uniform-batch, ragged-batch and serving "
                         "sub-blocks of the default line")
    return ap.parse_args()


def workload(name: str, rank: int):
    from paper_2409_08090_gb300 import workloads as W
    if name == "single_medium":
        s = W.single_large(seed=W.BASE_SEED + 1 + 1000 * rank, nd=250_000, nf=3_000_000)
        desc = ("single_medium (profiling size): Nd=2.5e5 over [0,3650) d with seasonal gaps; "
                "Nf=3e6, f0=1/3650, df=1/18250")
        return s, desc
    if name == "single_small":
        s = W.single_small(seed=W.BASE_SEED + 1000 * rank)
        desc = "single_small: Nd=1e3 over [0,100) d, Nf=1.2e4, f0=0.01, df=0.002"
    else:
        s = W.single_large(seed=W.BASE_SEED + 1 + 1000 * rank)
        desc = ("single_large: Nd=1e6 over [0,3650) d with 120-d seasonal gaps, 3 sinusoids, "
                "lognormal dy; Nf=1.2e7, f0=1/3650, df=1/18250")
    return s, desc


def eps_for(precision: str) -> float:
    return 1e-6 if precision == "fp32" else 1e-9


# --------------------------------------------------------------------- helpers

class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms in the background."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        finally:
            os.unlink(self.path)
        if not rows:
            return None

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4)
                          if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def measured_hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def source_digest() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2409_08090_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        h.update(f.encode())
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str, precision: str, workload: str):
    """DRAM bytes per launch from a committed ncu summary of this kernel on this
    workload, if it was taken on the current kernel sources (same digest);
    else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        d = json.load(open(path))
    except (OSError, ValueError):
        return None
    ent = d.get(f"{kernel}:{precision}:{workload}")
    if not ent or ent.get("source_digest") != source_digest():
        return None
    return ent.get("dram_bytes_per_launch")


def fp32_issue_roof(sms: int, mhz: float | None = None) -> dict:
    """Roof of the FP64 path's double-float FFTs: they run on the FP32 units,
    one FP32 operation per lane per clock (128 lanes per SM).  In the code's
    double-float arithmetic an addition takes 11 FP32 operations (Knuth's
    two-sum of the high parts, the low parts added, a renormalising fast
    two-sum) and a multiplication 7 (the fma two-product plus the cross terms
    and a renormalisation); a radix-2 butterfly's 10 flops are 6 additions and
    4 multiplications, 94 FP32 operations, so one FP64-equivalent flop costs 9.4
    FP32 operations."""
    if mhz is None:
        try:
            mhz = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["sm_max_mhz"])
        except (OSError, KeyError, ValueError):
            mhz = 2070.0
    ops = sms * 128 * mhz * 1e6
    return {"tflops": ops / 9.4 / 1e12,
            "derivation": f"{sms} SMs x 128 FP32 lanes x {mhz:.0f} MHz = {ops / 1e12:.1f} T FP32 "
                          "ops/s; 9.4 FP32 ops per double-float flop (add 11, mul 7; a "
                          "radix-2 butterfly's 6 adds + 4 muls)"}


def algorithmic_bytes(info, nd: int, nf: int, precision: str) -> dict:
    """Bytes each kernel must move (per launch, per periodogram)."""
    rs = 4 if precision == "fp32" else 8
    cx = 2 * rs
    n = info.n
    pts = 3 * nd * (4 + rs + cx)          # cell, offset, strength per transform
    return {
        "pass_a_spread_fft": 3 * n * cx + pts,          # H written once
        # H read once, P written, the deconvolution factor of each needed mode
        # (pass-B order table: one entry per output frequency)
        "pass_b_fft_deconv_power": 3 * n * cx + 8 * nf + rs * nf,
        "preprocess": 24 * nd + 3 * nd * (4 + rs + cx) + nd * (4 + rs + cx),
        "bin_sort": 2 * (3 * nd * (4 + rs + cx)) // 1,
    }


def dist_setup():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = False
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
        pg = True
    return world, rank, local, pg


def barrier(pg):
    if pg:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(x: float, pg, device) -> float:
    if not pg:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------- CPU oracle

def oracle_sample(s, seconds: float, seed: int = 4242):
    """Time the FP64 oracle on seeded random frequencies of the workload; the
    count is scaled from a short pilot so the sample takes about `seconds`.
    Returns (k, P_oracle, elapsed_s, threads)."""
    import numpy as np
    import oracle
    oracle.build()
    rng = np.random.default_rng(seed)
    pilot = 64
    k = rng.choice(s.nf, pilot, replace=False).astype(np.int64)
    oracle.periodogram(s.t, s.y, s.dy, s.f0, s.df, k[:16])      # thread start-up
    t0 = time.perf_counter()
    oracle.periodogram(s.t, s.y, s.dy, s.f0, s.df, k)
    dt = time.perf_counter() - t0
    nk = int(max(pilot, min(s.nf, pilot * seconds / max(dt, 1e-6))))
    k = np.sort(rng.choice(s.nf, nk, replace=False)).astype(np.int64)
    t0 = time.perf_counter()
    P = oracle.periodogram(s.t, s.y, s.dy, s.f0, s.df, k)
    dt = time.perf_counter() - t0
    return k, P, dt, oracle.threads()


# ------------------------------------------------------------------ reference arm

def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import numpy as np
    import oracle
    oracle.build()
    s, desc = workload(args.workload, 0)
    rng = np.random.default_rng(99)
    # one step = the oracle on a bounded frequency sample of the same series
    pilot = rng.choice(s.nf, 8, replace=False).astype(np.int64)
    t0 = time.perf_counter()
    oracle.periodogram(s.t, s.y, s.dy, s.f0, s.df, pilot)
    per_freq = (time.perf_counter() - t0) / 8
    budget_s = 150.0 / max(1, args.steps + args.warmup)
    nk = int(max(8, min(s.nf, budget_s / max(per_freq, 1e-9))))
    times = []
    for i in range(args.warmup + args.steps):
        k = rng.choice(s.nf, nk, replace=False).astype(np.int64)
        t0 = time.perf_counter()
        oracle.periodogram(s.t, s.y, s.dy, s.f0, s.df, k)
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    frac = nk / s.nf
    value = args.steps * frac / sum(times)
    cores = oracle.threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": desc, "precision": "fp64 direct sums", "nd": s.nd, "nf": s.nf},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{nk} seeded random frequencies of the {s.nf}-frequency "
                                   f"grid per step (all {s.nd} points)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------ our arm

def run_ours(args):
    import numpy as np
    import torch

    world, rank, local, pg = dist_setup()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)

    import paper_2409_08090_gb300 as nl
    nl.build.build()
    nl.load_library()

    s, desc = workload(args.workload, rank)
    eps = eps_for(args.precision)
    plan = nl.Plan(s.nd, s.nf, eps, args.precision, device=local, upsampling=args.upsampling)
    info = plan.info
    t = torch.tensor(s.t, dtype=torch.float64, device=device)
    y = torch.tensor(s.y, dtype=torch.float64, device=device)
    dy = torch.tensor(s.dy, dtype=torch.float64, device=device)
    out = torch.empty(s.nf, dtype=torch.float64, device=device)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=device)   # 256 MB > L2

    for _ in range(args.warmup):
        plan.execute(t, y, dy, s.f0, s.df, out=out, sync=False)
    st = nl.ls_sync(plan.handle)
    if st != 0:
        raise SystemExit(f"device status after warm-up: {nl.ls_status_str(st)}")

    nl.ls_timing_enable(plan.handle, True)
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    barrier(pg)
    torch.cuda.synchronize()
    k0 = nl.ls_kernel_launches()
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(float(i))                 # evict L2 (outside the step's events)
        ev0[i].record()
        plan.execute(t, y, dy, s.f0, s.df, out=out, sync=False)
        ev1[i].record()
    torch.cuda.synchronize()
    kernels = nl.ls_kernel_launches() - k0
    barrier(pg)
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    st = nl.ls_sync(plan.handle)
    if st != 0:
        raise SystemExit(f"device status after timing: {nl.ls_status_str(st)}")
    step_ms = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
    stage_ms, nexec = nl.ls_timing_report(plan.handle)
    nl.ls_timing_enable(plan.handle, False)
    total_ms = allreduce_max(sum(step_ms), pg, device)
    value = world * args.steps / (total_ms * 1e-3)

    # -- dominant kernel roofline (spread + FFT passes), live event timing
    avg = {name: stage_ms[i] / max(nexec, 1) for i, name in enumerate(nl.STAGE_NAMES)}
    alg = algorithmic_bytes(info, s.nd, s.nf, args.precision)
    dom = max(("pass_a_spread_fft", "pass_b_fft_deconv_power"), key=lambda k: avg[k])
    peak, peak_kind = measured_hbm_peak()
    kern_gbs = {k: alg[k] / (avg[k] * 1e-3) / 1e9 for k in alg if avg.get(k, 0) > 0}
    kname = "k_passA" if dom == "pass_a_spread_fft" else "k_passB"
    roofline = {"bound": "hbm", "kernel": kname, "achieved": kern_gbs[dom], "peak": peak,
                "peak_kind": f"{peak_kind} hbm_gbs (copy)", "unit": "GB/s",
                "frac": kern_gbs[dom] / peak,
                "traffic": recorded_traffic(kname, args.precision, args.workload),
                "algorithmic_bytes": alg[dom], "avg_ms": avg[dom]}
    spread_fft_ms = avg["pass_a_spread_fft"] + avg["pass_b_fft_deconv_power"]
    spread_fft_bytes = alg["pass_a_spread_fft"] + alg["pass_b_fft_deconv_power"]

    P_gpu = out.cpu().numpy()

    # -- end to end through the C-ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        th = torch.from_numpy(s.t).pin_memory().numpy()
        yh = torch.from_numpy(s.y).pin_memory().numpy()
        dyh = torch.from_numpy(s.dy).pin_memory().numpy()
        ph = torch.empty(s.nf, dtype=torch.float64).pin_memory().numpy()
        nsteps = max(4, min(args.steps, 10))
        plan.execute_host(th, yh, dyh, s.f0, s.df, out=ph)
        barrier(pg)
        t0 = time.perf_counter()
        for _ in range(nsteps):
            plan.execute_host(th, yh, dyh, s.f0, s.df, out=ph)
        dt_serial = allreduce_max(time.perf_counter() - t0, pg, device)
        # Two host threads, each with its own plan, CUDA stream and pinned
        # buffers, calling the same host-buffer entry point: one periodogram's
        # copies overlap the other's kernels (the way a service would call it).
        import threading
        plan2 = nl.Plan(s.nd, s.nf, eps, args.precision, device=local,
                        upsampling=args.upsampling)
        bufs = [(th, yh, dyh, ph)]
        bufs.append(tuple(torch.from_numpy(a.copy()).pin_memory().numpy()
                          for a in (s.t, s.y, s.dy)) +
                    (torch.empty(s.nf, dtype=torch.float64).pin_memory().numpy(),))
        streams = [torch.cuda.Stream(device=device) for _ in range(2)]
        per = nsteps // 2

        def worker(i):
            pl = plan if i == 0 else plan2
            with torch.cuda.stream(streams[i]):
                for _ in range(per):
                    a, b_, c_, o = bufs[i]
                    pl.execute_host(a, b_, c_, s.f0, s.df, out=o)

        worker(1)                      # warm the second plan
        barrier(pg)
        t0 = time.perf_counter()
        th2 = [threading.Thread(target=worker, args=(i,)) for i in range(2)]
        for x in th2:
            x.start()
        for x in th2:
            x.join()
        dt = allreduce_max(time.perf_counter() - t0, pg, device)
        plan2.close()
        e2e = {"value": world * 2 * per / dt, "unit": UNIT,
               "h2d_bytes_per_step": 3 * 8 * s.nd, "d2h_bytes_per_step": 8 * s.nf,
               "steps": 2 * per, "host_buffers": "pinned", "api": "Plan.execute_host",
               "concurrency": "2 host threads, a plan and a CUDA stream each",
               "serial": {"value": world * nsteps / dt_serial, "steps": nsteps,
                          "concurrency": "1 host thread"}}

    # -- the library FFT as a reference for the FFT step: cuFFT (through
    # torch.fft) on the same three fine grids, complex, in the plan's precision,
    # out of place.  Our FFT is fused with spreading (pass A) and with
    # deconvolution and power (pass B); cuFFT alone does none of that.
    fft_ref = None
    if info.n <= 64_000_000 and not args.no_fft_reference:
        cdt = torch.complex64 if args.precision == "fp32" else torch.complex128
        grids = torch.randn(3, info.n, dtype=cdt, device=device)
        for _ in range(3):
            torch.fft.fft(grids)
        torch.cuda.synchronize()
        fe0 = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        fe1 = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        for i in range(5):
            flush.fill_(float(i))
            fe0[i].record()
            torch.fft.fft(grids)
            fe1[i].record()
        torch.cuda.synchronize()
        fms = sorted(a.elapsed_time(b) for a, b in zip(fe0, fe1))
        fft_ref = {"library": "cuFFT via torch.fft.fft (reference only, not on the path)",
                   "grids": 3, "n": int(info.n), "dtype": str(cdt).replace("torch.", ""),
                   "ms_median": fms[len(fms) // 2],
                   "ours_passes_ms": spread_fft_ms,
                   "note": "library: the three n-point FFTs alone; ours: pass A (spread + "
                           "column FFTs + twiddle) plus pass B (row FFTs + deconvolution + power)"}
        del grids

    # -- small problems: launch-bound, so compare direct calls with a CUDA-graph
    # replay of the same pipeline (back to back on resident buffers, no flush)
    graph = None
    if s.nf <= 1_000_000:
        calls = 200
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(calls):
            plan.execute(t, y, dy, s.f0, s.df, out=out, sync=False)
        torch.cuda.synchronize()
        direct = calls / (time.perf_counter() - t0)
        g = plan.graph(t, y, dy, s.f0, s.df, out=out)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(calls):
            g.replay()
        torch.cuda.synchronize()
        replay = calls / (time.perf_counter() - t0)
        g.sync()
        graph = {"direct": direct, "graph": replay, "unit": UNIT, "calls": calls,
                 "note": "back to back on resident buffers, no L2 flush (launch-bound regime)"}
        del g
    plan.close()

    # -- the paper's precision: the FP64 path (eps 1e-9) on the same series,
    # timed like the headline (L2 flushed, CUDA events), with its own accuracy
    # block (same oracle sample) and two roofs: HBM for pass A's algorithmic
    # bytes, and the FP32 issue rate its double-float FFTs run on
    fp64 = None
    P64 = None
    if not args.no_fp64_path and args.precision == "fp32":
        p64 = nl.Plan(s.nd, s.nf, 1e-9, "fp64", device=local)
        info64 = p64.info
        for _ in range(3):
            p64.execute(t, y, dy, s.f0, s.df, out=out, sync=False)
        nl.ls_timing_enable(p64.handle, True)
        n64 = args.steps
        a = [torch.cuda.Event(enable_timing=True) for _ in range(n64)]
        b = [torch.cuda.Event(enable_timing=True) for _ in range(n64)]
        for i in range(n64):
            flush.fill_(float(i))
            a[i].record()
            p64.execute(t, y, dy, s.f0, s.df, out=out, sync=False)
            b[i].record()
        torch.cuda.synchronize()
        if nl.ls_sync(p64.handle) != 0:
            raise SystemExit("device status after the FP64 steps")
        ms64 = [x.elapsed_time(z) for x, z in zip(a, b)]
        sm64, c64 = nl.ls_timing_report(p64.handle)
        avg64 = {nm: sm64[i] / max(c64, 1) for i, nm in enumerate(nl.STAGE_NAMES)}
        P64 = out.cpu().numpy()
        alg64 = algorithmic_bytes(info64, s.nd, s.nf, "fp64")
        hbm64 = alg64["pass_a_spread_fft"] / (avg64["pass_a_spread_fft"] * 1e-3) / 1e9
        props = torch.cuda.get_device_properties(local)
        fft_flops = 3 * 5 * info64.n * float(np.log2(info64.n))
        passes_s = (avg64["pass_a_spread_fft"] + avg64["pass_b_fft_deconv_power"]) * 1e-3
        roof = fp32_issue_roof(props.multi_processor_count)
        fp64 = {"value": n64 / (sum(ms64) * 1e-3), "unit": UNIT, "eps": 1e-9, "steps": n64,
                "ms_per_step": sum(ms64) / n64, "p50_ms": statistics.median(ms64),
                "config": {"n": info64.n, "n1": info64.n1, "n2": info64.n2,
                           "width": info64.width, "sigma": info64.sigma},
                "stage_ms": avg64,
                "roofline": {
                    "hbm": {"bound": "hbm", "kernel": "k_passA", "achieved": hbm64,
                            "peak": peak, "unit": "GB/s", "frac": hbm64 / peak,
                            "algorithmic_bytes": alg64["pass_a_spread_fft"]},
                    "fp32_issue": {"bound": "alu", "achieved": fft_flops / passes_s / 1e12,
                                   "peak": roof["tflops"], "unit": "TFLOP/s",
                                   "frac": fft_flops / passes_s / 1e12 / roof["tflops"],
                                   "work": "5 n log2 n flops per fine-grid FFT, 3 grids, over "
                                           "pass A + pass B time (which also spread, "
                                           "deconvolve and evaluate the power)",
                                   "derivation": roof["derivation"]}}}
        p64.close()

    # -- batched and served workloads (BASELINE's configurations 3-5), compact
    extras = {}
    if world == 1 and args.workload == "single_large" and not args.no_extras:
        import copy

        def sub(**kw):
            a2 = copy.copy(args)
            a2.__dict__.update(kw)
            return a2
        del flush
        torch.cuda.empty_cache()
        uni = run_batch(sub(workload="uniform_batch", steps=5, warmup=2, batch_scale=1.0,
                            batch_mode="graph"))
        extras["uniform_batch"] = compact_batch(uni)
        rag = run_batch(sub(workload="ragged_batch", steps=3, warmup=1, batch_scale=1.0,
                            batch_mode="graph", no_e2e=True))
        extras["ragged_batch"] = compact_batch(rag)
        extras["ragged_batch"]["note"] = (
            "10,000 series as configured; e2e left out here (its two pinned output buffers "
            "would hold 28 GB of host memory): bench.py --workload ragged_batch reports it")
        srv = run_serving(sub(batch_scale=1.0, serving_results="host"))
        extras["serving"] = compact_serving(srv)
        plain = srv["plain_fp64_one_at_a_time"]["value_by_eps"]
        top32 = srv["per_rate"].get("20000_fp32", {}).get("periodograms_per_s")
        extras["equal_accuracy"] = {
            "plain_fp64_eps_1e-6_per_s": plain.get("eps_1e-06"),
            "batched_fp32_over_plain_fp64": rag["value"] / plain["eps_1e-06"],
            "served_fp32_over_plain_fp64": (top32 / plain["eps_1e-06"]) if top32 else None,
            "note": "FP32 at eps 1e-6 against the plain one-at-a-time FP64 path at eps 1e-6 "
                    "(the same rel-l2 class), on series drawn like the ragged batch; served: "
                    "saturated at 20,000 offered requests/s"}

    if rank != 0:
        if pg:
            import torch.distributed as dist
            dist.destroy_process_group()
        return 0

    cpu = None
    accuracy = None
    if not args.no_cpu_baseline and world == 1:
        k, P_o, dt, cores = oracle_sample(s, args.cpu_seconds)
        nk = len(k)
        cpu = {"value": (nk / s.nf) / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{nk} seeded random frequencies of the {s.nf}-frequency grid, all "
                         f"{s.nd} points, FP64 direct sums ({dt:.1f} s)"}
        P_g = P_gpu[k]
        accuracy = {"rel_l2": float(np.linalg.norm(P_g - P_o) / np.linalg.norm(P_o)),
                    "max_abs": float(np.max(np.abs(P_g - P_o))),
                    "frequencies": nk, "against": "FP64 oracle (direct sums)"}
        if fp64 is not None:
            d64 = P64[k] - P_o
            fp64["accuracy"] = {"rel_l2": float(np.linalg.norm(d64) / np.linalg.norm(P_o)),
                                "max_abs": float(np.max(np.abs(d64))), "frequencies": nk,
                                "against": "FP64 oracle (direct sums), the same sample"}

    ms_sorted = sorted(step_ms)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": sum(step_ms) / len(step_ms),
        "p50_ms": statistics.median(step_ms),
        "p99_ms": ms_sorted[min(len(ms_sorted) - 1, int(round(0.99 * (len(ms_sorted) - 1))))],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision == "fp32" else "f64", "data": "synthetic",
        "config": {"workload": desc, "nd": s.nd, "nf": s.nf, "eps": eps,
                   "precision": args.precision, "n": info.n, "n1": info.n1, "n2": info.n2,
                   "width": info.width, "sigma": info.sigma,
                   "l2": "flushed between steps (256 MB write, untimed)",
                   "parallelism": f"independent series per GPU x{world}"},
        "roofline": roofline,
        "spread_fft": {"ms": spread_fft_ms, "algorithmic_bytes": spread_fft_bytes,
                       "achieved_gbs": spread_fft_bytes / (spread_fft_ms * 1e-3) / 1e9,
                       "frac_of_peak": spread_fft_bytes / (spread_fft_ms * 1e-3) / 1e9 / peak},
        "stage_ms": avg, "stage_gbs": kern_gbs,
        "accuracy": accuracy, "cpu_baseline": cpu, "e2e": e2e, "fp64_path": fp64,
        "graph_replay": graph, "fft_reference": fft_ref,
        **extras,
        "gpu_launches": kernels,
        "clocks": clk, "wall_s": wall,
    }
    print(json.dumps(line), flush=True)
    if pg:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------- batch workloads

def batch_workload(name: str, rank: int, scale: float = 1.0):
    """Packed many-series workload: (offsets, t, y, dy, f0[], df[], nf[], desc)."""
    import numpy as np
    from paper_2409_08090_gb300 import workloads as W
    if name == "uniform_batch":
        ns = max(8, int(4096 * scale))
        t, Y, dy, f0, df, nf = W.uniform_batch(seed=W.BASE_SEED + 2 + 1000 * rank, nseries=ns)
        nd = t.shape[0]
        # shared time array: t and dy hold nd values, Y the series row by row
        offsets = np.arange(ns + 1, dtype=np.int64) * nd
        desc = (f"uniform_batch: {ns} series on one time array (shared-times path), Nd=1e4 over "
                "[0,1000) d, Nf=1.2e5, f0=1e-3, df=1e-4, dy=1")
        return (offsets, t, Y.reshape(-1), dy, np.full(ns, f0), np.full(ns, df),
                np.full(ns, nf, np.int64), desc)
    ns = max(16, int(10_000 * scale))
    series = W.ragged_batch(seed=W.BASE_SEED + 3 + 1000 * rank, nseries=ns)
    offsets = np.zeros(ns + 1, dtype=np.int64)
    offsets[1:] = np.cumsum([s.nd for s in series])
    desc = (f"ragged_batch: {ns} series, Nd log-uniform in [100, 1e5], baselines log-uniform in "
            "[10, 3650] d with gaps, lognormal dy, Nf = 12 Nd, df = 1/(5T), f0 = df")
    return (offsets, np.concatenate([s.t for s in series]), np.concatenate([s.y for s in series]),
            np.concatenate([s.dy for s in series]), np.array([s.f0 for s in series]),
            np.array([s.df for s in series]), np.array([s.nf for s in series], np.int64), desc)


def run_batch(args):
    import numpy as np
    import torch

    world, rank, local, pg = dist_setup()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    import paper_2409_08090_gb300 as nl
    nl.build.build()
    nl.load_library()

    offsets, th, yh, dyh, f0, df, nf, desc = batch_workload(args.workload, rank, args.batch_scale)
    ns = len(nf)
    eps = eps_for(args.precision)
    plan = nl.Plan(2, 1, eps, args.precision, device=local, upsampling=args.upsampling)
    t = torch.from_numpy(th).to(device)
    y = torch.from_numpy(yh).to(device)
    dy = torch.from_numpy(dyh).to(device)
    out = torch.empty(int(nf.sum()), dtype=torch.float64, device=device)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=device)
    shared = args.workload == "uniform_batch"
    nd0 = int(offsets[1] - offsets[0])

    def direct():
        if shared:
            plan.execute_shared(t, y.view(ns, nd0), dy, float(f0[0]), float(df[0]), int(nf[0]),
                                out=out.view(ns, int(nf[0])), sync=False)
        else:
            plan.execute_batch(t, y, dy, offsets, f0, df, nf, out=out, sync=False)

    # prepared layout (host work once) and its recorded graph
    tp0 = time.perf_counter()
    if shared:
        pb = plan.prepare_shared(ns, nd0, float(f0[0]), float(df[0]), int(nf[0]))
        yv, outv = y.view(ns, nd0), out.view(ns, int(nf[0]))
    else:
        pb = plan.prepare_batch(offsets, f0, df, nf)
        yv, outv = y, out
    prepare_s = time.perf_counter() - tp0

    def prepared():
        pb.run(t, yv, dy, out=outv, sync=False)

    k0 = nl.ls_kernel_launches()
    prepared()
    kernels_per_step = nl.ls_kernel_launches() - k0
    graph = pb.graph(t, yv, dy, out=outv)
    modes = {"direct": direct, "prepared": prepared, "graph": graph.replay}
    step = modes[args.batch_mode]

    # the other modes, briefly (3 steps each, L2 flushed), for the record
    mode_rates = {}
    for name, fn in modes.items():
        fn()
        torch.cuda.synchronize()
        ms, host = [], []
        for i in range(3):
            flush.fill_(float(i))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            h0 = time.perf_counter()
            fn()
            host.append((time.perf_counter() - h0) * 1e3)
            b.record()
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        mode_rates[name] = {"periodograms_per_s": ns / (statistics.median(ms) * 1e-3),
                            "ms": statistics.median(ms), "host_ms": statistics.median(host)}
    for _ in range(args.warmup):
        step()
    st = nl.ls_sync(plan.handle)
    if st != 0:
        raise SystemExit(f"{args.workload}: device status after warm-up: {nl.ls_status_str(st)}")
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    barrier(pg)
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(float(i))
        ev0[i].record()
        step()
        ev1[i].record()
    torch.cuda.synchronize()
    barrier(pg)
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    st = nl.ls_sync(plan.handle)
    if st != 0:
        raise SystemExit(f"{args.workload}: device status after timing: {nl.ls_status_str(st)}")
    step_ms = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
    total_ms = allreduce_max(sum(step_ms), pg, device)
    value = world * ns * args.steps / (total_ms * 1e-3)
    pb_info = pb.describe()
    P_gpu = out.cpu().numpy()
    out_off = np.zeros(ns, dtype=np.int64)
    out_off[1:] = np.cumsum(nf)[:-1]

    # whole-step roofline: what one batch must move
    cx = 8 if args.precision == "fp32" else 16
    cells = 0
    if shared:
        p = nl.ls_choose_params(int(nf[0]), eps, nl._prec_code(args.precision), max_nd=nd0,
                                upsampling=args.upsampling)
        cells = (ns + 2) * p["n"]
    for k in range(0 if shared else ns):
        p = nl.ls_choose_params(int(nf[k]), eps, nl._prec_code(args.precision),
                                max_nd=int(offsets[k + 1] - offsets[k]), upsampling=args.upsampling)
        cells += 3 * p["n"]
    alg = 8 * (th.size + yh.size + dyh.size) + 8 * int(nf.sum()) + 2 * cells * cx
    peak, peak_kind = measured_hbm_peak()
    achieved = alg / (sum(step_ms) / len(step_ms) * 1e-3) / 1e9
    roofline = {"bound": "hbm", "kernel": "whole batch step (all kernels)", "achieved": achieved,
                "peak": peak, "peak_kind": f"{peak_kind} hbm_gbs (copy)", "unit": "GB/s",
                "frac": achieved / peak, "traffic": None, "algorithmic_bytes": alg}

    e2e = None
    if not args.no_e2e:
        tp = torch.from_numpy(th).pin_memory()
        yp = torch.from_numpy(yh).pin_memory()
        dp = torch.from_numpy(dyh).pin_memory()
        phs = [torch.empty(out.numel(), dtype=torch.float64).pin_memory() for _ in range(2)]
        # serial: copy in, compute, copy out and wait, step after step
        nser = 2
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(nser):
            t.copy_(tp, non_blocking=True)
            y.copy_(yp, non_blocking=True)
            dy.copy_(dp, non_blocking=True)
            step()
            phs[0].copy_(out, non_blocking=True)
            torch.cuda.synchronize()
        dt_serial = allreduce_max(time.perf_counter() - t0, pg, device)
        # pipelined over two buffer sets: step i+1's inputs go in and step i-1's
        # results come out (copy streams) while step i computes
        t1, y1, dy1, o1 = (a.clone() for a in (t, y, dy, out))   # valid values for recording
        sets = [(t, y, dy, out), (t1, y1, dy1, o1)]
        views = [(yv, outv),
                 (y1.view(ns, nd0), o1.view(ns, int(nf[0]))) if shared else (y1, o1)]
        graph1 = pb.graph(t1, views[1][0], dy1, out=views[1][1]) \
            if args.batch_mode == "graph" else None

        def run_set(k):
            tk, _, dyk, _ = sets[k]
            yk, ok = views[k]
            if args.batch_mode == "graph":
                (graph if k == 0 else graph1).replay()
            elif args.batch_mode == "prepared":
                pb.run(tk, yk, dyk, out=ok, sync=False)
            elif shared:
                plan.execute_shared(tk, yk, dyk, float(f0[0]), float(df[0]), int(nf[0]), out=ok,
                                    sync=False)
            else:
                plan.execute_batch(tk, yk, dyk, offsets, f0, df, nf, out=ok, sync=False)

        nsteps = max(4, min(args.steps, 8))
        cs = torch.cuda.current_stream(device)
        h2d, d2h = torch.cuda.Stream(device=device), torch.cuda.Stream(device=device)
        ev_in, ev_done, ev_out = ([torch.cuda.Event() for _ in range(nsteps)] for _ in range(3))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(nsteps):
            k = i % 2
            tk, yk, dyk, ok = sets[k]
            with torch.cuda.stream(h2d):
                if i >= 2:
                    h2d.wait_event(ev_done[i - 2])     # step i-2 has read this set's inputs
                tk.copy_(tp, non_blocking=True)
                yk.copy_(yp, non_blocking=True)
                dyk.copy_(dp, non_blocking=True)
                ev_in[i].record(h2d)
            cs.wait_event(ev_in[i])
            if i >= 2:
                cs.wait_event(ev_out[i - 2])           # this set's results are copied out
            run_set(k)
            ev_done[i].record(cs)
            with torch.cuda.stream(d2h):
                d2h.wait_event(ev_done[i])
                phs[k].copy_(ok, non_blocking=True)
                ev_out[i].record(d2h)
        torch.cuda.synchronize()
        dt = allreduce_max(time.perf_counter() - t0, pg, device)
        if nl.ls_sync(plan.handle) != 0:
            raise SystemExit("device status after the e2e steps")
        e2e = {"value": world * ns * nsteps / dt, "unit": UNIT,
               "h2d_bytes_per_step": int(8 * (th.size + yh.size + dyh.size)), "d2h_bytes_per_step": int(8 * nf.sum()),
               "steps": nsteps, "host_buffers": "pinned",
               "api": {"graph": "GraphedBatch.replay", "prepared": "PreparedBatch.run",
                       "direct": "Plan.execute_batch"}[args.batch_mode],
               "pipelining": "two device buffer sets; host-to-device and device-to-host copies on "
                             "their own streams overlap the neighbouring steps' compute",
               "serial": {"value": world * ns * nser / dt_serial, "steps": nser,
                          "pipelining": "none (copy in, compute, copy out, wait)"}}
        del graph1
    del graph
    pb.close()
    plan.close()
    if rank != 0:
        return None
    cpu = accuracy = None
    if not args.no_cpu_baseline and world == 1:
        import oracle
        oracle.build()
        rng = np.random.default_rng(7)
        pick = rng.choice(ns, min(8, ns), replace=False)
        errs, tot_freq, tot_time = [], 0, 0.0
        for k in pick:
            a, b = offsets[k], offsets[k + 1]
            ts, ds = (th, dyh) if shared else (th[a:b], dyh[a:b])
            kk = np.sort(rng.choice(int(nf[k]), min(int(nf[k]), 256), replace=False)).astype(np.int64)
            t0 = time.perf_counter()
            P_o = oracle.periodogram(ts, yh[a:b], ds, f0[k], df[k], kk)
            tot_time += time.perf_counter() - t0
            tot_freq += len(kk) / nf[k]
            P_g = P_gpu[out_off[k] + kk]
            errs.append((np.linalg.norm(P_g - P_o) / np.linalg.norm(P_o), np.max(np.abs(P_g - P_o))))
        cpu = {"value": tot_freq / tot_time, "unit": UNIT, "cores": oracle.threads(),
               "kind": "oracle", "sample": f"{len(pick)} random series x <=256 random frequencies"}
        accuracy = {"rel_l2_max": float(max(e[0] for e in errs)),
                    "max_abs": float(max(e[1] for e in errs)), "series": len(pick),
                    "against": "FP64 oracle (direct sums)"}
    ms_sorted = sorted(step_ms)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": sum(step_ms) / len(step_ms),
        "p50_ms": statistics.median(step_ms),
        "p99_ms": ms_sorted[min(len(ms_sorted) - 1, int(round(0.99 * (len(ms_sorted) - 1))))],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision == "fp32" else "f64", "data": "synthetic",
        "config": {"workload": desc, "series": ns, "points": int(offsets[-1]),
                   "frequencies": int(nf.sum()), "eps": eps, "precision": args.precision,
                   "l2": "flushed between steps (256 MB write, untimed)",
                   "parallelism": f"independent batches per GPU x{world}"},
        "roofline": roofline, "accuracy": accuracy, "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": kernels_per_step * args.steps, "clocks": clk, "wall_s": wall,
        "batch_mode": args.batch_mode, "modes": mode_rates, "prepare_s": prepare_s,
        "prepared_layout": pb_info,
    }
    if pg:
        import torch.distributed as dist
        dist.destroy_process_group()
    return line


def run_serving(args):
    """Poisson arrivals of ragged-mix requests (half FP32 at eps 1e-6, half FP64
    at eps 1e-9) into the continuous-batching server; p50/p99 latency and
    periodograms/s per arrival rate, beside the plain one-at-a-time FP64 path."""
    import threading

    import numpy as np
    import torch

    import paper_2409_08090_gb300 as nl
    from paper_2409_08090_gb300 import workloads as W
    from paper_2409_08090_gb300.serving import PeriodogramServer
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if int(os.environ.get("RANK", "0")) != 0:
        return None
    nl.build.build()
    nl.load_library()
    pool = W.ragged_batch(seed=W.BASE_SEED + 4, nseries=max(64, int(600 * args.batch_scale)))
    rates = [200.0, 1000.0, 5000.0]
    duration = 2.0 * args.batch_scale
    srv = PeriodogramServer(memory_budget=60 << 30, streams=2, max_batch=4096,
                            results=args.serving_results)
    if args.serving_copy_limit is not None:
        srv.copy_limit = int(args.serving_copy_limit)
    # warm the plans and every grid class of the pool once (a class's tables
    # are built on its first request), so the timed runs allocate nothing
    warm = [srv.submit(s.t, s.y, s.dy, s.f0, s.df, s.nf, p) for s in pool
            for p in ("fp32", "fp64")]
    for f in warm:
        f.result(timeout=600)
    del warm, f
    per_rate = {}
    runs = [(r, "mixed") for r in rates] + [(rates[-1], "fp32"), (4 * rates[-1], "fp32")]
    # a few served results of the busiest mixed run are kept for the accuracy
    # check against the oracle (the cpu_baseline leg)
    kept, kept_req = {}, {}
    for rate, mix in runs:
        n = max(16, int(rate * duration))
        arrivals = W.poisson_arrivals(rate, n, seed=int(rate))
        rng = np.random.default_rng(int(rate) + 1)
        picks = rng.integers(0, len(pool), n)
        if mix == "mixed":
            precs = np.where(rng.random(n) < 0.5, "fp32", "fp64")
        else:
            precs = np.full(n, "fp32")
        keep = set()
        if mix == "mixed" and rate == rates[-1] and not args.no_cpu_baseline:
            for p in ("fp32", "fp64"):
                keep.update(int(i) for i in np.flatnonzero(precs == p)[:4])
            kept_req.update({i: (int(picks[i]), str(precs[i])) for i in keep})
        srv.completed.clear()
        t0 = time.perf_counter()
        left = [n]
        failures = []
        all_done = threading.Event()
        lock = threading.Lock()

        def consume(i, f):
            # the client reads each result as it arrives and then drops it
            exc = f.exception()
            if exc is not None:
                failures.append(repr(exc))
            elif i in keep:
                kept[i] = f.result()
            elif args.serving_results == "host":
                _ = float(f.result()[0])
            with lock:
                left[0] -= 1
                if left[0] == 0:
                    all_done.set()

        def client():
            for i in range(n):
                delay = t0 + arrivals[i] - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
                s = pool[picks[i]]
                srv.submit(s.t, s.y, s.dy, s.f0, s.df, s.nf, str(precs[i])).add_done_callback(
                    functools.partial(consume, i))

        th = threading.Thread(target=client)
        th.start()
        th.join()
        if not all_done.wait(timeout=600) or failures:
            raise SystemExit(f"serving run at {rate}/s did not complete: {failures[:3]}")
        st = srv.stats()
        st["offered_rate"] = rate
        st["precisions"] = "50/50 fp32 eps 1e-6 / fp64 eps 1e-9" if mix == "mixed" else "fp32 eps 1e-6"
        st["frequencies_per_request_mean"] = float(np.mean([pool[k].nf for k in picks]))
        per_rate[(str(int(rate)) if mix == "mixed" else f"{int(rate)}_fp32")] = st
    srv.close()
    # plain one-at-a-time FP64 path (plans reused, plan creation not timed)
    plans = {}
    sample = [pool[k] for k in np.random.default_rng(3).integers(0, len(pool), 96)]
    dev = torch.device("cuda:0")
    tens = [(torch.tensor(s.t, device=dev), torch.tensor(s.y, device=dev),
             torch.tensor(s.dy, device=dev)) for s in sample]
    plain = {}
    for eps64 in (1e-9, 1e-6):
        for s in sample:
            if (s.nf, eps64) not in plans:
                plans[(s.nf, eps64)] = nl.Plan(s.nd, s.nf, eps64, "fp64")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for s, (t, y, dy) in zip(sample, tens):
            plans[(s.nf, eps64)].execute(t, y, dy, s.f0, s.df)
        torch.cuda.synchronize()
        plain[f"eps_{eps64:g}"] = len(sample) / (time.perf_counter() - t0)
    for p in plans.values():
        p.close()
    cpu = accuracy = None
    if kept:
        import oracle
        oracle.build()
        rng = np.random.default_rng(17)
        errs = {"fp32": [], "fp64": []}
        tot_freq = tot_time = 0.0
        for i, res in sorted(kept.items()):
            k_pool, prec = kept_req[i]
            s = pool[k_pool]
            P = res.cpu().numpy() if hasattr(res, "cpu") else np.asarray(res)
            k = np.sort(rng.choice(s.nf, min(s.nf, 256), replace=False)).astype(np.int64)
            t0 = time.perf_counter()
            P_o = oracle.periodogram(s.t, s.y, s.dy, s.f0, s.df, k)
            tot_time += time.perf_counter() - t0
            tot_freq += len(k) / s.nf
            errs[prec].append((float(np.linalg.norm(P[k] - P_o) / np.linalg.norm(P_o)),
                               float(np.max(np.abs(P[k] - P_o)))))
        cpu = {"value": tot_freq / tot_time, "unit": UNIT, "cores": oracle.threads(),
               "kind": "oracle",
               "sample": f"{len(kept)} served requests x <=256 random frequencies"}
        accuracy = {p: {"rel_l2_max": max(e[0] for e in v), "max_abs": max(e[1] for e in v),
                        "requests": len(v)} for p, v in errs.items() if v}
        accuracy["against"] = "FP64 oracle (direct sums), requests of the busiest mixed run"
        kept.clear()
    top = per_rate[str(int(rates[-1]))]
    line = {
        "metric": METRIC, "value": top.get("periodograms_per_s"), "unit": UNIT, "n_gpus": world,
        "steps": None, "warmup": 1, "p50_ms": top.get("p50_ms"), "p99_ms": top.get("p99_ms"),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic",
        "config": {"workload": "serving: Poisson arrivals of ragged-mix series (Nd log-uniform "
                               "in [100, 1e5], Nf = 12 Nd), 50/50 FP32 eps 1e-6 / FP64 eps 1e-9, "
                               "60 GB admission budget, 2 streams",
                   "results": args.serving_results, "copy_limit": srv.copy_limit,
                   "pool_series": len(pool), "duration_s": duration},
        "per_rate": per_rate,
        "plain_fp64_one_at_a_time": {"value_by_eps": plain, "unit": UNIT, "series": len(sample),
                                     "note": "ls_execute per request, plans reused, same pool"},
        "accuracy": accuracy, "cpu_baseline": cpu,
    }
    return line


def compact_batch(line: dict) -> dict:
    """The batch line's figures for a sub-block of the default line."""
    keep = ("value", "unit", "ms_per_step", "p50_ms", "p99_ms", "steps", "gpu_launches",
            "batch_mode", "prepare_s")
    out = {k: line.get(k) for k in keep}
    out["workload"] = line["config"]["workload"]
    out["series"] = line["config"]["series"]
    out["roofline"] = {k: line["roofline"][k] for k in ("bound", "achieved", "peak", "unit", "frac")}
    out["accuracy"] = line.get("accuracy")
    out["modes"] = {k: v["periodograms_per_s"] for k, v in line.get("modes", {}).items()}
    e2e = line.get("e2e")
    out["e2e"] = None if e2e is None else {k: e2e[k] for k in ("value", "unit", "h2d_bytes_per_step",
                                                              "d2h_bytes_per_step")}
    return out


def compact_serving(line: dict) -> dict:
    """The serving line's figures for a sub-block of the default line."""
    keep = ("requests", "p50_ms", "p99_ms", "periodograms_per_s", "offered_rate", "batches",
            "peak_device_bytes", "plan_bytes", "budget")
    return {"per_rate": {r: {k: v.get(k) for k in keep} for r, v in line["per_rate"].items()},
            "plain_fp64_one_at_a_time": line["plain_fp64_one_at_a_time"],
            "accuracy": line.get("accuracy"), "config": line["config"]}


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload in ("uniform_batch", "ragged_batch"):
        line = run_batch(args)
    elif args.workload == "serving":
        line = run_serving(args)
    else:
        return run_ours(args)
    if line is not None:
        print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
