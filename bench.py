"""Benchmark: CS-WGS point-cloud holograms on GB300.

One step = the whole hot path for a batch of holograms resident in HBM: spot
preparation, 30 iterations (28 over random pixel subsets of 1/8 of the
pupil, 2 over all pixels), the final full back-propagation writing each phase
map and the full forward projection giving e and u; one persistent launch
per iteration for the whole batch, replayed from a CUDA graph.

Workload: 64 holograms of P = 1152 (M = 1152^2), N = 100 spots, alpha, beta
~ U[-P/4, P/4] cycles, gamma ~ U[-10, 10] waves, theta^0 ~ U[0, 2 pi), one
seed per hologram.  Prints one JSON line: holograms/s, p50/p99 latency, the
roofline of the dominant iteration kernel (tensor cores: algorithmic flops
against the measured dense BF16 peak; CUDA cores: sine/cosine results against
the SFU peak, or complex multiply-adds against the FP32 peak), the FP64 GPU
baseline with its per-hologram latency, the compressed-iteration sweep over
N and c, the headline shape on a rotated 10 x 10 grid, the serving streams
(Poisson arrivals of mixed requests), the FP64 CPU oracle on a bounded
sample, and an end-to-end number through the C ABI with host buffers.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--quick]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "holograms/s and p50/p99 latency at M=1152^2, N=100, e,u>=0.9 vs FP64 GPU baseline"
SFU_PER_CLK_PER_SM = 16       # sine/cosine results per clock per SM (CUDA arithmetic throughput table)
FP32_LANES_PER_SM = 128       # FP32 fused multiply-adds per clock per SM
# DRAM bytes (read + write) per launch of the tensor-core iteration kernel at
# the default workload, from a one-kernel ncu capture of this bench with the
# caches left as the preceding launches leave them (two compressed launches;
# the two full iterations and the final pass, averaged: the factor tables are
# read once per launch, dirty lines of the R' table kernel are written back
# during it, the final pass writes the phase maps), keyed by launch kind and
# the tile-shape marker of the kernel that ran it.  Each is reported only
# while the sources of its kernel hash to the value they had when measured.
TRAFFIC_MEASURED = {("sub", 1): {"sha": "bfe821e4fddf3d48", "bytes": 300988928},
                    ("full", 2): {"sha": "bfe821e4fddf3d48", "bytes": 379298987}}
KERNEL_SOURCES = {"sub": ("cswgs_device.cuh", "tile.cuh", "kernels_fp32.cu"),
                  "full": ("cswgs_device.cuh", "tile.cuh", "kernels_fp32.cu", "kernels_tc.cu")}


def kernel_sha(kind):
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kind]:
        with open(os.path.join(ROOT, "paper_2003_05293_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(args, tile):
    default = (args.batch, args.P, args.N, args.c, args.iters) == (64, 1152, 100, 0.125, 30)
    out = []
    for kind, marker in (("sub", tile["threads"]), ("full", tile["full_threads"])):
        m = TRAFFIC_MEASURED.get((kind, marker))
        src = "full" if kind == "sub" and marker == SUBSET_TC else kind
        out.append(m["bytes"] if m and default and m["sha"] == kernel_sha(src) else None)
    return tuple(out)


# full_threads markers of the tensor-core kernels: kernel name, threads per block
TC_KERNELS = {2: ("iter_full_tcws_kernel (warp-specialised: 8 epilogue warps, a producer warp, a GEMM 1 warp "
                   "and a GEMM 2 warp)", 352)}


def kernel_name(tile, kind):
    """The kernel a launch kind ran on, from the batch's launch shapes."""
    if kind == "sub":
        if tile["threads"] == SUBSET_TC:
            return "iter_full_tcws_kernel (tensor cores: every pixel through both products, u zero outside S_j)"
        if tile["threads"] == SUBSET_GATHER:
            return ("iter_subset_gather_kernel (CUDA cores: the pixels of S_j only, one complex multiply-add per "
                    "pair and pass from the separable factors)")
        return "iter_subset_kernel<%d, %d> (CUDA cores: the pixels of S_j only, direct phasors)" % (
            tile["threads"], tile["pixels_per_thread"])
    if tile["full_threads"] in TC_KERNELS:
        return TC_KERNELS[tile["full_threads"]][0]
    return "iter_full_kernel<%d> (CUDA cores, separable)" % tile["full_threads"]


def dtype_label(tile):
    """The arithmetic the path computes in: FP32, or FP32-class split-BF16
    products accumulated in FP32 on the tensor cores."""
    if tile["threads"] == SUBSET_TC or tile["full_threads"] in TC_KERNELS:
        return "f32-class: split-bf16 x3 products, f32 accumulate (tensor cores); f32 epilogues; f64 e, u"
    return "f32 (f64 e, u)"


# threads marker of compressed iterations on the warp-specialised tensor-core
# kernel (dense products, u zero outside the subset), and on the subset-only
# gather kernel (CUDA cores, separable factors)
SUBSET_TC = 1
SUBSET_GATHER = 3


def tensor_peak():
    """The measured sustained dense BF16 peak (TFLOP/s) and its basis."""
    try:
        mp = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(mp["bf16_tflops_sustained"]), "measured (cuBLAS BF16, sustained: timed inside the step)"
    except (OSError, ValueError, KeyError):
        return 1700.0, "fallback (sustained)"


def subset_roofline(tile, pairs_sub_launch, n_sub, sub_ms, full_ms, sm_count, max_mhz, probe, traffic, args):
    """Roofline of the compressed-iteration launches.  On the CUDA-core kernel:
    2 SFU results (sin, cos) per subset pixel-spot pair and pass against the
    SFU peak.  On the tensor cores: algorithmic flops, 8 per subset pair and
    pass (one complex multiply-add), against the dense BF16 peak; the kernel
    runs every pixel (M / Mp times the subset) with 3 BF16 products per real
    product."""
    share = 100 * sub_ms / max(1e-9, sub_ms + full_ms)
    if tile["threads"] == SUBSET_TC:
        peak, basis = tensor_peak()
        ach = 8.0 * pairs_sub_launch * n_sub / (sub_ms * 1e-3) / 1e12 if n_sub else 0.0
        Mp = math.floor(args.c * args.P * args.P)
        return {"bound": "tensor", "pipe": "tcgen05 kind::f16 (BF16 in, FP32 accumulate)", "achieved": ach,
                "peak": peak, "unit": "TFLOP/s", "frac": ach / peak, "traffic": traffic,
                "peak_basis": "%s dense BF16 peak" % basis,
                "flops_basis": "8 flops (complex multiply-add) per subset pixel-spot pair and pass",
                "kernel": "iter_full_tcws_kernel on compressed launches: every pixel through both products, u zero "
                          "outside the subset (%d per step, %.1f%% of the step)" % (n_sub, share),
                "issued_tensor_flops_per_algorithmic": 3.0 * args.P * args.P / max(1, Mp),
                "ms_per_launch": sub_ms / max(1, n_sub),
                "sincos_equivalent": {
                    "achieved": 2.0 * pairs_sub_launch * n_sub / (sub_ms * 1e-3) / 1e9 if n_sub else 0.0,
                    "sfu_peak": sm_count * SFU_PER_CLK_PER_SM * max_mhz * 1e6 / 1e9, "unit": "G sincos/s",
                    "what": "the method's sine/cosine results per second (2 per subset pixel-spot pair and pass) "
                            "that the separable tensor-core products stand in for, against the SFU's peak: the "
                            "SFU roofline of a direct-phasor kernel does not bound this one"},
                "tile": {"threads": TC_KERNELS[2][1], "blocks": tile["blocks"], "pixels": "128 rows x 64 columns"}}
    if tile["threads"] == SUBSET_GATHER:
        fma_peak = sm_count * FP32_LANES_PER_SM * 2 * max_mhz * 1e6 / 1e12     # TFLOP/s
        ach = 8.0 * pairs_sub_launch * n_sub / (sub_ms * 1e-3) / 1e12 if n_sub else 0.0
        return {"bound": "alu", "pipe": "FP32 FMA", "achieved": ach, "peak": fma_peak, "unit": "TFLOP/s",
                "frac": ach / fma_peak, "traffic": traffic,
                "peak_basis": "%d SMs x %d lanes x 2 flops x %.0f MHz (of derived)"
                              % (sm_count, FP32_LANES_PER_SM, max_mhz),
                "flops_basis": "8 flops (complex multiply-add) per subset pixel-spot pair and pass",
                "kernel": "iter_subset_gather_kernel on compressed launches: the pixels of S_j only (%d per step, "
                          "%.1f%% of the step)" % (n_sub, share),
                "ms_per_launch": sub_ms / max(1, n_sub)}
    sfu_peak = sm_count * SFU_PER_CLK_PER_SM * max_mhz * 1e6 / 1e9           # G sin-or-cos/s
    ach = 2.0 * pairs_sub_launch * n_sub / (sub_ms * 1e-3) / 1e9 if n_sub else 0.0
    return {"bound": "alu", "pipe": "SFU sine/cosine", "achieved": ach, "peak": sfu_peak,
            "unit": "G sincos/s", "frac": ach / sfu_peak, "traffic": traffic,
            "kernel": "iter_kernel, compressed-iteration launches (%d per step, %.1f%% of the step)" % (n_sub, share),
            "peak_basis": "%d SMs x %d/clk x %.0f MHz (of derived; probe measured %.0f G/s)"
                          % (sm_count, SFU_PER_CLK_PER_SM, max_mhz, probe / 1e9),
            "ms_per_launch": sub_ms / max(1, n_sub),
            "tile": {k: tile[k] for k in ("threads", "pixels_per_thread", "blocks")}}


def launches_per_step(tile, n_sub, n_full):
    """Kernel launches of one batch step (square pupils): the per-spot
    preparation, the tensor-core constant tables (once per hologram); per
    compressed iteration on the tensor cores its R' tables, the kernel, the
    tails and the subset-mask draws (side stream), on the gather kernel the
    mask draws, the kernel and the tails, on the direct-phasor kernel one
    launch; per full pass the kernel plus, on the tensor cores, its R' tables
    and its tails."""
    ft = tile["full_threads"]
    sub = tile["threads"]
    tc = ft in TC_KERNELS or sub == SUBSET_TC
    per_sub = 4 if sub == SUBSET_TC else (3 if sub == SUBSET_GATHER else 1)
    per_full = 3 if ft in TC_KERNELS else 1
    return 1 + (1 if tc else 0) + n_sub * per_sub + n_full * per_full


def full_roofline(tile, achieved_tflops, fma_peak, sm_count, max_mhz, traffic, n_launches, full_ms):
    """Roofline of the full-iteration and final launches: the tensor-core kernel
    against the measured dense BF16 peak (its operands are BF16 halves), the
    CUDA-core kernel against the FP32 FMA peak.  Achieved = algorithmic flops:
    8 per pixel-spot pair and pass (one complex multiply-add)."""
    base = {"achieved": achieved_tflops, "unit": "TFLOP/s", "traffic": traffic,
            "flops_basis": "8 flops (complex multiply-add) per pixel-spot pair and pass",
            "ms_per_launch": full_ms / max(1, n_launches)}
    if tile["full_threads"] in TC_KERNELS:
        peak, basis = tensor_peak()
        base.update({"bound": "tensor", "pipe": "tcgen05 kind::f16 (BF16 in, FP32 accumulate)", "peak": peak,
                     "frac": achieved_tflops / peak, "peak_basis": "%s dense BF16 peak" % basis,
                     "kernel": "%s, full-iteration and final launches (%d per step)"
                               % (TC_KERNELS[tile["full_threads"]][0], n_launches),
                     "issued_tensor_flops_per_algorithmic": 3,
                     "note": "each real product is 3 BF16 products (hi hi + hi lo + lo hi) for FP32-class "
                             "accuracy, so the tensor pipe runs 3x the algorithmic flops",
                     "tile": {"threads": TC_KERNELS[tile["full_threads"]][1], "blocks": tile["full_blocks"],
                              "pixels": "128 rows x 64 columns"}})
    else:
        base.update({"bound": "alu", "pipe": "FP32 FMA", "peak": fma_peak, "frac": achieved_tflops / fma_peak,
                     "peak_basis": "%d SMs x %d lanes x 2 flops x %.0f MHz (of derived)"
                                   % (sm_count, FP32_LANES_PER_SM, max_mhz),
                     "kernel": "iter_full_kernel, separable full-iteration and final launches (%d per step)"
                               % n_launches,
                     "tile": {"threads": tile["full_threads"], "blocks": tile["full_blocks"],
                              "pixels": "threads/4 rows x 64 columns, 4 x 4 per thread"}})
    return base


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--P", type=int, default=1152)
    ap.add_argument("--N", type=int, default=100)
    ap.add_argument("--c", type=float, default=0.125)
    ap.add_argument("--iters", type=int, default=30)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--tune-cache", default=None, help="autotuner JSON cache (read, and written when tuning)")
    ap.add_argument("--serve-rates", default="60,240",
                    help="Poisson arrival rates (req/s) of the mixed serving streams")
    ap.add_argument("--serve-seconds", type=float, default=60.0, help="length of each mixed arrival stream")
    ap.add_argument("--serve-headline-rate", type=float, default=1000.0,
                    help="arrival rate of the extra stream of the batch workload's holograms (3 s)")
    ap.add_argument("--no-sweep", action="store_true", help="skip the compressed-iteration sweep (N x c)")
    ap.add_argument("--no-grid100", action="store_true", help="skip the headline shape on rotated 10 x 10 grids")
    ap.add_argument("--no-sfu-leg", action="store_true",
                    help="skip the CUDA-core compressed-iteration kernel timed at the workload")
    ap.add_argument("--quick", action="store_true",
                    help="short serving streams (5 s) and no oracle comparisons of the sweep")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-fp16", action="store_true")
    ap.add_argument("--no-scenarios", action="store_true")
    ap.add_argument("--compare", action="store_true",
                    help="the paper's computational comparison instead of the throughput run: RS, WGS and CS-WGS "
                         "(c = 2^-1 .. 2^-8) on its scenarios, quality against single-hologram latency and at "
                         "fixed time budgets")
    ap.add_argument("--no-paper-setup", action="store_true",
                    help="skip the leg with the paper's optics (round aperture, Gaussian beam, windows, SLM frames)")
    return ap.parse_args()


def problems(args, rank):
    """This rank's share of the job: its own batch of holograms (seeds never shared
    between ranks), so the work scales with the number of GPUs (weak scaling)."""
    return [workloads.problem(args.P, args.N, 10.0, args.c, args.iters, seed=rank * 100000 + h)
            for h in range(args.batch)]


def max_over_ranks(x, world, device):
    """The largest value of x over all ranks (the job's time is its slowest rank's)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(per_rank_holograms, world, steps, slowest_ms):
    """Whole-job holograms/s: every rank's holograms over the slowest rank's time."""
    return per_rank_holograms * world * steps / (slowest_ms * 1e-3)


def workload_config(args, extra=None):
    cfg = {"workload": "CS-WGS batch of %d point-cloud holograms, P=%d (M=%d), N=%d, c=%g, %d iterations "
                       "(%d compressed + 2 full) + final pass" % (args.batch, args.P, args.P * args.P, args.N,
                                                                args.c, args.iters, args.iters - 2),
           "P": args.P, "M": args.P * args.P, "N": args.N, "subset_fraction": args.c,
           "iterations": args.iters, "full_iterations": 2, "batch": args.batch,
           "spots": "alpha,beta~U[-P/4,P/4] cycles, gamma~U[-10,10] waves, a=1, theta0~U[0,2pi)"}
    if extra:
        cfg.update(extra)
    return cfg


def pairs_per_hologram(args):
    Mp = math.floor(args.c * args.P * args.P)
    M = args.P * args.P
    F = min(2, args.iters)
    return args.N * (2 * (args.iters - F) * Mp + 2 * F * M + 2 * M)


# ---------------------------------------------------------------- clocks --
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = [r.split(",") for r in out.strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------- serving --
def serve_probe(args, local, rate, seconds, mix):
    """Continuous batching under a Poisson arrival stream: requests are submitted
    at their arrival times (cswgs_submit) and collected as they finish
    (cswgs_wait); returns throughput and submit-to-result latency.  mix: the
    serving workload's mixed requests (P in {768, 1024, 1152}, N uniform on
    {10, 100, 1000}, i.e. log-uniform on that grid, gamma ~ U[-20, 20], c = 1/8,
    20 iterations); else the batch workload's holograms."""
    import queue
    import threading

    import torch

    from paper_2003_05293_gb300 import Plan

    if mix:
        stream = workloads.arrivals(rate, seconds, seed=7)
        what = ("mixed: P in {768,1024,1152}, N uniform on {10,100,1000} (log-uniform on that grid), "
                "gamma~U[-20,20], c=1/8, 20 iterations")
    else:
        rng = np.random.Generator(np.random.PCG64(7))
        t, stream = 0.0, []
        while True:
            t += float(rng.exponential(1.0 / rate))
            if t >= seconds:
                break
            stream.append((t, workloads.problem(args.P, args.N, 10.0, args.c, args.iters, seed=10**6 + len(stream))))
        what = "P=%d, N=%d, c=%g, %d iterations (the batch workload's holograms)" % (args.P, args.N, args.c, args.iters)
    maxP = max(pb.P for _, pb in stream)
    nbuf = 192
    bufs = [torch.empty(maxP * maxP, dtype=torch.float32, device="cuda") for _ in range(nbuf)]
    free = queue.Queue()
    for i in range(nbuf):
        free.put(i)
    plan = Plan(device=local, precision="fp32", max_batch=64, max_N=1024, max_P=max(2048, maxP))
    # warm the serving path (tuning, kernel loading) with a few requests
    for pb in [stream[i][1] for i in range(min(4, len(stream)))]:
        plan.wait(plan.submit(pb, bufs[0][:pb.M]), 120.0)
    results, tickets = [], queue.Queue()

    def collect():
        while True:
            item = tickets.get()
            if item is None:
                return
            tk, b = item
            results.append(plan.wait(tk, 600.0))
            free.put(b)

    th = threading.Thread(target=collect)
    th.start()
    t0 = time.perf_counter()
    for at, pb in stream:
        delay = at - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(delay)
        b = free.get()
        tickets.put((plan.submit(pb, bufs[b][:pb.M]), b))
    tickets.put(None)
    th.join()
    wall = time.perf_counter() - t0
    st = plan.serve_stats()
    plan.close()
    lat = [r["latency_ms"] for r in results if r["status"] == 0]
    qms = [r["queue_ms"] for r in results if r["status"] == 0]
    return {"what": what, "rate_hz": rate, "seconds": seconds, "requests": len(stream),
            "completed": len(lat), "holograms_per_s": len(lat) / wall,
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "max": float(np.max(lat))},
            "queue_ms": {"p50": float(np.percentile(qms, 50)), "p99": float(np.percentile(qms, 99))},
            "launches": st["launches"], "device_busy_s": st["busy_ms"] / 1e3,
            "api": "cswgs_submit / cswgs_wait, continuous batching, device outputs"}


# -------------------------------------------------------- reference arm --
def run_reference(args, rank, world):
    """The FP64 CPU oracle on the host cores, one hologram of the workload per step."""
    if rank != 0:
        return
    import oracle
    pbs = problems(args, 0)
    cores = oracle.threads()
    times = []
    for s in range(args.warmup + args.steps):
        pb = pbs[s % len(pbs)]
        t0 = time.perf_counter()
        oracle.solve(pb.P, pb.xyz, c=pb.c, iterations=pb.iterations, seed=pb.seed)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = len(times) / total
    sample = "one hologram of the workload per step (P=%d, N=%d, c=%g, %d iterations), FP64" % (
        args.P, args.N, args.c, args.iters)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "holograms/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args, {"batch": 1}),
            "cpu_baseline": {"value": value, "unit": "holograms/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "holograms/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# -------------------------------------------------------------- our arm --
def run_compare(args, local):
    """Section 5's comparison, on synthetic stand-ins of its scenarios with its
    optics: random superposition (I = 0), WGS (c = 1) and CS-WGS (c = 2^-1 ..
    2^-8, the last two iterations full), each at several iteration counts.  Per
    configuration: the device time of one hologram alone (CUDA events on the
    plan's stream, median of 3) and e, u over 10 orientations and initial
    phases.  Then, per time budget, the best e * u each method reaches within
    it."""
    import torch

    from paper_2003_05293_gb300 import Plan
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    plan = Plan(device=local, precision="fp32", stream=stream.cuda_stream, tune_cache=args.tune_cache)
    P = args.P
    waist = 6000.0 / 9.2 * P / 1152
    pupil = dict(aperture="round", waist=waist, subset_mode="windows")
    out = torch.empty(P * P, dtype=torch.float32, device="cuda")
    methods = [("RS", 1.0, [0])] + [("WGS", 1.0, [1, 2, 3, 5, 8, 12, 20, 30, 50])]
    methods += [("CS-WGS", 2.0 ** -k, [3, 5, 8, 12, 20, 30, 50]) for k in range(1, 9)]
    budgets_ms = [0.25, 0.5, 1.0, 2.0, 4.0]
    result = {}
    for name in workloads.SCENARIOS:
        rows = []
        for meth, c, iters in methods:
            for I in iters:
                pbs = [workloads.scenario(name, P, seed=s, c=c, iterations=I) for s in range(10)]
                for q in pbs:
                    q.extra.update(pupil)
                    q.extra["full_iterations"] = I if meth == "WGS" else min(2, I)
                q = pbs[0]
                kw = dict(full_iterations=q.extra["full_iterations"], **pupil)
                plan.solve(q.xyz, P, c, I, q.seed, out=out, **kw)           # warm-up (graph, tuning)
                ts = []
                for _ in range(3):
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    plan.solve(q.xyz, P, c, I, q.seed, out=out, **kw)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    ts.append(e0.elapsed_time(e1))
                res = plan.solve_batch(pbs)
                es = np.array([r["e"] for r in res])
                us = np.array([r["u"] for r in res])
                rows.append({"method": meth, "c": c, "iterations": I, "ms": float(np.median(ts)),
                             "e": float(es.mean()), "u": float(us.mean()), "u_min": float(us.min())})
        best = {}
        for b in budgets_ms:
            best[str(b)] = {}
            for meth in ("RS", "WGS", "CS-WGS"):
                fit = [r for r in rows if r["method"] == meth and r["ms"] <= b]
                if fit:
                    r = max(fit, key=lambda r: r["e"] * r["u"])
                    best[str(b)][meth] = {k: r[k] for k in ("c", "iterations", "ms", "e", "u")}
        result[name] = {"N": int(workloads.scenario(name, P, 0).N), "runs": rows, "best_within_budget_ms": best}
    plan.close()
    print(json.dumps({"metric": "hologram quality at a fixed single-hologram time budget", "P": P,
                      "pupil": "round aperture of P px, Gaussian beam waist %.1f px, windows" % waist,
                      "timing": "device time of one hologram alone (CUDA events), median of 3",
                      "quality": "mean e, u over 10 orientations and initial phases", "scenarios": result}),
          flush=True)


def timed_batch(plan, pbs, outs, flush, stream, steps, warmup, world):
    """Device time (ms, max over ranks) of `steps` graph replays of a batch, an
    L2 flush before each (CUDA events on the plan's stream); the results, the
    per-launch times of the last run and the launch shapes."""
    import torch
    b = plan.batch(pbs, outs)
    for _ in range(warmup):
        flush.fill_(1)
        b.run()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        flush.fill_(1)
        b.run()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1), world, "cuda")
    res, kt, tile = b.results(), b.kernel_times(), b.tile_shape()
    b.close()
    return ms, res, kt, tile


def fp64_latency(p64, pbs, stream):
    """The plain FP64 solver, one hologram at a time: device time of each solve
    (CUDA events on the plan's stream), holograms/s and p50/p99."""
    import torch
    o = torch.empty(max(pb.M for pb in pbs), dtype=torch.float32, device="cuda")
    pb = pbs[0]
    p64.solve(pb.xyz, pb.P, pb.c, 2, pb.seed, out=o[:pb.M])      # warm-up
    torch.cuda.synchronize()
    ts = []
    for pb in pbs:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        p64.solve(pb.xyz, pb.P, pb.c, pb.iterations, pb.seed, out=o[:pb.M])
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return {"value": 1e3 * len(ts) / sum(ts), "unit": "holograms/s", "holograms": len(ts),
            "latency_ms": {"p50": float(np.percentile(ts, 50)), "p99": float(np.percentile(ts, 99)),
                           "all": [round(t, 2) for t in ts]},
            "what": "plain double-precision kernels, one hologram per solve (device time of each)"}


def parity_entry(phase, res, ref, which):
    d = (np.asarray(phase, dtype=np.float64) - ref["phase"] + np.pi) % (2 * np.pi) - np.pi
    return {"hologram": which, "phase_rms_rad": float(np.sqrt(np.mean(d * d))),
            "abs_de": abs(res["e"] - ref["e"]), "abs_du": abs(res["u"] - ref["u"]),
            "tolerance": {"phase_rms_rad": 1e-3, "abs_de": 1e-3, "abs_du": 1e-3}}


def e2e_leg(args, plan, pbs, world, B):
    """End to end through the C ABI's host-buffer batches: every step copies its
    hologram requests' spots (host) in and its phase maps and e, u (host) out.
    Two batches alternate (update and run one, collect the other), so one
    batch's map copies overlap the other's computation.  Timed with the host
    clock over K steps, inputs staged and outputs written inside the region."""
    import torch

    def run(make_out):
        outs = [[make_out(pb) for pb in pbs] for _ in range(2)]
        hb = [plan.host_batch(pbs, outs[0]), plan.host_batch(pbs, outs[1])]
        steps = [[workloads.Problem(P=pb.P, xyz=pb.xyz, amp=pb.amp, c=pb.c, iterations=pb.iterations,
                                    seed=pb.seed + 7919 * k) for pb in pbs] for k in range(args.e2e_steps)]
        for b in hb:                      # warm-up: graph capture, first copies
            b.run()
        for b in hb:
            b.results()
        torch.cuda.synchronize()
        max_over_ranks(0.0, world, "cuda")
        t0 = time.perf_counter()
        for k in range(args.e2e_steps):
            b = hb[k % 2]
            if k >= 2:
                b.results()
            b.update(steps[k], outs[k % 2])
            b.run()
        for k in range(max(0, args.e2e_steps - 2), args.e2e_steps):
            hb[k % 2].results()
        dt = max_over_ranks(time.perf_counter() - t0, world, "cuda")
        for b in hb:
            b.close()
        return B * world * args.e2e_steps / dt
    v_pageable = run(lambda pb: np.empty(pb.M, dtype=np.float32))
    v_pinned = run(lambda pb: torch.empty(pb.M, dtype=torch.float32, pin_memory=True).numpy())
    return {"value": max(v_pageable, v_pinned), "unit": "holograms/s",
            "h2d_bytes_per_step": int(sum(pb.N * 3 * 8 for pb in pbs)),
            "d2h_bytes_per_step": int(sum(pb.M * 4 + 16 for pb in pbs)),
            "api": "cswgs_batch_create_host / cswgs_batch_update / cswgs_batch_run / cswgs_batch_results: host "
                   "spot arrays in (staged through pinned memory), host phase maps (pinned: copy engines; pageable: "
                   "the copy kernel) and e, u out; two batches alternate so that one's copies overlap the other's "
                   "computation",
            "steps": args.e2e_steps, "pageable_host_outputs": v_pageable, "pinned_host_outputs": v_pinned}


def sfu_leg(args, pbs, flush, stream, world, local, sm_count, max_mhz, probe):
    """The batch with its compressed iterations pinned to the CUDA-core kernel
    (256 threads x 4 pixels: the pixels of S_j only, each phasor a fixed-point
    argument and two SFU results), full passes as tuned: compressed ms per
    launch and the SFU fraction (2 sine-or-cosine results per subset pixel-spot
    pair and pass)."""
    import tempfile

    import torch

    from paper_2003_05293_gb300 import Plan
    B = len(pbs)
    entries = {"P%d_N%d_B%d_c%d" % (128 * p, 2 ** n, 2 ** b, c): [256, 4, 2]
               for p in range(1, 17) for n in range(4, 13) for b in range(0, 8) for c in range(0, 17)}
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "tune_sfu.json")
        with open(path, "w") as f:
            json.dump({"format": "cswgs-tune-3", "entries": entries}, f)
        with Plan(device=local, precision="fp32", max_batch=max(64, B), max_N=max(1024, args.N),
                  stream=stream.cuda_stream, tune_cache=path) as plan:
            outs = [torch.empty(pb.M, dtype=torch.float32, device="cuda") for pb in pbs]
            steps = max(3, args.steps // 2)
            ms, res, kt, tile = timed_batch(plan, pbs, outs, flush, stream, steps, args.warmup, world)
    n_sub = args.iters - min(2, args.iters)
    sub_ms = sum(kt[1:1 + n_sub]) / max(1, n_sub)
    Mp = math.floor(args.c * args.P * args.P)
    pairs = B * 2.0 * args.N * Mp
    sfu_peak = sm_count * SFU_PER_CLK_PER_SM * max_mhz * 1e6
    ach = 2.0 * pairs / (sub_ms * 1e-3)
    return {"value": job_throughput(B, world, steps, ms), "unit": "holograms/s", "compressed_ms_per_launch": sub_ms,
            "kernel": kernel_name(tile, "sub"),
            "sfu_roofline": {"bound": "alu", "pipe": "SFU sine/cosine", "achieved": ach / 1e9, "peak": sfu_peak / 1e9,
                             "unit": "G sincos/s", "frac": ach / sfu_peak,
                             "peak_basis": "%d SMs x %d/clk x %.0f MHz (probe measured %.0f G/s)"
                                           % (sm_count, SFU_PER_CLK_PER_SM, max_mhz, probe / 1e9)},
            "what": "compressed iterations on the CUDA cores (the subset's pixels only), full passes on the tensor cores"}


def sweep_leg(args, plan, flush, stream, world, B, rank, local):
    """The precision workload's compressed-iteration sweep at P = args.P: N in
    {100, 300} x c in {1/4, 1/8, 1/16}, a batch of B holograms each (the
    autotuner picks the kernels per c), with per-launch times; the FP64 GPU
    solver at the same shape.  Returns the entries and, per (N, c), the first
    hologram's problem, map and result for the oracle comparison."""
    import torch

    import tempfile

    from paper_2003_05293_gb300 import Plan
    runs, keep = [], {}
    n_sub = args.iters - min(2, args.iters)
    # a plan with the compressed iterations pinned to the subset-only gather kernel
    tmp = tempfile.TemporaryDirectory()
    gpath = os.path.join(tmp.name, "tune_gather.json")
    with open(gpath, "w") as f:
        json.dump({"format": "cswgs-tune-3",
                   "entries": {"P%d_N%d_B%d_c%d" % (128 * p, 2 ** n, 2 ** b, c): [SUBSET_GATHER, 1, 2]
                               for p in range(1, 17) for n in range(4, 13) for b in range(0, 8) for c in range(17)}},
                  f)
    gplan = Plan(device=local, precision="fp32", max_batch=max(64, B), max_N=1024, stream=stream.cuda_stream,
                 tune_cache=gpath)
    with Plan(device=local, precision="fp64", stream=stream.cuda_stream) as p64:
        for N in workloads.LARGE_N:
            for c in workloads.LARGE_C:
                pbs = [workloads.problem(args.P, N, 10.0, c, args.iters, seed=rank * 100000 + 50000 + h)
                       for h in range(B)]
                outs = [torch.empty(pb.M, dtype=torch.float32, device="cuda") for pb in pbs]
                ms, res, kt, tile = timed_batch(plan, pbs, outs, flush, stream, max(3, args.steps // 2),
                                                args.warmup, world)
                steps = max(3, args.steps // 2)
                sub_ms = sum(kt[1:1 + n_sub]) / max(1, n_sub)
                full_ms = sum(kt[1 + n_sub:]) / max(1, len(kt) - 1 - n_sub)
                Mp = math.floor(c * args.P * args.P)
                pairs = B * 2.0 * N * Mp
                entry = {"N": N, "c": c, "value": job_throughput(B, world, steps, ms), "unit": "holograms/s",
                         "ms_per_step": ms / steps, "compressed_ms_per_launch": sub_ms,
                         "full_ms_per_launch": full_ms,
                         "compressed_kernel": kernel_name(tile, "sub"),
                         "compressed_method_tflops": 8.0 * pairs / (sub_ms * 1e-3) / 1e12,
                         "e_mean": float(np.mean([r["e"] for r in res])),
                         "u_mean": float(np.mean([r["u"] for r in res])), "tile": tile}
                keep[(N, c)] = (pbs[0], outs[0].cpu().numpy(), res[0])
                if N <= 192:
                    gms, gres, gkt, gtile = timed_batch(gplan, pbs, outs, flush, stream, 3, args.warmup, world)
                    entry["gather_compressed_ms_per_launch"] = sum(gkt[1:1 + n_sub]) / max(1, n_sub)
                    entry["gather_value"] = job_throughput(B, world, 3, gms)
                    entry["gather_kernel"] = kernel_name(gtile, "sub")
                entry["fp64_gpu"] = fp64_latency(p64, pbs[:3 if N * c > 50 else 5], stream)
                runs.append(entry)
                del outs
    # the serving workload's smallest clouds: the tensor-core kernel pads the
    # spots to a 128-spot block, the gather kernel to a multiple of 32
    small = []
    for N in (10,):
        for c in workloads.LARGE_C:
            pbs = [workloads.problem(args.P, N, 10.0, c, args.iters, seed=rank * 100000 + 70000 + h) for h in range(B)]
            outs = [torch.empty(pb.M, dtype=torch.float32, device="cuda") for pb in pbs]
            ms, res, kt, tile = timed_batch(plan, pbs, outs, flush, stream, 3, args.warmup, world)
            gms, gres, gkt, gtile = timed_batch(gplan, pbs, outs, flush, stream, 3, args.warmup, world)
            small.append({"N": N, "c": c, "value": job_throughput(B, world, 3, ms),
                          "compressed_ms_per_launch": sum(kt[1:1 + n_sub]) / max(1, n_sub),
                          "compressed_kernel": kernel_name(tile, "sub"),
                          "gather_compressed_ms_per_launch": sum(gkt[1:1 + n_sub]) / max(1, n_sub),
                          "gather_value": job_throughput(B, world, 3, gms),
                          "e_mean": float(np.mean([r["e"] for r in res])),
                          "gather_e_mean": float(np.mean([r["e"] for r in gres]))})
            del outs
    gplan.close()
    tmp.cleanup()
    return {"P": args.P, "batch": B, "iterations": args.iters,
            "what": "compressed-iteration sweep of the precision workload: a batch per (N, c), FP32 path as tuned; "
                    "compressed_method_tflops counts 8 flops per subset pixel-spot pair and pass",
            "runs": runs, "small_n": small}, keep


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.compare:
        if rank == 0:
            run_compare(args, local)
        return

    import torch
    import torch.distributed as dist

    from paper_2003_05293_gb300 import Plan

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    pbs = problems(args, rank)
    B = len(pbs)
    # one non-default stream for everything: the plan's kernels, the L2 flush
    # and the timing events (the legacy default stream has handle 0, which
    # would make the plan create a stream of its own)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    plan = Plan(device=local, precision="fp32", max_batch=max(64, B), max_N=max(1024, args.N),
                stream=stream.cuda_stream, tune_cache=args.tune_cache)
    outs = [torch.empty(pb.M, dtype=torch.float32, device="cuda") for pb in pbs]
    batch = plan.batch(pbs, outs)
    total_pairs, iter_pairs = batch.pairs()
    tile = batch.tile_shape()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")   # > L2 (129 MB)

    for _ in range(args.warmup):          # the same work as a timed step (loads every kernel)
        flush.fill_(1)
        batch.run()
        batch.results()

    # timed region: K steps queued back to back on one stream (an L2 flush
    # before each), a CUDA event after each; one synchronisation at the end
    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    step_ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev0.record(stream)
    for k in range(args.steps):
        flush.fill_(1)                       # evict L2 between steps
        batch.run()                          # graph launch on the same stream
        step_ev[k].record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    total_ms = max_over_ranks(ev0.elapsed_time(step_ev[-1]), world, "cuda")
    value = job_throughput(B, world, args.steps, total_ms)
    res = batch.results()
    # per-step device time (flush + graph) from consecutive events
    step_ms = [ev0.elapsed_time(step_ev[0])] + [step_ev[k - 1].elapsed_time(step_ev[k])
                                                 for k in range(1, args.steps)]
    # per-launch device times of the last timed step (events inside the graph)
    kts = [batch.kernel_times()]

    # rooflines of the iteration kernels, per launch kind (measured live, CUDA
    # events recorded inside the graph around every launch of the last timed
    # step): on the tensor cores algorithmic flops (8 per pixel-spot pair and
    # pass) against the measured dense BF16 peak; on the CUDA cores 2 SFU
    # results per pair and pass (compressed launches) against the SFU peak, or
    # 8 flops per pair and pass (separable full passes) against the FP32 peak.
    props = torch.cuda.get_device_properties(local)
    sm_count = props.multi_processor_count
    max_mhz = 2070.0
    try:
        mp = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        max_mhz = float(mp.get("sm_max_mhz", max_mhz))
    except (OSError, ValueError):
        pass
    n_sub = args.iters - min(2, args.iters)
    Mp = math.floor(args.c * args.P * args.P)
    pairs_sub_launch = B * 2.0 * args.N * Mp
    pairs_full_launch = B * 2.0 * args.N * args.P * args.P
    sub_ms = sum(sum(k[1:1 + n_sub]) for k in kts) / len(kts)
    full_ms = sum(sum(k[1 + n_sub:]) for k in kts) / len(kts)
    n_full_launches = len(kts[0]) - 1 - n_sub
    fma_peak = sm_count * FP32_LANES_PER_SM * 2 * max_mhz * 1e6 / 1e12       # TFLOP/s
    fma_achieved = 8.0 * pairs_full_launch * n_full_launches / (full_ms * 1e-3) / 1e12
    probe, probe_mhz = plan.sincos_peak()
    TRAFFIC_SUB, TRAFFIC_FULL = measured_traffic(args, tile)

    eu = [(r["e"], r["u"]) for r in res]
    line = {"metric": METRIC, "value": value, "unit": "holograms/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": dtype_label(tile), "data": "synthetic",
            "config": workload_config(args, {"l2": "flushed between steps (256 MB write), inside the timed region",
                                             "parallelism": "replicas" if world > 1 else "single GPU"}),
            "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99)),
                           "steps": [round(x, 3) for x in step_ms],
                           "what": "device time of one batch step (L2 flush + whole hot path for every hologram "
                                   "of the batch): a hologram submitted with its batch is done after it"},
            "quality": {"e_mean": float(np.mean([a for a, _ in eu])), "u_mean": float(np.mean([b for _, b in eu])),
                        "u_min": float(np.min([b for _, b in eu])), "e_min": float(np.min([a for a, _ in eu]))},
            "roofline": subset_roofline(tile, pairs_sub_launch, n_sub, sub_ms, full_ms, sm_count, max_mhz, probe,
                                        TRAFFIC_SUB, args),
            "roofline_full_passes": full_roofline(tile, fma_achieved, fma_peak, sm_count, max_mhz, TRAFFIC_FULL,
                                                  n_full_launches, full_ms),
            "gpu_launches": args.steps * launches_per_step(tile, n_sub, n_full_launches),
            "kernel_times_from": "CUDA events recorded inside the graph around each launch, last timed step",
            "clocks": clk}

    # the half-precision sincos option for the compressed iterations
    if not args.no_fp16:
        p16 = Plan(device=local, precision="fp32_fp16sincos", max_batch=max(64, B), max_N=max(1024, args.N),
                   stream=stream.cuda_stream)
        outs16 = [torch.empty(pb.M, dtype=torch.float32, device="cuda") for pb in pbs]
        b16 = p16.batch(pbs, outs16)
        for _ in range(args.warmup):
            flush.fill_(1)
            b16.run()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            flush.fill_(1)
            b16.run()
        e1.record(stream)
        torch.cuda.synchronize()
        ms16 = max_over_ranks(e0.elapsed_time(e1), world, "cuda")
        r16 = b16.results()
        kt16 = b16.kernel_times()
        d_e = max(abs(a["e"] - b["e"]) for a, b in zip(r16, res))
        d_u = max(abs(a["u"] - b["u"]) for a, b in zip(r16, res))
        d_ph = max(float(torch.sqrt(torch.mean((torch.remainder(o16 - o + math.pi, 2 * math.pi) - math.pi) ** 2)))
                   for o16, o in zip(outs16, outs))
        t16 = b16.tile_shape()
        what16 = ("compressed iterations on the tensor cores with FP16 forward-projection products (FP32 "
                  "accumulation); full iterations and the final pass FP32-class" if t16["threads"] == SUBSET_TC else
                  "compressed iterations with half-precision sincos (packed FP16 on the FMA pipe); full "
                  "iterations and the final pass FP32")
        line["fp16_sincos"] = {"value": job_throughput(B, world, args.steps, ms16), "unit": "holograms/s",
                               "ms_per_step": ms16 / args.steps,
                               "compressed_ms_per_launch": sum(kt16[1:1 + n_sub]) / max(1, n_sub),
                               "vs_fp32": {"max_abs_de": d_e, "max_abs_du": d_u, "max_phase_rms_rad": d_ph},
                               "tile": t16, "what": what16}
        b16.close()
        p16.close()

    # the CUDA-core compressed-iteration kernel (direct phasors on the SFU, the
    # pixels of S_j only) at the same workload, pinned through a tune cache:
    # its time per launch and its fraction of the SFU's sine/cosine peak, beside
    # the tensor-core kernel the autotuner picks
    if not args.no_sfu_leg:
        line["cuda_core_compressed"] = sfu_leg(args, pbs, flush, stream, world, local, sm_count, max_mhz, probe)

    # FP64 GPU baseline (plain double-precision kernels), one hologram at a time:
    # per-hologram device time (CUDA events on the plan's stream)
    if not args.no_fp64:
        with Plan(device=local, precision="fp64", stream=stream.cuda_stream) as p64:
            fp = fp64_latency(p64, pbs[:6], stream)
        fp["speedup_fp32_batched"] = value / fp["value"] / world
        line["fp64_gpu_baseline"] = fp

    # end to end through the C ABI: host inputs in, host phase maps and e, u out
    if not args.no_e2e:
        line["e2e"] = e2e_leg(args, plan, pbs, world, B)

    # the headline shape on the paper's regular pattern (a rotated 10 x 10 grid,
    # one orientation and initial phase per hologram), where e, u >= 0.9 hold
    if not args.no_grid100:
        gpbs = [workloads.scenario("grid100", args.P, seed=rank * 100000 + h, c=args.c, iterations=args.iters)
                for h in range(B)]
        gouts = [torch.empty(pb.M, dtype=torch.float32, device="cuda") for pb in gpbs]
        gms, gres, gkt, _ = timed_batch(plan, gpbs, gouts, flush, stream, args.steps, args.warmup, world)
        line["headline_grid100"] = {
            "value": job_throughput(B, world, args.steps, gms), "unit": "holograms/s", "ms_per_step": gms / args.steps,
            "e_mean": float(np.mean([r["e"] for r in gres])), "e_min": float(np.min([r["e"] for r in gres])),
            "u_mean": float(np.mean([r["u"] for r in gres])), "u_min": float(np.min([r["u"] for r in gres])),
            "what": "the headline batch shape (%d holograms, P=%d, N=100, c=%g, %d iterations) on rotated 10 x 10 "
                    "spot grids (one orientation and initial phase per hologram)" % (B, args.P, args.c, args.iters)}
        del gouts

    # the compressed-iteration sweep of the precision workload: N in {100, 300}
    # x c in {1/4, 1/8, 1/16} at P = 1152, a batch each, the FP64 GPU solver
    # at the same shape; the first hologram of each is compared with the oracle
    # in the CPU leg below
    sweep_keep = {}
    if not args.no_sweep:
        line["compressed_sweep"], sweep_keep = sweep_leg(args, plan, flush, stream, world, B, rank, local)

    # the paper's scenarios (Section 5): 10 orientations and initial phases of
    # each, as one batch through the same path
    if not args.no_scenarios:
        qual = {}
        for name in workloads.SCENARIOS:
            spb = [workloads.scenario(name, args.P, seed=s, c=args.c, iterations=args.iters) for s in range(10)]
            r = plan.solve_batch(spb)
            es = np.array([x["e"] for x in r])
            us = np.array([x["u"] for x in r])
            qual[name] = {"N": spb[0].N, "e_mean": float(es.mean()), "e_std": float(es.std()),
                          "u_mean": float(us.mean()), "u_std": float(us.std()),
                          "e_min": float(es.min()), "u_min": float(us.min())}
        line["quality_paper_scenarios"] = qual

    # the paper's own optics and output (Section 4: round aperture P pixels
    # across, 6 mm beam waist on 9.2 um pixels; Section 3: one random
    # reordering of the pupil, gray frames of a 1920 x 1152 panel)
    if not args.no_paper_setup:
        from paper_2003_05293_gb300 import SlmFrame
        waist = 6000.0 / 9.2 * args.P / 1152
        lut = torch.arange(256, dtype=torch.int32, device="cuda").to(torch.uint8)
        W, Hh = max(1920, args.P), max(1152, args.P)
        frames = [torch.zeros((Hh, W), dtype=torch.uint8, device="cuda") for _ in pbs]
        ppbs = []
        for pb, fr in zip(pbs, frames):
            q = workloads.Problem(P=pb.P, xyz=pb.xyz, amp=pb.amp, c=pb.c, iterations=pb.iterations, seed=pb.seed,
                                  extra=dict(aperture="round", waist=waist, subset_mode="windows",
                                             slm=SlmFrame(fr, lut, offset_x=(W - pb.P) // 2, offset_y=(Hh - pb.P) // 2)))
            ppbs.append(q)
        bp = plan.batch(ppbs, None)
        for _ in range(args.warmup):
            flush.fill_(1)
            bp.run()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            flush.fill_(1)
            bp.run()
        e1.record(stream)
        torch.cuda.synchronize()
        msp = max_over_ranks(e0.elapsed_time(e1), world, "cuda")
        rp = bp.results()
        ktp = bp.kernel_times()
        bp.close()
        sq = {}
        if not args.no_scenarios:
            for name in workloads.SCENARIOS:
                spb = [workloads.scenario(name, args.P, seed=s, c=args.c, iterations=args.iters) for s in range(10)]
                for q in spb:
                    q.extra.update(aperture="round", waist=waist, subset_mode="windows")
                r = plan.solve_batch(spb)
                es = np.array([x["e"] for x in r])
                us = np.array([x["u"] for x in r])
                sq[name] = {"e_mean": float(es.mean()), "u_mean": float(us.mean()), "u_min": float(us.min())}
        line["paper_setup"] = {
            "value": job_throughput(B, world, args.steps, msp), "unit": "holograms/s", "ms_per_step": msp / args.steps,
            "compressed_ms_per_launch": sum(ktp[1:1 + n_sub]) / max(1, n_sub),
            "full_ms_per_launch": sum(ktp[1 + n_sub:]) / max(1, len(ktp) - 1 - n_sub),
            "e_mean": float(np.mean([x["e"] for x in rp])), "u_mean": float(np.mean([x["u"] for x in rp])),
            "u_min": float(np.min([x["u"] for x in rp])), "scenarios": sq,
            "what": "the same batch with a round aperture of P pixels, Gaussian beam of %.1f px waist, subsets as "
                    "windows of one random order, and each hologram also written as an 8-bit gray frame (256-level "
                    "table) into its own %d x %d panel buffer" % (waist, W, Hh)}
        del frames

    # continuous-batching server under Poisson arrival streams: the serving
    # workload's mixed requests at each rate, and an extra stream of the batch
    # workload's holograms
    if not args.no_serve:
        secs = 5.0 if args.quick else args.serve_seconds
        runs = [serve_probe(args, local, float(r), secs, True) for r in args.serve_rates.split(",") if r]
        runs.append(serve_probe(args, local, args.serve_headline_rate, 3.0, False))
        line["serve"] = runs

    # the FP64 CPU oracle on a bounded sample (rank 0, single GPU runs only)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        pb = pbs[0]
        t0 = time.perf_counter()
        ref = oracle.solve(pb.P, pb.xyz, c=pb.c, iterations=pb.iterations, seed=pb.seed)
        dt = time.perf_counter() - t0
        # the same hologram from the timed batch against the oracle (wrapped phase
        # RMS over the map, e and u)
        line["parity_vs_oracle"] = parity_entry(outs[0].cpu().numpy(), res[0], ref,
                                                "the batch's first (P=%d, N=%d)" % (pb.P, pb.N))
        line["cpu_baseline"] = {"value": 1.0 / dt, "unit": "holograms/s", "cores": oracle.threads(),
                                "kind": "oracle",
                                "sample": "1 hologram of the workload (P=%d, N=%d, c=%g, %d iterations), FP64 C "
                                          "with OpenMP, %.1f s" % (pb.P, pb.N, pb.c, pb.iterations, dt)}
        if not args.quick:
            for entry in line.get("compressed_sweep", {}).get("runs", []):
                q, ph, r = sweep_keep[(entry["N"], entry["c"])]
                ref = oracle.solve(q.P, q.xyz, c=q.c, iterations=q.iterations, seed=q.seed)
                entry["parity_vs_oracle"] = parity_entry(ph, r, ref, "the batch's first")
    batch.close()
    plan.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
