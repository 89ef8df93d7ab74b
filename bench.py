"""Benchmark: stratified Monte Carlo integration with heuristic tree search.

One step = one whole integration (every level of the tree: sampling kernel,
selection kernels, final reduction) of the 6-D oscillating integrand
sin(x1+...+x6) on [0,10]^6 with k=4 (4096 cells), n=2^16 points per cell and
trial, 10 trials, depth 3, sigma multiplier 1.5, in the FP32-evaluation /
FP64-accumulation mode, under the library's default budget (2^24 cells per
level, 2^40 points per run).  The metric is points evaluated per second
(Gsamples/s).  Inputs are synthetic: the integrand is a formula.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Beside the headline the line carries: the same workload in FP64 and in the
FP32-Kahan mode; the 512-integral batch; the 8-D corner peak in the three
precisions; time to a relative error of 1e-4 (9-D Gaussian); the paper's
parameter sets (Sec. 3); the kernels' arithmetic error against the oracle on
sampled level-1 tiles; and the oracle timed on the host cores.

--impl reference times the FP64 CPU oracle (the from-scratch reference of
the method) on the host cores, on a bounded sample of the same workload.
--peaks measures the pipe rates that bound the sampling kernel.
Under torchrun every rank integrates its own independent problem (seed +
rank): weak scaling, no collective on the data path.
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
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gsamples/s per GB300 (stratified MC + tree search, sin(sum x) 6-D)"
INTEGRAND_TEXT = {"sin_sum": "sin(sum x)", "gauss_norm": "normalised Gaussian",
                  "genz_corner": "Genz corner peak", "genz_gauss": "Genz Gaussian",
                  "genz_osc": "Genz oscillatory", "genz_prodpeak": "Genz product peak"}
UNIT = "Gsamples/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", default="sin6d")
    p.add_argument("--precision", default="fp32_fp64acc")
    p.add_argument("--n", type=int, default=None, help="override points per cell (small "
                   "profiling cases only; the bench line is invalid with it)")
    p.add_argument("--depth", type=int, default=None, help="override depth (profiling only)")
    p.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison leg")
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU-baseline leg")
    p.add_argument("--no-batch", action="store_true", help="skip the batched leg")
    p.add_argument("--no-tta", action="store_true", help="skip the time-to-accuracy leg")
    p.add_argument("--no-legs", action="store_true",
                   help="skip the FP32-Kahan, corner-peak and paper-parameter legs")
    p.add_argument("--paper", action="store_true",
                   help="run the paper's parameter sets (Sec. 3) instead of the benchmark")
    p.add_argument("--peaks", action="store_true",
                   help="measure the pipe rates that bound the sampling kernel (zmc_pipe_probe)")
    p.add_argument("--peaks-iters", type=int, default=None,
                   help="fixed iterations per probe kind (small profiling runs)")
    p.add_argument("--batch-compare", action="store_true",
                   help="the 512-integral batch against the same integrals run one by one")
    p.add_argument("--batch-count", type=int, default=512,
                   help="integrals in --batch-compare (smaller: profiling cases)")
    p.add_argument("--batch-level1", action="store_true",
                   help="--batch-compare with level-1-only budgets and no single runs "
                        "(a small case for ncu)")
    p.add_argument("--no-singles", action="store_true",
                   help="--batch-compare without the one-by-one runs (launch lists)")
    return p.parse_args()


def workload(args):
    from paper_1902_07916_gb300 import workloads
    w = workloads.WORKLOADS[args.workload]()
    if args.n is not None:
        w = w.with_(n=args.n)
    if args.depth is not None:
        w = w.with_(depth=args.depth)
    return w


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(world, value):
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def allreduce_sum(world, value):
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def weak_scaling_value(world, local_ms, local_samples):
    """Whole-job throughput: every rank integrated its own problem, so the
    job's points are the sum over ranks and its time the slowest rank's.
    Returns (max ms over ranks, total points, Gsamples/s)."""
    t_max = allreduce_max(world, local_ms)
    total = allreduce_sum(world, local_samples)
    return t_max, total, total / (t_max * 1e-3) / 1e9


# ------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.proc = None
        self.file = None

    def __enter__(self):
        try:
            self.file = tempfile.TemporaryFile(mode="w+")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or self.file is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        self.file.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.file:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        load = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------- our arm

def philox_multiplies_per_sample(d: int, fp64: bool) -> float:
    """Algorithmic integer work per point: per dimension and group of points
    one Philox4x32-10 block in the FP64 stream (four 32-bit words, four
    points) or a pair in the FP32 stream (eleven 23-bit fields, eleven
    points).  A block is ten rounds of two 32x32->64-bit products; of those
    twenty, the two that depend only on (trial, slot, level) are taken once
    per stream and round 1's product of the block counter is an arithmetic
    progression (additions), which leaves 17 wide multiplies per block."""
    return d * (1.0 / 4.0 if fp64 else 2.0 / 11.0) * 17


def fp32_flops_per_sample(integrand: str, d: int) -> int:
    """Counted FP32 flops per point of the FP32 modes (an FMA is 2, a multiply
    or add 1; the one hardware sine/cosine/exp2/reciprocal per point is an XU
    op, not a flop): the fold over the dimensions, the finishing function with
    its range reduction (sine and cosine in turns: a subtraction, the multiply
    by 2 pi and the hardware sine's own scaling; the Gaussians in the log2
    domain: the exponent's multiply and its offset from the lane's reference),
    and the reduction (S1 += f, S2 = fma(f, f, S2): 3)."""
    if integrand == "genz_corner":
        e = d + 1
        return 2 * d + e.bit_length() + bin(e).count("1") + 3
    per = {"constant": 3, "linear": 2 * d + 4, "sin_sum": 2 * d + 6,
           "gauss_norm": 4 * d + 5, "genz_osc": 2 * d + 7, "genz_prodpeak": 5 * d + 3,
           "genz_gauss": 4 * d + 5}
    return per[integrand]


def algorithmic_bytes_per_launch(cells_per_level, n, trials, fp64):
    """Bytes the sampling kernel must move per launch, averaged over the
    step's levels: one (S1, S2) pair of doubles written per work unit (under
    the default work plan a (cell, trial) tile is cut into `chunks` units so
    that a level has at least 2^18 of them, each of at least 1024 point
    groups of 4 points in FP64 or 11 in the FP32 modes); its reads (the
    parameters, 2.9 KB, and the parent list, 4 d bytes per flagged cell) are
    below 0.01% of that and left out."""
    group = 4 if fp64 else 11
    ngroups = -(-n // group)
    total, launches = 0, 0
    for cells in cells_per_level:
        if cells <= 0:
            continue
        tiles = cells * trials
        want = -(-(1 << 18) // tiles)
        most = max(1, ngroups // 1024)
        chunks = max(1, want) if want < most else most
        total += 16 * tiles * chunks
        launches += 1
    return total / max(launches, 1)


# DRAM bytes of the sampling kernel per launch on this benchmark's step (sin6d,
# FP32-mixed; levels 1 and 2), from one ncu capture of the metrics
# dram__bytes_read.sum and dram__bytes_write.sum, and the SHA-256 of the
# kernel's sources it was taken on (profiles/zmc_eval_reduce_sin6d_traffic.md).
TRAFFIC_CAPTURE = {
    "workload": "sin6d", "fp64": False,
    "bytes_per_launch": (420608 + 0 + 11427072 + 182042624) / 2,
    "sources_sha256": "5df126020831591c2a38cc67cd66e4362e279a1edc22ea16d0f0f70cf059c70b",
}
KERNEL_SOURCES = ["eval_kernel.cuh", "zmc_device.cuh", "zmc_layout.h"]


def kernel_sources_sha256() -> str:
    """SHA-256 of the kernel's sources with comments and blank lines removed,
    so that the capture stays valid across comment edits and no longer."""
    import hashlib
    import re
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1902_07916_gb300", "csrc", name)) as f:
            text = f.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        lines = [ln.rstrip() for ln in text.splitlines() if ln.strip()]
        h.update("\n".join(lines).encode())
    return h.hexdigest()


def traffic_per_launch(w, fp64):
    c = TRAFFIC_CAPTURE
    if w.name != c["workload"] or fp64 != c["fp64"] or kernel_sources_sha256() != c[
            "sources_sha256"]:
        return None
    return round(c["bytes_per_launch"])


# Wide (32x32->64-bit) integer multiplies per SM per clock on this GPU: the
# IMAD.WIDE issue rate (half the 64-lane IMAD rate), which bounds the
# sampling kernel; a Philox-only loop measures 1.49 blocks/clk/SM = 29.8.
WIDE_MULS_PER_SM_CLK = 32


def run_ours(args, world, rank, local):
    import torch
    from paper_1902_07916_gb300 import build as libbuild
    libbuild.build()
    from paper_1902_07916_gb300 import zmc

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    w = workload(args)
    seed = w.seed + rank
    prec = zmc.PRECISIONS[args.precision]
    it = zmc.Integrator(w.dim, w.lo, w.hi, w.k, w.n, w.trials, w.depth, w.sigma_multiplier,
                        seed, w.integrand, w.params, precision=prec)
    zmc.zmc_set_profiling(it.h, True)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 129 MB L2

    for _ in range(max(args.warmup, 0)):
        it.enqueue(stream)
    torch.cuda.synchronize(dev)

    step_ms, eval_ms, samples, results = [], [], [], []
    barrier(world)
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clocks:
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            it.enqueue(stream)
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            per_level, _ = zmc.zmc_profile(it.h, w.depth)
            eval_ms.append(sum(per_level))
            r = it.read_result(stream)
            samples.append(r.samples)
            results.append(r)
    torch.cuda.synchronize(dev)
    barrier(world)
    clk = clocks.summary()
    kernels_per_run, h2d_bytes, d2h_bytes = zmc.zmc_run_info(it.h)

    total_ms = sum(step_ms)
    t_max, all_samples, value = weak_scaling_value(world, total_ms, float(sum(samples)))

    # roofline of the dominant kernel (the sampling kernel)
    ops = sum(samples) * philox_multiplies_per_sample(w.dim, prec == zmc.ZMC_FP64)
    eval_s = sum(eval_ms) * 1e-3
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    max_mhz = clk.get("sm_max_mhz") or 2070.0
    peak = WIDE_MULS_PER_SM_CLK * sms * max_mhz * 1e6 / 1e12   # T wide multiplies / s
    achieved = ops / eval_s / 1e12

    # end to end: the public call with host result, per step
    e2e_t = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        r = it.integrate(stream)
        e2e_t.append(time.perf_counter() - t0)
    e2e_value = allreduce_sum(world, float(r.samples * len(e2e_t))) / allreduce_max(
        world, sum(e2e_t)) / 1e9

    fp64 = None
    if not args.no_fp64 and rank == 0 and prec != zmc.ZMC_FP64:
        it64 = zmc.Integrator(w.dim, w.lo, w.hi, w.k, w.n, w.trials, w.depth,
                              w.sigma_multiplier, seed, w.integrand, w.params,
                              precision=zmc.ZMC_FP64)
        # warm-up on level 1 alone (same kernel: loads it and fills the
        # launch-shape tuner's cache), then one timed run of the whole tree
        # (its graph is captured on the host before the launch, which adds
        # milliseconds at most)
        with zmc.Integrator(w.dim, w.lo, w.hi, w.k, w.n, w.trials, 1, w.sigma_multiplier,
                            seed, w.integrand, w.params, precision=zmc.ZMC_FP64) as warm:
            warm.integrate(stream)
        torch.cuda.synchronize(dev)
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        it64.enqueue(stream)
        e1.record(stream)
        r64 = it64.read_result(stream)
        ms64 = e0.elapsed_time(e1)
        it64.close()
        ref = results[-1]
        fp64 = {"value": r64.samples / (ms64 * 1e-3) / 1e9, "unit": UNIT, "steps": 1,
                "warmup": "one level-1 run", "speedup_of_headline": value / (r64.samples / (ms64 * 1e-3) / 1e9),
                "result": r64.value, "std": r64.std,
                "headline_minus_fp64_over_std": (ref.value - r64.value) / r64.std
                if r64.std > 0 else None,
                "levels_run": r64.levels_run, "flagged_per_level": r64.flagged_per_level}
    it.close()

    batched = None
    if rank == 0 and not args.no_batch:
        batched = run_batched(zmc, stream, prec)

    tta = None
    if rank == 0 and world == 1 and not args.no_tta:
        tta = run_tta(zmc, stream)

    kahan = corner = paper = None
    traces = {}
    if rank == 0 and not args.no_legs:
        from paper_1902_07916_gb300 import workloads as wl
        if prec != zmc.ZMC_FP32_KAHAN:
            kahan = run_leg(zmc, w.with_(seed=seed), "fp32_kahan", stream)
        # the 8-D corner peak (k=4, n=2^15, 16 trials, depth 5, m=1) in the
        # three precisions: compensated FP32 against FP64 accumulation
        cw = wl.corner8d()
        corner = {"workload": "corner8d: Genz corner peak (1 + a.x)^-9 on [0,1]^8, a_i ~ "
                              "U(0.5,5) from seed 0, k=4, n=2^15, trials=16, depth=5, m=1, "
                              "default budget", "legs": [run_leg(zmc, cw, p, stream)
                                                         for p in ("fp32_kahan", "fp32_fp64acc",
                                                                   "fp64")]}
        paper = paper_rows(zmc, stream)
        if world == 1 and not args.no_cpu:
            for p in dict.fromkeys([args.precision, "fp32_kahan", "fp64"]):
                traces[("head", p)] = level1_sums(zmc, w.with_(seed=seed), p, stream)
            for p in ("fp32_kahan", "fp32_fp64acc", "fp64"):
                traces[("corner", p)] = level1_sums(zmc, cw, p, stream)

    cpu = None
    mixed_error = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(w, target_s=12.0)
        if traces:
            # the kernels' arithmetic error against the oracle, per precision
            ww = w.with_(seed=seed)
            mixed_error = {"headline_workload": [error_vs_oracle(ww, p, traces[("head", p)])
                                                 for (kind, p) in traces if kind == "head"],
                           "corner8d": [error_vs_oracle(cw, p, traces[("corner", p)])
                                        for (kind, p) in traces if kind == "corner"]}

    if rank != 0:
        return None
    r = results[-1]
    try:
        exact = exact_value(w)
    except ValueError:
        exact = None
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(t_max / max(args.steps, 1), 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 eval / f64 accum" if prec == zmc.ZMC_FP32_FP64ACC else args.precision,
        "data": "synthetic (analytic integrand, Philox counter-based points)",
        "config": {
            "workload": "%s: %s on [%g,%g]^%d, k=%d, n=%d, trials=%d, depth=%d, m=%g, "
                        "budget 2^24 cells/level, 2^40 points/run" % (
                            w.name, INTEGRAND_TEXT.get(w.integrand, w.integrand), w.lo[0],
                            w.hi[0], w.dim, w.k, w.n, w.trials, w.depth, w.sigma_multiplier),
            "precision": args.precision, "seed": w.seed, "parallelism": "replicas x%d" % world,
            "l2": "flushed between steps (256 MiB write, outside the timed events)",
            "samples_per_step": r.samples, "levels_run": r.levels_run,
            "cells_per_level": r.cells_per_level, "flagged_per_level": r.flagged_per_level,
            "status": r.status, "result": r.value, "std": r.std,
            "work_plan": r.work_plan,
            "exact": exact,
            "result_minus_exact_over_std": (r.value - exact) / r.std
            if exact is not None and r.std > 0 else None,
        },
        "roofline": {
            "bound": "alu", "kernel": "zmc_eval_reduce (fused Philox/evaluate/reduce)",
            "achieved": round(achieved, 3), "peak": round(peak, 3),
            "unit": "T 32x32->64-bit multiplies/s",
            "frac": round(achieved / peak, 4),
            "peak_basis": "%d IMAD.WIDE/clk/SM x %d SMs x %.0f MHz (max SM clock)" % (
                WIDE_MULS_PER_SM_CLK, sms, max_mhz),
            "work_per_sample": philox_multiplies_per_sample(w.dim, prec == zmc.ZMC_FP64),
            "kernel_ms_per_step": round(sum(eval_ms) / len(eval_ms), 3),
            "kernel_share_of_step": round(sum(eval_ms) / total_ms, 4),
            "fp32_flops_per_sample": None if prec == zmc.ZMC_FP64 else fp32_flops_per_sample(
                w.integrand, w.dim),
            "fp32_flop_frac": None if prec == zmc.ZMC_FP64 else round(
                fp32_flops_per_sample(w.integrand, w.dim) * sum(samples) / eval_s
                / (2 * 128 * sms * max_mhz * 1e6), 4),
            "algorithmic_bytes": round(algorithmic_bytes_per_launch(
                r.cells_per_level, w.n, w.trials, prec == zmc.ZMC_FP64)),
            "traffic": traffic_per_launch(w, prec == zmc.ZMC_FP64),
            "traffic_basis": "ncu dram__bytes_read.sum + dram__bytes_write.sum per launch, "
                             "mean over one step's launches; null unless the kernel sources "
                             "match the capture",
        },
        "clocks": clk,
        "e2e": {"value": round(e2e_value, 3), "unit": UNIT, "h2d_bytes_per_step": h2d_bytes,
                "d2h_bytes_per_step": d2h_bytes},
        "gpu_launches": kernels_per_run * args.steps,
        "fp64": fp64,
        "fp32_kahan": kahan,
        "batched": batched,
        "corner8d": corner,
        "time_to_accuracy": tta,
        "paper": paper,
        "mixed_error_vs_oracle": mixed_error,
        "cpu_baseline": cpu,
    }
    return line


# ------------------------------------------------------- precision legs

def run_leg(zmc, w, prec_name, stream, steps=2):
    """One workload in one precision: a warm-up run (launch-shape tuning,
    graph capture), then `steps` timed runs of the captured graph with CUDA
    events on the launching stream, L2 flushed before each."""
    import torch
    prec = zmc.PRECISIONS[prec_name]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    with zmc.Integrator(w.dim, w.lo, w.hi, w.k, w.n, w.trials, w.depth, w.sigma_multiplier,
                        w.seed, w.integrand, w.params, precision=prec) as it:
        it.integrate(stream)
        ms, r = [], None
        for _ in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            it.enqueue(stream)
            e1.record(stream)
            r = it.read_result(stream)
            ms.append(e0.elapsed_time(e1))
    try:
        exact = exact_value(w)
    except ValueError:
        exact = None
    return {"precision": prec_name, "value": round(r.samples * steps / (sum(ms) * 1e-3) / 1e9, 3),
            "unit": UNIT, "steps": steps, "ms_per_step": round(sum(ms) / steps, 3),
            "samples_per_step": r.samples, "result": r.value, "std": r.std, "exact": exact,
            "result_minus_exact_over_std": (r.value - exact) / r.std
            if exact is not None and r.std > 0 else None,
            "levels_run": r.levels_run, "flagged_per_level": r.flagged_per_level,
            "status": r.status}


def level1_sums(zmc, w, prec_name, stream):
    """Level-1 (S1, S2) per (cell, trial) as the sampling kernel produced them:
    a traced depth-1 run (level 1's streams and work units do not depend on
    the depth)."""
    with zmc.Integrator(w.dim, w.lo, w.hi, w.k, w.n, w.trials, 1, w.sigma_multiplier, w.seed,
                        w.integrand, w.params, precision=zmc.PRECISIONS[prec_name]) as it:
        it.trace(True)
        it.integrate(stream)
        return it.trace_level(1)["sums"]


ERROR_TILES = 64


def error_vs_oracle(w, prec_name, sums):
    """The kernel's arithmetic error on ERROR_TILES sampled level-1 cells (all
    their trials): the FP64 oracle recomputes those tiles on the same points
    (the FP32 stream for the FP32 modes).  S1 errors are given relative to
    the tile's scale sqrt(n S2) + |S1| (S1 of an oscillating integrand cancels)
    and per cell as the error of the cell's mean in units of its spread over
    trials (arithmetic error against Monte Carlo noise)."""
    import numpy as np
    from oracle import zmc_oracle as O
    C = sums.shape[0]
    rng = np.random.default_rng(2024)
    cells = np.sort(rng.choice(C, size=min(C, ERROR_TILES), replace=False))
    ref = O.cell_sums(w.seed, 1, w.lo, w.hi, w.k, w.n, w.trials, w.integrand, w.params, cells,
                      O.level1_cells(w.k, w.dim)[cells], fp32_uniforms=prec_name != "fp64")
    got = sums[cells]
    d1 = np.abs(got[..., 0] - ref[..., 0])
    scale = np.sqrt(w.n * np.abs(ref[..., 1])) + np.abs(ref[..., 0])
    volume = float(np.prod(O.level_widths(w.lo, w.hi, w.k, 1)))
    _, mean_ref, spread_ref = O.cell_statistics(ref, volume, w.n)
    _, mean_got, _ = O.cell_statistics(got, volume, w.n)
    pos = spread_ref > 0
    return {"precision": prec_name, "cells": int(cells.size), "tiles": int(cells.size * w.trials),
            "points": int(cells.size * w.trials * w.n),
            "stream": "FP64 stream" if prec_name == "fp64" else "FP32 stream",
            "max_rel_s1_err": float("%.3g" % float(np.max(d1 / scale))),
            "max_cell_mean_err_over_spread": float("%.3g" % float(
                np.max(np.abs(mean_got - mean_ref)[pos] / spread_ref[pos]))) if pos.any() else None,
            "test_tolerance_rel_s1": 1e-12 if prec_name == "fp64" else 2e-5}


def paper_rows(zmc, stream, fp64_max_samples=int(4e9)):
    """The paper's parameter sets (Sec. 3, Tab. 1-4) once each after a
    warm-up, FP32-mixed for all and FP64 for those of at most
    fp64_max_samples points; host wall clock around zmc_integrate."""
    rows = []
    for label, table, w in paper_runs():
        exact = exact_value(w)
        for prec in ("fp32_fp64acc", "fp64"):
            if prec == "fp64" and w.k ** w.dim * w.n * w.trials > fp64_max_samples:
                continue
            with zmc.Integrator(w.dim, w.lo, w.hi, w.k, w.n, w.trials, w.depth,
                                w.sigma_multiplier, w.seed, w.integrand, w.params,
                                precision=zmc.PRECISIONS[prec]) as it:
                it.integrate(stream)
                t0 = time.perf_counter()
                r = it.integrate(stream)
                dt = time.perf_counter() - t0
            rows.append({"run": label, "paper_table": table, "precision": prec,
                         "cells_per_dim": w.k, "points_per_cell": w.n, "trials": w.trials,
                         "depth": w.depth, "sigma_multiplier": w.sigma_multiplier,
                         "result": r.value, "std": r.std, "closed_form": exact,
                         "seconds": round(dt, 4), "samples": r.samples,
                         "gsamples_per_s": round(r.samples / dt / 1e9, 2),
                         "levels_run": r.levels_run, "flagged_per_level": r.flagged_per_level,
                         "status": r.status})
    return rows


# ----------------------------------------------------------- batched leg

BATCH_MAX_SAMPLES = 1 << 32     # per integral: about 2x the largest level 1


def run_batched(zmc, stream, prec, steps: int = 3):
    """512 Genz integrals (d 2..9, k 2..6, n 2^10..2^15, depth 1..4, 8 trials,
    m = 2) through zmc_integrate_batch: one persistent sampling kernel per
    level.  Timed end to end per call (parameters up, results down)."""
    import torch
    from paper_1902_07916_gb300 import workloads
    ws = workloads.genz_batch(512, seed=0)
    hs = []
    try:
        for w in ws:
            h = zmc.zmc_create(w.dim, w.lo, w.hi, w.k, w.n, w.trials, w.depth,
                               w.sigma_multiplier, w.seed)
            hs.append(h)
            zmc.zmc_set_integrand(h, w.integrand, w.params)
            zmc.zmc_set_precision(h, prec)
            zmc.zmc_set_limits(h, 1 << 24, max(BATCH_MAX_SAMPLES, w.level1_samples()))
        zmc.zmc_integrate_batch(hs, stream)                 # warm-up: buffers, graphs
        times, res = [], None
        for _ in range(steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res = zmc.zmc_integrate_batch(hs, stream)
            times.append(time.perf_counter() - t0)
        samples = sum(r.samples for r in res)
        return {"value": round(samples / (sum(times) / len(times)) / 1e9, 3), "unit": UNIT,
                "integrals": len(ws), "samples_per_call": samples,
                "ms_per_call": round(1e3 * sum(times) / len(times), 2), "steps": steps,
                "budget": "2^32 points per integral (or its level 1)",
                "budget_stopped": sum(1 for r in res if r.status == zmc.ZMC_ERR_BUDGET),
                "timing": "host wall clock around zmc_integrate_batch (uploads, all levels, "
                          "result download)"}
    finally:
        for h in hs:
            zmc.zmc_destroy(h)


# ------------------------------------------------------ time to accuracy

TTA_TARGET = 1e-4
TTA_SEEDS = 5
TTA_N = [1 << e for e in range(10, 23)]
TTA_SWEEP_BUDGET_S = 90.0
TTA_FP64_BUDGET_S = 75.0


def exact_value(w) -> float:
    """Closed form of a workload whose integrand is a product of (or the sine
    of a sum of) one-dimensional terms: the normalised Gaussian integrates to
    a product of erf differences, sin(sum x) to the imaginary part of a
    product of (e^{i h} - e^{i l}) / i (Eqs. 1-2 of Sec. 3)."""
    if w.integrand == "gauss_norm":
        s = w.params[0] * math.sqrt(2.0)
        return math.prod(0.5 * (math.erf(h / s) - math.erf(l / s)) for l, h in zip(w.lo, w.hi))
    if w.integrand == "sin_sum":
        z = complex(1.0, 0.0)
        for l, h in zip(w.lo, w.hi):
            z *= (complex(math.cos(h), math.sin(h)) - complex(math.cos(l), math.sin(l))) / 1j
        return z.imag
    if w.integrand == "genz_corner":
        return corner_peak_exact(w.lo, w.hi, w.params)
    raise ValueError("no closed form for " + w.integrand)


def corner_peak_exact(lo, hi, a) -> float:
    """int over the box of (1 + a.x)^-(d+1): integrating each dimension in
    turn, 1 / (d! prod a_i) times the alternating sum over the box's vertices
    v of (-1)^(number of upper coordinates of v) / (1 + a.v), in exact
    rationals (the sum cancels badly in floating point)."""
    from fractions import Fraction
    import itertools
    d = len(a)
    fa = [Fraction(x) for x in a]
    flo, fhi = [Fraction(x) for x in lo], [Fraction(x) for x in hi]
    total = Fraction(0)
    for upper in itertools.product((0, 1), repeat=d):
        s = 1 + sum(ai * (h if u else l) for ai, l, h, u in zip(fa, flo, fhi, upper))
        total += Fraction((-1) ** sum(upper)) / s
    return float(total / (math.factorial(d) * math.prod(fa)))


def median_first(firsts):
    """Median over seeds of the first n meeting a criterion (unmet = never):
    (n, seed) of the median seed, or (None, None) when fewer than half met it."""
    order = sorted(range(len(firsts)), key=lambda i: (firsts[i] is None, firsts[i] or 0, i))
    mid = order[len(order) // 2]
    return (firsts[mid], mid) if firsts[mid] is not None else (None, None)


def run_tta(zmc, stream):
    """Time to a relative error of 1e-4 on the 9-D normalised Gaussian
    (sigma 0.1 on [-1,1]^9, k = 3, 8 trials, depth 4, m = 2) at n = 2^10,
    2^11, ... points per cell and trial.  Two criteria per seed: the error
    against the closed form, |value - exact| / |exact| <= 1e-4, and the
    stated error, 3 std / |value| <= 1e-4; each is the median over five seeds
    of the first n that meets it.  The five seeds run as one batched call per
    n (a batched result equals the single run bit for bit).  At the median
    seed's n, a single FP32-mixed run and an FP64 run are timed; the FP64
    stream draws other points, so its error at that n is an independent draw
    of the same estimator's error and is reported beside its time.  Every time
    is host wall clock around the first call on a fresh handle: parameters up,
    buffers, graph capture, all levels and the result down."""
    import torch
    from paper_1902_07916_gb300 import workloads
    w = workloads.gauss9d()
    exact = exact_value(w)
    crit = {"rel_err": lambda r: abs(r.value - exact) / abs(exact),
            "three_std": lambda r: 3.0 * r.std / abs(r.value) if r.value else math.inf}
    first = {c: [None] * TTA_SEEDS for c in crit}
    batch_s, sweep = {}, []

    def handle(n, seed, prec):
        h = zmc.zmc_create(w.dim, w.lo, w.hi, w.k, n, w.trials, w.depth, w.sigma_multiplier,
                           seed)
        zmc.zmc_set_integrand(h, w.integrand, w.params)
        zmc.zmc_set_precision(h, prec)
        return h

    def timed_single(n, seed, prec):
        h = handle(n, seed, prec)
        try:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = zmc.zmc_integrate(h, stream)
            return time.perf_counter() - t0, r
        finally:
            zmc.zmc_destroy(h)

    # untimed: load the kernels and fill the launch-shape tuner's cache
    for prec in (zmc.ZMC_FP32_FP64ACC, zmc.ZMC_FP64):
        timed_single(TTA_N[0], 0, prec)

    t_start = time.perf_counter()
    for n in TTA_N:
        hs = [handle(n, s, zmc.ZMC_FP32_FP64ACC) for s in range(TTA_SEEDS)]
        try:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res = zmc.zmc_integrate_batch(hs, stream)
            batch_s[n] = time.perf_counter() - t0
        finally:
            for h in hs:
                zmc.zmc_destroy(h)
        row = {"n": n, "batch_call_s": round(batch_s[n], 4), "samples_seed0": res[0].samples}
        for c, f in crit.items():
            errs = [f(r) for r in res]
            row[c] = [float("%.3g" % e) for e in errs]
            for i, e in enumerate(errs):
                if first[c][i] is None and e <= TTA_TARGET:
                    first[c][i] = n
        sweep.append(row)
        if all(x is not None for c in crit for x in first[c]):
            break
        if time.perf_counter() - t_start > TTA_SWEEP_BUDGET_S:
            break

    out = {"workload": "gauss9d: normalised Gaussian sigma=0.1 on [-1,1]^9, k=3, trials=8, "
                       "depth=4, m=2, default budget; n doubled from 2^10",
           "target": TTA_TARGET, "seeds": TTA_SEEDS, "exact": exact,
           "timing": "host wall clock, first zmc_integrate(_batch) call on fresh handles",
           "sweep": sweep}
    for c in crit:
        n_med, seed = median_first(first[c])
        entry = {"first_n_per_seed": first[c], "median_n": n_med}
        if n_med is not None:
            t32, r32 = timed_single(n_med, seed, zmc.ZMC_FP32_FP64ACC)
            entry.update({"seed": seed, "fp32_mixed_s": round(t32, 4),
                          "batched_s_per_integral": round(batch_s[n_med] / TTA_SEEDS, 4),
                          "batched_call_s": round(batch_s[n_med], 4),
                          "fp32_mixed_err": float("%.3g" % crit[c](r32))})
            if t32 * 14 <= TTA_FP64_BUDGET_S:
                t64, r64 = timed_single(n_med, seed, zmc.ZMC_FP64)
                entry.update({"fp64_s": round(t64, 4),
                              "fp64_err": float("%.3g" % crit[c](r64)),
                              "fp64_met_target": crit[c](r64) <= TTA_TARGET,
                              "fp64_over_fp32_mixed": round(t64 / t32, 2)})
            else:
                entry["fp64_s"] = None
                entry["fp64_note"] = "not run: estimated over %.0f s" % TTA_FP64_BUDGET_S
        out[c] = entry
    return out


# ------------------------------------------------------ CPU baseline

def cpu_baseline(w, target_s: float = 12.0, max_cells: int | None = None):
    """The FP64 oracle on the host cores: level-1 (cell, trial) sums of the
    first M cells of the workload, M doubled until the run takes target_s."""
    import numpy as np
    from oracle import zmc_oracle as O
    threads = O.default_threads()
    coords_all = O.level1_cells(w.k, w.dim)
    M = 1
    limit = max_cells or coords_all.shape[0]
    while True:
        t0 = time.perf_counter()
        O.cell_sums(w.seed, 1, w.lo, w.hi, w.k, w.n, w.trials, w.integrand, w.params,
                    np.arange(M), coords_all[:M], threads=threads)
        dt = time.perf_counter() - t0
        if dt >= target_s or M >= limit:
            break
        M = min(limit, max(M * 2, int(M * target_s / max(dt, 1e-3) * 1.1)))
    samples = M * w.trials * w.n
    return {"value": round(samples / dt / 1e9, 5), "unit": UNIT, "cores": threads,
            "kind": "oracle",
            "sample": "level-1 sums of the first %d of %d cells x %d trials x %d points "
                      "(%.3g points, %.1f s)" % (M, coords_all.shape[0], w.trials, w.n,
                                                  samples, dt)}


def run_reference(args, world, rank):
    if rank != 0:
        return None
    import numpy as np
    from oracle import zmc_oracle as O
    w = workload(args)
    threads = O.default_threads()
    coords_all = O.level1_cells(w.k, w.dim)
    # each step: a bounded sample of level-1 cells, sized to ~2 s on the host
    M = 1
    while True:
        t0 = time.perf_counter()
        O.cell_sums(w.seed, 1, w.lo, w.hi, w.k, w.n, w.trials, w.integrand, w.params,
                    np.arange(M), coords_all[:M], threads=threads)
        dt = time.perf_counter() - t0
        if dt >= 1.0 or M >= coords_all.shape[0]:
            break
        M = min(coords_all.shape[0], max(2 * M, int(M * 2.0 / max(dt, 1e-3))))
    for _ in range(args.warmup):
        O.cell_sums(w.seed, 1, w.lo, w.hi, w.k, w.n, w.trials, w.integrand, w.params,
                    np.arange(M), coords_all[:M], threads=threads)
    times = []
    for s in range(args.steps):
        lo_c = (s * M) % coords_all.shape[0]
        idx = (np.arange(M) + lo_c) % coords_all.shape[0]
        t0 = time.perf_counter()
        O.cell_sums(w.seed, 1, w.lo, w.hi, w.k, w.n, w.trials, w.integrand, w.params,
                    idx, coords_all[idx], threads=threads)
        times.append(time.perf_counter() - t0)
    samples = M * w.trials * w.n
    value = samples * len(times) / sum(times) / 1e9
    sample = ("per step: level-1 sums of %d cells x %d trials x %d points (%.3g points)"
              % (M, w.trials, w.n, samples))
    return {
        "impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * sum(times) / len(times), 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (analytic integrand, Philox counter-based points)",
        "config": {"workload": "%s (CPU oracle, bounded sample)" % w.name,
                   "precision": "fp64"},
        "cpu_baseline": {"value": round(value, 5), "unit": UNIT, "cores": threads,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 5), "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }


# ------------------------------------------------------ paper parameter sets

def paper_runs():
    """The paper's own parameter sets (Sec. 3), one GB300: (name, table,
    workload).  Points per cell follow each version: n2^D for the TensorFlow
    and multiprocessing runs, a flat count for the Ray runs."""
    from paper_1902_07916_gb300.workloads import Workload
    f1 = lambda name, k, n, T, depth, m: Workload(name, "sin_sum", 6, [0.0] * 6, [10.0] * 6,
                                                  k, n, T, depth, m, 0)
    f2 = lambda name, d, k, n, T, depth, m: Workload(name, "gauss_norm", d, [-1.0] * d,
                                                     [1.0] * d, k, n, T, depth, m, 0, [0.01])
    return [
        ("f1 TF", "Tab. 1", f1("E1_tf", 3, 20 ** 6, 5, 2, 5.0)),
        ("f1 Numba-MP", "Tab. 1", f1("E1_mp", 6, 10 ** 6, 5, 2, 5.0)),
        ("f2 9-D Numba-MP", "Tab. 2", f2("E2_mp", 9, 3, 3 ** 9, 5, 4, 5.0)),
        ("f1 Ray", "Tab. 3", f1("E3_ray", 12, 10 ** 4, 5, 1, 5.0)),
        ("f2 9-D Ray", "Tab. 4", f2("E4_ray9", 9, 3, 10 ** 4, 5, 4, 4.0)),
        ("f2 12-D Ray", "Tab. 4", f2("E4_ray12", 12, 3, 10 ** 4, 5, 4, 4.0)),
    ]


def run_paper(args):
    """Each of the paper's parameter sets once (after a warm-up), FP64 and
    FP32-mixed, timed end to end through zmc_integrate; results with the
    closed forms, as context rows beside the paper's tables."""
    import torch
    from paper_1902_07916_gb300 import build as libbuild
    libbuild.build()
    from paper_1902_07916_gb300 import zmc
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    return {"paper_parameter_sets": paper_rows(zmc, stream, fp64_max_samples=1 << 62),
            "gpu": torch.cuda.get_device_name(0)}


# ------------------------------------------------------------ pipe rates

# zmc_pipe_probe kinds: (name, kind id, what one chain step issues).  Every
# thread runs 8 independent chains; one iteration is one step of each.
PROBE_KINDS = [
    ("imad_wide", 0, "one mad.wide.u32 (32x32->64-bit product)"),
    ("imad", 1, "one mad.lo.u32"),
    ("imad_hi", 2, "one mad.hi.u32"),
    ("hilo_paired", 3, "high and low half of one product + a three-input XOR"),
    ("hilo_split", 4, "the same, low half's multiplier from a kernel parameter"),
    ("lop3", 5, "one three-input XOR"),
    ("ffma", 6, "one FP32 fma"),
    ("dfma", 7, "one FP64 fma"),
    ("philox", 8, "one Philox4x32-10 block as the sampling kernel forms it"),
    ("philox_split", 9, "one Philox4x32-10 block with split high/low products"),
]
PROBE_CHAINS = 8
PROBE_THREADS = 256
PROBE_CTAS_PER_SM = 4
PROBE_TARGET_MS = 40.0


def per_sm_rates(records, ops_per_cta):
    """Rates from the CTAs' (clock64 start, end, ns start, end, smid) records:
    per SM, the operations of the CTAs it ran over its own cycle span."""
    by_sm = {}
    for c0, c1, t0, t1, sm, _ in records:
        by_sm.setdefault(sm, []).append((c0, c1, t0, t1))
    rates, mhz, ctas = [], [], []
    for recs in by_sm.values():
        span = max(r[1] for r in recs) - min(r[0] for r in recs)
        ns = max(r[3] for r in recs) - min(r[2] for r in recs)
        rates.append(len(recs) * ops_per_cta / span)
        mhz.append(1e3 * span / ns)
        ctas.append(len(recs))
    return rates, mhz, ctas


def run_peaks(args):
    """Every probe kind once at a calibrated length (about 40 ms), 4 CTAs of
    256 threads per SM on average.  Rates are thread-level operations per SM
    per clock: per SM, the work of the CTAs it ran over its own %clock64 span
    (median over SMs); the SM clock the kernel saw is that span over the
    %globaltimer span, and nvidia-smi's clocks are sampled alongside."""
    import torch
    from paper_1902_07916_gb300 import build as libbuild
    libbuild.build()
    from paper_1902_07916_gb300 import zmc
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    blocks = sms * PROBE_CTAS_PER_SM
    sink = torch.empty(blocks * PROBE_THREADS, dtype=torch.int32, device=dev)
    clocks_buf = torch.empty(blocks * 6, dtype=torch.int64, device=dev)

    def launch(kind, iters):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            zmc.zmc_pipe_probe(kind, iters, blocks, PROBE_THREADS, sink.data_ptr(),
                               clocks_buf.data_ptr(), stream)
            e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1), clocks_buf.cpu().view(blocks, 6).tolist()

    rows = {}
    with ClockSampler(0) as clk:
        for name, kind, what in PROBE_KINDS:
            iters = args.peaks_iters
            if iters is None:
                base = 64 if name == "dfma" else 4096
                launch(kind, base)                                  # warm-up
                ms, _ = launch(kind, base)
                iters = max(16, int(base * PROBE_TARGET_MS / max(ms, 1e-3)))
            ms, recs = launch(kind, iters)
            ops_cta = PROBE_THREADS * iters * PROBE_CHAINS
            rates, mhz, ctas = per_sm_rates(recs, ops_cta)
            rows[name] = {
                "what": what, "iters": iters, "event_ms": round(ms, 4),
                "per_sm_per_clk": round(statistics.median(rates), 3),
                "per_sm_per_clk_min_max": [round(min(rates), 3), round(max(rates), 3)],
                "warp_inst_per_sm_per_clk": round(statistics.median(rates) / 32, 4),
                "sm_mhz_in_kernel": round(statistics.median(mhz), 1),
                "ctas_per_sm_min_max": [min(ctas), max(ctas)], "sms_used": len(rates),
                "event_rate_per_sm_per_clk_at_max_clock": round(
                    blocks * ops_cta / (ms * 1e-3) / sms / (statistics.median(mhz) * 1e6), 3),
            }
    return {"pipe_rates": rows, "unit": "thread-level operations (or Philox blocks) per SM "
            "per clock", "sms": sms, "ctas": blocks, "threads": PROBE_THREADS,
            "chains_per_thread": PROBE_CHAINS, "gpu": torch.cuda.get_device_name(0),
            "clocks": clk.summary()}


def run_batch_compare(args):
    """The Genz batch through zmc_integrate_batch (best of three calls after a
    warm-up) against the same integrals run one by one through zmc_integrate
    (each after its own warm-up run), with points per second and the
    fraction of the IMAD.WIDE roofline (17 d / 5 wide multiplies per point)
    per dimension and per family."""
    import collections
    import torch
    from paper_1902_07916_gb300 import build as libbuild
    libbuild.build()
    from paper_1902_07916_gb300 import workloads, zmc
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    peak = WIDE_MULS_PER_SM_CLK * sms * 2070e6
    ws = workloads.genz_batch(args.batch_count, seed=0)
    hs = []
    try:
        for w in ws:
            h = zmc.zmc_create(w.dim, w.lo, w.hi, w.k, w.n, w.trials, w.depth,
                               w.sigma_multiplier, w.seed)
            hs.append(h)
            zmc.zmc_set_integrand(h, w.integrand, w.params)
            zmc.zmc_set_precision(h, args.precision)
            budget = w.level1_samples() if args.batch_level1 else max(
                BATCH_MAX_SAMPLES, w.level1_samples())
            zmc.zmc_set_limits(h, 1 << 24, budget)
        res = zmc.zmc_integrate_batch(hs, stream)
        times = []
        for _ in range(3 if not args.batch_level1 else 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res = zmc.zmc_integrate_batch(hs, stream)
            times.append(time.perf_counter() - t0)
        tb = min(times)
        out = {"integrals": len(ws), "precision": args.precision,
               "batch_s": round(tb, 4), "batch_gsamples_s": round(
                   sum(r.samples for r in res) / tb / 1e9, 2),
               "cells_per_level": [sum(int(r.cells_per_level[L]) for r in res
                                       if L < len(r.cells_per_level))
                                   for L in range(max(w.depth for w in ws))]}
        if args.batch_level1 or args.no_singles:
            return out
        single = []
        for w, h in zip(ws, hs):
            zmc.zmc_integrate(h, stream)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = zmc.zmc_integrate(h, stream)
            single.append((w, r, time.perf_counter() - t0))
    finally:
        for h in hs:
            zmc.zmc_destroy(h)
    ts = sum(s for _, _, s in single)
    muls = lambda w, r: r.samples * philox_multiplies_per_sample(w.dim, False)
    agg = collections.defaultdict(lambda: [0, 0.0, 0.0, 0])
    for w, r, s in single:
        for key in ("d=%d" % w.dim, w.integrand, "n=%d" % w.n):
            a = agg[key]
            a[0] += r.samples
            a[1] += muls(w, r)
            a[2] += s
            a[3] += 1
    all_muls = sum(muls(w, r) for w, r, _ in single)
    out.update({
        "singles_sum_s": round(ts, 4),
        "singles_gsamples_s": round(sum(r.samples for _, r, _ in single) / ts / 1e9, 2),
        "batch_wide_mult_frac": round(all_muls / tb / peak, 4),
        "singles_wide_mult_frac": round(all_muls / ts / peak, 4),
        "samples_weighted_dim": round(sum(r.samples * w.dim for w, r, _ in single)
                                      / sum(r.samples for _, r, _ in single), 3),
        "singles_by": {k: {"integrals": v[3], "seconds": round(v[2], 4),
                           "gsamples_s": round(v[0] / v[2] / 1e9, 1),
                           "wide_mult_frac": round(v[1] / v[2] / peak, 3)}
                       for k, v in sorted(agg.items())},
        "timing": "host wall clock around each call; peak = 32 IMAD.WIDE/clk/SM at 2070 MHz"})
    return out


def main():
    args = parse()
    world, rank, local = dist_env()
    if args.paper:
        print(json.dumps(run_paper(args)), flush=True)
        return
    if args.peaks:
        print(json.dumps(run_peaks(args)), flush=True)
        return
    if args.batch_compare:
        print(json.dumps(run_batch_compare(args)), flush=True)
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    try:
        if args.impl == "reference":
            line = run_reference(args, world, rank)
        else:
            line = run_ours(args, world, rank, local)
        if line is not None:
            print(json.dumps(line), flush=True)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
