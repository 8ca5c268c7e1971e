#!/usr/bin/env python3
"""Benchmark of the GB300 light-curve generator (Sartori et al. 2019, Sec. 2.1).

Workload (one step = one whole generator run over one batch): 4096 curves of
N = 2^16 samples, dt = 1 day, Eq. 3 PSD (f_br = 1/300 d^-1, slopes 1 / 2),
broken-power-law ERDF on [-4, 0] (break -1.5, slopes +0.4 / -2.5), seeds
0..4095, 200 amplitude-adjustment iterations, FP32 with FP64 twiddles and
variance sums.  Metric: light-curve samples x iterations per second.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun every rank generates its own 4096-curve batch (curve ids offset
by rank, no collective on the data path: weak scaling); the step time is the
max over ranks.  --impl reference times the FP64 CPU oracle on the host cores
on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1909_06374_gb300 import workloads  # noqa: E402

NCURVES, LOG2N, ITERS = 4096, 16, 200
METRIC = "light-curve samples x E13 iterations per second"
UNIT = "sample*iter/s"
ALG_BYTES_PER_SAMPLE_ITER = 14  # read x 4 + read A 2 + read s 4 + write x 4 (FP32)
# Algorithmic bytes of one argsort (all radix passes) per element, FP32 keys:
# pass 0 reads the value and writes key + position (12 B), passes 1-2 read and
# write key + position (16 B each), the last reads key + position and the
# sorted draw and writes the state (16 B).  FP64: 8 passes of 8-byte keys.
SORT_BYTES_PER_ELEMENT = {4: 12 + 16 + 16 + 16, 8: 20 + 6 * 24 + 28}
# The sample sort's scatter group (FP32): the bucket scatter reads the value and its
# bucket byte and writes value + position (13 B), the on-chip finish reads them
# back, reads the sorted draws and writes the state (16 B).
BUCKET_SCATTER_BYTES_PER_ELEMENT = 13 + 16
# DRAM bytes (read + write) of the four FP32 scatter passes per element, from
# one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum of the four
# scatter launches of one argsort over 512 curves x 2^16 samples)
SCATTER_DRAM_BYTES_PER_ELEMENT_FP32 = 1.8893e9 / 2 ** 25
# DRAM bytes (read + write) of one whole iteration per sample of the uniform
# batch, from one ncu capture of every kernel of an iteration over 512 curves
# x 2^16 (1218.3 MB read + 602.9 MB written; the working set exceeds L2 there
# as at 4096 curves).  The finish kernel's launch shape has changed since
# (fewer empty blocks, a tail launch), so the bench line reports it as the
# last capture's figure and leaves `traffic` null.
ITER_DRAM_BYTES_PER_SAMPLE = 1821.2e6 / 2 ** 25
ITER_DRAM_CAPTURE_CURRENT = False
# Bytes of the sample sort per element (FP32): histogram 4, bucket scatter 4 +
# 1 + 8, finish 8 + 4 + 4, bucket byte written 1
BUCKET_SORT_BYTES_PER_ELEMENT = 34
SAMPLE_SORT_LOG2 = (13, 20)  # FP32 lengths on the sample sort
FUSED_LOG2 = (10, 14)        # FP32 lengths the one-CTA fused kernel can take


def scheduled_bytes_per_sample_iter(jobs, esize, fused_elements):
    """HBM bytes the scheduled kernels move per sample-iteration (reads +
    writes at their algorithmic sizes), averaged over the batch's
    sample-iterations, beside the 14 B floor (28 B in FP64).  Multi-kernel
    curves: the transforms' passes (tile path, log2 M >= 12: P = ceil(log2 M /
    9) passes each way, 8 in FP64, the middle two fused into one kernel, so 2P -
    1 kernels that each read and write the complex array; radix-pass path: P
    passes each way and the spectral kernel), each 2 esize B per sample, plus
    the amplitudes (esize / 2 B per sample); then the argsort: the sample
    sort's 34 B per element, or the radix passes with their histograms
    (FP32: 4 x 4 + 60 = 76 B; FP64: 8 x 8 + 192 = 256 B).  Fused curves touch
    HBM once per launch of all iterations: 14 B per sample (FP32) / iterations.
    The fused curves are those of 2^10..2^top for the top length whose
    samples add up to the plan's fused samples (the path table's crossover,
    2^12 built in, or LC_RESIDENT_MAX_LOG2); with no such top the figure is
    not defined (None).  Without the Eq. 4 pass."""
    fp32 = esize == 4
    fused_ids = None
    for top in range(FUSED_LOG2[0] - 1, FUSED_LOG2[1] + 1):
        fused_len = [j for j in jobs if fp32 and FUSED_LOG2[0] <= int(j["log2n"]) <= top]
        if sum(1 << int(j["log2n"]) for j in fused_len) == fused_elements:
            fused_ids = {id(j) for j in fused_len}
            break
    if fused_ids is None:
        return None
    tot_b, tot_si = 0.0, 0
    for j in jobs:
        log2n, iters = int(j["log2n"]), int(j["iters"])
        n = 1 << log2n
        if iters <= 0:
            continue
        if id(j) in fused_ids:
            per = ALG_BYTES_PER_SAMPLE_ITER * esize / 4 / iters
        else:
            log2m = log2n - 1
            if log2m >= 12:
                p = -(-log2m // (9 if fp32 else 8))
                kernels = 2 * p - 1
            else:
                p = (1 if log2m % 4 else 0) + log2m // 4
                kernels = 2 * p + 1
            fft = kernels * 2 * esize + esize / 2
            if fp32 and SAMPLE_SORT_LOG2[0] <= log2n <= SAMPLE_SORT_LOG2[1]:
                sort = BUCKET_SORT_BYTES_PER_ELEMENT
            else:
                passes = esize  # 8-bit digits of esize-byte keys
                sort = passes * esize + SORT_BYTES_PER_ELEMENT[esize]  # histograms + scatter passes
            per = fft + sort
        tot_b += per * n * iters
        tot_si += n * iters
    return tot_b / tot_si if tot_si else None
WORKLOAD = (f"uniform batch: {NCURVES} curves x 2^{LOG2N} samples, dt=1 d, bending PL PSD "
            f"(f_br=1/300 d^-1, slopes 1 and 2), broken-PL ERDF [-4,0] break -1.5 slopes +0.4/-2.5, "
            f"{ITERS} E13 iterations, FP32")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--curves", type=int, default=NCURVES,
                    help="curves per GPU; anything but 4096 is a profiling case, not the bench workload")
    ap.add_argument("--log2n", type=int, default=LOG2N,
                    help="log2 of the curve length; anything but 16 is a profiling case")
    ap.add_argument("--workload", default="uniform", choices=["uniform", "single", "long", "ragged", "serving"],
                    help="uniform (default) is the benchmark line; the others are the remaining workloads")
    ap.add_argument("--serving-seconds", type=float, default=60.0)
    ap.add_argument("--serving-rate", type=float, default=200.0, help="requests per second of --workload serving")
    ap.add_argument("--headline-only", action="store_true",
                    help="print only the uniform-batch line (no single / long / ragged / serving lines)")
    ap.add_argument("--erdf", default=None, choices=["smooth_eq1", "table2", "lognormal"],
                    help="give every curve of the uniform workload this tabulated ERDF shape (Eq. 1 / Eq. 2); "
                         "a variant line, not the bench workload")
    ap.add_argument("--post", action="store_true",
                    help="also time the App. A estimators (periodogram, 64-lag structure function) on the output")
    ap.add_argument("--convergence", type=float, default=None, metavar="THRESHOLD",
                    help="run with the Eq. 4 convergence test on (every curve stops once delta < THRESHOLD; "
                         "0 = measure delta without stopping); a variant line, not the bench workload")
    return ap.parse_args()


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def jobs_for_rank(rank, ncurves=NCURVES, log2n=LOG2N):
    jobs = workloads.uniform(ncurves=ncurves, log2n=log2n, iters=ITERS)
    for j in jobs:
        j["seed"] += rank * ncurves
        j["curve_id"] += rank * ncurves
    return jobs


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.gpu)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# ------------------------------------------------------------------ oracle
def cpu_baseline_run(ncurves, iters, cores, jobs=None, prec=0):
    """The FP64 CPU oracle on `ncurves` curves of the workload (`iters`
    iterations each), or on the given jobs, one curve per host thread;
    returns samples*iter/s, the threads used and the seconds."""
    import oracle
    oracle.build()
    if jobs is None:
        jobs = workloads.uniform(ncurves=ncurves, log2n=LOG2N, iters=iters)
    t0 = time.perf_counter()
    _, used = oracle.generate_batch(jobs, prec=prec, nthreads=cores)
    dt = time.perf_counter() - t0
    return workloads.sample_iters(jobs) / dt, min(used, len(jobs)), dt  # threads that had a curve


def cpu_baseline_sample(workload, cores):
    """A bounded sample of a non-headline workload for the CPU oracle (a few to
    some tens of seconds of CPU work) and its description."""
    if workload == "single":
        return workloads.single(), 1, "the whole workload: 1 curve x 2^14 samples x 100 iterations, FP64"
    if workload == "long":
        jobs = [dict(j, log2n=22, iters=2) for j in workloads.long_curves()][:cores]
        return jobs, 0, (f"{len(jobs)} of the long curves' parameter sets at 2^22 samples (2^26 takes minutes "
                         "per oracle iteration) x 2 iterations, one curve per thread")
    jobs = [dict(j, iters=5) for j in workloads.ragged()[:cores]]
    return jobs, 0, (f"the first {len(jobs)} ragged curves (their own lengths 2^10..2^20 and parameters) x 5 "
                     "iterations, one curve per thread")


def run_reference(args):
    rank, world, local = dist_info()
    if rank != 0:
        return 0
    cores = os.cpu_count() or 1
    ncurves, iters = cores, 50
    for _ in range(args.warmup):
        cpu_baseline_run(ncurves, iters, cores)
    vals, dts = [], []
    used = cores
    for _ in range(args.steps):
        v, used, dt = cpu_baseline_run(ncurves, iters, cores)
        vals.append(v)
        dts.append(dt)
    value = sum(ncurves * (1 << LOG2N) * iters for _ in vals) / sum(dts)
    sample = f"{ncurves} curves x 2^{LOG2N} samples x {iters} iterations per step (one curve per thread)"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * statistics.mean(dts),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU arm
WORKLOAD_DESC = {
    "single": "single curve: 1 x 2^14 samples, 100 E13 iterations, FP64 (latency)",
    "long": "long curves: 8 x 2^26 samples, dt = 7 d, per-curve f_br / high slope, 50 E13 iterations, FP32",
    "ragged": ("ragged batch: 10000 curves, N log-uniform over 2^10..2^20, per-curve PSD and ERDF, "
               "100 E13 iterations, FP32"),
}


def rank_jobs(workload, rank, world, curves=NCURVES, log2n=LOG2N):
    """This rank's jobs of a workload, its precision (0 FP32, 1 FP64), dtype
    name and description.  uniform: every rank generates its own batch (curve
    ids offset by rank: weak scaling); single: rank 0 only; long, ragged: the
    job list sharded by work, every curve on exactly one rank."""
    if workload == "uniform":
        jobs = jobs_for_rank(rank, curves, log2n)
        desc = WORKLOAD if (curves, log2n) == (NCURVES, LOG2N) else \
            f"PROFILING CASE ({curves} curves x 2^{log2n}), not the bench workload"
        return jobs, 0, "f32", desc
    if workload == "single":
        return (workloads.single() if rank == 0 else []), 1, "f64", WORKLOAD_DESC["single"]
    full = workloads.long_curves() if workload == "long" else workloads.ragged()
    return workloads.shard_jobs(full, world)[rank], 0, "f32", WORKLOAD_DESC[workload]


class HostClock:
    """Wall clock around a region (for host-side tests of the step loop)."""

    def start(self):
        self.t0 = time.perf_counter()

    def stop(self):
        self.t1 = time.perf_counter()

    def ms(self):
        return 1000.0 * (self.t1 - self.t0)


class CudaClock:
    """CUDA events on `stream` around a region."""

    def __init__(self, stream):
        import torch
        self.stream = stream
        self.a = torch.cuda.Event(enable_timing=True)
        self.b = torch.cuda.Event(enable_timing=True)

    def start(self):
        self.a.record(self.stream)

    def stop(self):
        self.b.record(self.stream)

    def ms(self):
        return self.a.elapsed_time(self.b)


def timed_steps(step, steps, barrier, clock):
    """Exactly `steps` calls of step() between a barrier + clock on each side;
    returns this rank's milliseconds."""
    barrier()
    clock.start()
    for _ in range(steps):
        step()
    clock.stop()
    barrier()
    return clock.ms()


def reduce_over_ranks(v, dist, op):
    """max / sum of a float over the ranks (the value itself without a group)."""
    if dist is None:
        return float(v)
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(v)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def throughput(total_sample_iters, steps, max_ms):
    """Whole-job sample*iter/s: the work of all ranks over the slowest rank's time."""
    return total_sample_iters * steps / (max_ms / 1000.0)


def gpu_line(args, workload, steps, warmup, dist, e2e_on, cpu_on, extra=False):
    """Run one workload on this rank's GPU and return its JSON line (rank 0)
    or None."""
    import torch
    from paper_1909_06374_gb300 import (LC_FP32, LC_FP64, Plan, lc_generate_host, lc_plan_create,
                                        lc_plan_destroy, lc_plan_last_launches, lc_plan_profile, lc_plan_timing)
    from paper_1909_06374_gb300 import _abi
    rank, world, local = dist_info()
    jobs, po, dtype_name, desc = rank_jobs(workload, rank, world, args.curves, args.log2n)
    prec = LC_FP64 if po else LC_FP32
    if not jobs:  # single: the other ranks idle through the barriers
        jobs = []
    if args.erdf is not None and not extra:
        jobs = [dict(j, **workloads.ERDF_SHAPES[args.erdf]) for j in jobs]
        desc += f"; ERDF shape {args.erdf} (tabulated CDF)"
    samples = workloads.total_samples(jobs)
    sample_iters = workloads.sample_iters(jobs)
    esize = 4 if prec == LC_FP32 else 8
    stream = torch.cuda.current_stream()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    plan = Plan(jobs, prec, device=local) if jobs else None
    if plan is not None and args.convergence is not None and not extra:
        plan.set_convergence([args.convergence] * len(jobs))
        desc += f"; with the Eq. 4 convergence test (threshold {args.convergence:g})"
    out = plan.empty() if plan is not None else None
    launches = [0]

    def step():
        if plan is not None:
            plan.generate(out=out, stream=stream)
            launches[0] += lc_plan_last_launches(plan.handle)

    for _ in range(warmup):
        step()
    launches[0] = 0
    with ClockSampler(local) as clk:
        ms = timed_steps(step, steps, barrier, CudaClock(stream))
    max_ms = reduce_over_ranks(ms, dist, "max")
    conv = None
    if plan is not None and args.convergence is not None and not extra:
        import numpy as np
        # throughput counts the iterations the curves actually ran
        d, run = plan.convergence()
        sample_iters = sum((1 << int(j["log2n"])) * int(r) for j, r in zip(jobs, run))
        conv = {"threshold": args.convergence, "mean_iters_run": float(np.mean(run)),
                "median_last_delta": float(np.median([d[c, int(r) - 1] for c, r in enumerate(run) if r > 0]))}
    total_si = reduce_over_ranks(sample_iters, dist, "sum")
    value = throughput(total_si, steps, max_ms)
    ms_per_step = max_ms / steps

    roof, post, e2e = None, None, None
    if plan is not None:
        # iteration-stage time of one more run (events on the library's stream)
        plan.generate(out=out, stream=stream)
        it_ms, setup_ms = lc_plan_timing(plan.handle)[1], lc_plan_timing(plan.handle)[0]
        peak, peak_kind = measured_peaks()
        alg_per = ALG_BYTES_PER_SAMPLE_ITER * (2 if prec != LC_FP32 else 1)
        stage_gbs = alg_per * sample_iters / (it_ms / 1000.0) / 1e9
        # the dominant kernel group, timed with CUDA events on the library's
        # stream in one extra iteration launched kernel by kernel
        prof = lc_plan_profile(plan.handle)
        groups = {g: prof[g] for g in ("sort_scatter", "resident", "fft", "sort_hist_scan")}
        dominant = max(groups, key=groups.get)
        if dominant == "resident":
            launches_k = 1
            per_launch_bytes = alg_per * prof["fused_elements"]
            kernel = "k_resident_cta / k_resident_cluster (one launch = one iteration of every fused curve)"
            kernel_bytes_def = f"{alg_per} B per sample-iteration of the fused curves"
        else:
            dominant = "sort_scatter"
            launches_k = max(1, prof["scatter_launches"])
            nb = prof.get("bucket_elements", 0)
            nr = prof["sorted_elements"] - nb
            # every element of a radix-sorted class goes through all passes; every
            # element of a sample-sorted class through the bucket scatter and finish
            per_launch_bytes = (SORT_BYTES_PER_ELEMENT[esize] * nr + BUCKET_SCATTER_BYTES_PER_ELEMENT * nb) / launches_k
            if nb and not nr:
                kernel = "k_bk_scatter + k_bk_finish (sample-sort argsort: bucket scatter and on-chip ranking)"
                kernel_bytes_def = f"{BUCKET_SCATTER_BYTES_PER_ELEMENT} B per element (scatter 13 + finish 16)"
            else:
                kernel = "k_sort_scatter (radix passes of the argsort)" + (" and the sample-sort scatter" if nb else "")
                kernel_bytes_def = (f"{SORT_BYTES_PER_ELEMENT[esize]} B per element per radix argsort (all passes), "
                                    f"{BUCKET_SCATTER_BYTES_PER_ELEMENT} B per sample-sorted element, "
                                    "split evenly over the scatter launches")
        avg_ms = prof[dominant] / launches_k
        achieved = per_launch_bytes / (avg_ms / 1000.0) / 1e9
        ktraffic = None
        if dominant == "sort_scatter" and esize == 4 and not prof.get("bucket_elements", 0):
            ktraffic = SCATTER_DRAM_BYTES_PER_ELEMENT_FP32 * prof["sorted_elements"] / launches_k
        traffic, last_capture = None, None
        if workload == "uniform" and (args.curves, args.log2n) == (NCURVES, LOG2N) and ITER_DRAM_BYTES_PER_SAMPLE:
            if ITER_DRAM_CAPTURE_CURRENT:
                traffic = ITER_DRAM_BYTES_PER_SAMPLE * samples
            last_capture = {"dram_bytes_per_sample_iter": ITER_DRAM_BYTES_PER_SAMPLE,
                            "of": "every kernel of one iteration, 512 curves x 2^16, before the finish kernel's "
                                  "launched-slot change"}
        # The roofline unit is one amplitude-adjustment iteration of every curve
        # (one replay of the iteration graph): 14 B per sample-iteration (28 B in
        # FP64) over the iteration stage's CUDA-event time.  The dominant kernel's
        # figure against its own algorithmic bytes is kept beside it.
        n_iter = max(1, max(int(j["iters"]) for j in jobs))
        roof = {"bound": "hbm", "achieved": stage_gbs, "peak": peak, "unit": "GB/s", "frac": stage_gbs / peak,
                "traffic": traffic, "traffic_last_capture": last_capture,
                "kernel": "iteration stage: every kernel of one E13 iteration of every curve (one graph replay)",
                "alg_bytes_per_sample_iter": alg_per, "alg_bytes_per_launch": alg_per * sample_iters / n_iter,
                "launch_ms": it_ms / n_iter, "iterate_ms": it_ms, "peak_kind": peak_kind,
                "dominant_kernel": {"kernel": kernel, "achieved": achieved, "kernel_frac": achieved / peak,
                                    "launch_ms": avg_ms, "alg_bytes_per_launch": per_launch_bytes,
                                    "traffic": ktraffic, "alg_bytes_definition": kernel_bytes_def},
                "group_ms_one_iteration": {g: prof[g] for g in groups},
                "scheduled_bytes_per_sample_iter": scheduled_bytes_per_sample_iter(jobs, esize,
                                                                                   prof["fused_elements"]),
                "setup_ms": setup_ms}

        if args.post and not extra:
            import numpy as np
            from paper_1909_06374_gb300 import lc_periodogram, lc_structure_function
            lags = np.unique(np.logspace(0, np.log2(min(1 << int(j["log2n"]) for j in jobs) - 1), 64,
                                         base=2).astype(np.uint32))
            nh = sum((1 << int(j["log2n"])) // 2 + 1 for j in jobs)
            pbuf = torch.empty(nh, dtype=torch.float64, device="cuda")
            sbuf = torch.empty((len(jobs), lags.size), dtype=torch.float64, device="cuda")
            for _ in range(2):
                lc_periodogram(plan.handle, out, False, pbuf, stream)
                lc_structure_function(plan.handle, out, lags, sbuf, stream)
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            reps = 5
            e0.record(stream)
            for _ in range(reps):
                lc_periodogram(plan.handle, out, False, pbuf, stream)
            e1.record(stream)
            for _ in range(reps):
                lc_structure_function(plan.handle, out, lags, sbuf, stream)
            e2.record(stream)
            torch.cuda.synchronize()
            pm, sm = e0.elapsed_time(e1) / reps, e1.elapsed_time(e2) / reps
            # algorithmic bytes: the series read once (and the spectrum written) / once per lag
            pb = samples * esize + nh * 8
            sb = samples * esize * lags.size
            post = {"periodogram_ms": pm, "periodogram_gbs": pb / (pm / 1e3) / 1e9,
                    "sf_ms": sm, "sf_lags": int(lags.size), "sf_gbs_one_read_per_lag": sb / (sm / 1e3) / 1e9,
                    "sf_pair_terms_per_s": float(sum(((1 << int(j["log2n"])) - int(l)) for j in jobs for l in lags))
                    / (sm / 1e3)}

    # end-to-end through the host entry point: job table in, series out
    if e2e_on and args.convergence is None:
        host = torch.empty(max(samples, 1), dtype=torch.float32 if prec == LC_FP32 else torch.float64).pin_memory()
        jb = _abi.job_array(jobs) if jobs else None
        h2d = len(jobs) * _abi.ctypes.sizeof(_abi.LcJob)
        e2e_steps = max(1, min(steps, 2))

        def e2e_step():
            if jobs:
                h = lc_plan_create(jb, prec, local)
                lc_generate_host(h, host, None, stream)
                lc_plan_destroy(h)

        dt_ms = timed_steps(e2e_step, e2e_steps, barrier, HostClock())
        e2e = {"value": throughput(total_si, e2e_steps, reduce_over_ranks(dt_ms, dist, "max")), "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": samples * esize,
               "what": "lc_plan_create (job table upload) + lc_generate_host (pinned output) + lc_plan_destroy"}

    cpu = None
    if rank == 0 and cpu_on and args.erdf is None and args.convergence is None:
        cores = os.cpu_count() or 1
        if workload == "uniform":
            v, used, dt = cpu_baseline_run(cores, ITERS, cores)
            sample = f"{cores} curves x 2^{LOG2N} samples x {ITERS} iterations (one curve per thread, {dt:.1f} s)"
        else:
            cjobs, cprec, sample = cpu_baseline_sample(workload, cores)
            v, used, dt = cpu_baseline_run(0, 0, cores, jobs=cjobs, prec=cprec)
            sample += f" ({dt:.1f} s)"
        cpu = {"value": v, "unit": UNIT, "cores": used, "kind": "oracle", "sample": sample}

    if plan is not None:
        plan.close()
    if rank != 0:
        return None
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
            "warmup": warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak" if workload == "uniform" else "strong", "vs_baseline": None,
            "dtype": dtype_name, "data": "synthetic",
            "config": {"workload": desc, "curves_per_gpu": len(jobs), "samples_per_gpu": samples,
                       "sample_iters_per_gpu": sample_iters,
                       "l2": ("inputs larger than L2" if samples * esize * 3 > 129e6 else
                              "working set inside L2 (latency workload)"),
                       "parallelism": (f"curves sharded over {world} GPU(s), no collective"
                                       if world > 1 or workload != "single" else "one curve on one GPU")},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches[0],
            "clocks": clk.summary()}
    if extra:
        line["line"] = f"additional workload: {workload}"
    if conv is not None:
        line["convergence"] = conv
    if post is not None:
        line["postproc"] = post
    return line


def run_gpu(args):
    import torch
    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    line = gpu_line(args, args.workload, args.steps, args.warmup, dist, e2e_on=not args.no_e2e,
                    cpu_on=not args.no_cpu_baseline)
    if rank == 0:
        print(json.dumps(line), flush=True)
    extras = (world == 1 and args.workload == "uniform" and not args.headline_only and args.erdf is None
              and args.convergence is None and not args.post and (args.curves, args.log2n) == (NCURVES, LOG2N))
    if extras:
        # the other workloads, one line each, after the headline: the
        # single-curve latency (FP64), the long curves and the ragged batch
        for w, k in (("single", max(3, min(args.steps, 20))), ("long", 3), ("ragged", 2)):
            print(json.dumps(gpu_line(args, w, k, 3, None, e2e_on=False, cpu_on=not args.no_cpu_baseline,
                                      extra=True)), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    if extras:
        # serving: the named 200 req/s stream, and 50 req/s (a load the server sustains)
        for rate in (200.0, 50.0):
            print(json.dumps(serving_line(args, rate)), flush=True)
    return 0


# ------------------------------------------------------------------ serving
def serving_line(args, rate):
    """Poisson request stream replayed in real time against (a) the
    continuous-batching server and (b) the plain path that runs one job at a
    time (plan, generate to host, destroy) in arrival order."""
    import numpy as np
    import torch
    from paper_1909_06374_gb300 import (LC_FP32, lc_generate_host, lc_plan_create, lc_plan_destroy, lc_poll,
                                        lc_server_create, lc_server_destroy, lc_submit)
    from paper_1909_06374_gb300 import _abi
    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    stream = workloads.serving_stream(rate=rate, duration=args.serving_seconds)
    total_si = sum((1 << j["log2n"]) * j["iters"] for _, j in stream)
    cap = 2.0 * args.serving_seconds + 60.0

    def summarize(lat, done_si, makespan, unfinished):
        lat = np.array(lat) if lat else np.array([np.nan])
        return {"throughput": done_si / makespan, "unit": UNIT, "p50_ms": float(np.percentile(lat, 50)),
                "p99_ms": float(np.percentile(lat, 99)), "finished": int(len(lat) - np.isnan(lat).sum()),
                "unfinished": unfinished, "makespan_s": makespan}

    with ClockSampler(local) as clk:
        # (a) server
        server = lc_server_create(local, 0, LC_FP32)
        big = np.empty(1 << 24, dtype=np.float32)
        lat, pending = [], {}
        t0 = time.perf_counter()
        i = 0
        done_si = 0
        while True:
            now = time.perf_counter() - t0
            while i < len(stream) and stream[i][0] <= now:
                t, j = stream[i]
                tk = lc_submit(server, j)
                pending[tk] = (j, t)
                i += 1
            for tk in list(pending):
                j, t = pending[tk]
                st, ns = lc_poll(server, tk, big)
                if st == _abi.LC_OK:
                    lat.append(ns / 1e6)
                    done_si += (1 << j["log2n"]) * j["iters"]
                    del pending[tk]
            if i >= len(stream) and not pending:
                break
            if now > cap:
                break
            time.sleep(0.0005)
        makespan = time.perf_counter() - t0
        lc_server_destroy(server)
        srv = summarize(lat, done_si, makespan, len(pending) + len(stream) - i)

        # (b) plain path, same stream, one job at a time
        host = torch.empty(1 << 24, dtype=torch.float32).pin_memory()
        lat2, done2 = [], 0
        t0 = time.perf_counter()
        k = 0
        for t, j in stream:
            now = time.perf_counter() - t0
            if now > cap:
                break
            if now < t:
                time.sleep(t - now)
            h = lc_plan_create([j], LC_FP32, local)
            lc_generate_host(h, host)
            lc_plan_destroy(h)
            lat2.append((time.perf_counter() - t0 - t) * 1e3)
            done2 += (1 << j["log2n"]) * j["iters"]
            k += 1
        makespan2 = time.perf_counter() - t0
        plain = summarize(lat2, done2, makespan2, len(stream) - k)
    offered = total_si / args.serving_seconds
    return {"metric": "serving: light-curve samples x E13 iterations per second; p50/p99 latency",
            "value": srv["throughput"], "unit": UNIT, "n_gpus": 1, "higher_is_better": True, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"Poisson {rate:g} req/s for {args.serving_seconds:g} s, "
                                   "N log-uniform 2^12..2^24, iterations 20..200, per-job PSD/ERDF",
                       "jobs": len(stream), "offered_sample_iters_per_s": offered},
            "server": srv, "plain_one_job_at_a_time": plain,
            "server_saturated": srv["unfinished"] > 0 or srv["throughput"] < 0.95 * offered,
            "clocks": clk.summary()}


def run_serving(args):
    rank, world, local = dist_info()
    if rank != 0:
        return 0
    print(json.dumps(serving_line(args, args.serving_rate)), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "serving":
        return run_serving(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
