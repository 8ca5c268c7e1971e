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
WORKLOAD = (f"uniform batch: {NCURVES} curves x 2^{LOG2N} samples, dt=1 d, bending PL PSD "
            f"(f_br=1/300 d^-1, slopes 1/2), broken-PL ERDF [-4,0] break -1.5 slopes +0.4/-2.5, "
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
    return ap.parse_args()


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def jobs_for_rank(rank, ncurves=NCURVES):
    jobs = workloads.uniform(ncurves=ncurves, log2n=LOG2N, iters=ITERS)
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
def cpu_baseline_run(ncurves, iters, cores):
    """The FP64 CPU oracle on `ncurves` curves of the workload (`iters`
    iterations each), one curve per host thread; returns samples*iter/s."""
    import oracle
    oracle.build()
    jobs = workloads.uniform(ncurves=ncurves, log2n=LOG2N, iters=iters)
    t0 = time.perf_counter()
    _, used = oracle.generate_batch(jobs, prec=0, nthreads=cores)
    dt = time.perf_counter() - t0
    return ncurves * (1 << LOG2N) * iters / dt, used, dt


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
def run_gpu(args):
    import torch
    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1909_06374_gb300 import LC_FP32, Plan, lc_generate_host, lc_plan_create, lc_plan_destroy, \
        lc_plan_last_launches, lc_plan_timing
    from paper_1909_06374_gb300 import _abi

    jobs = jobs_for_rank(rank, args.curves)
    samples = args.curves << LOG2N
    sample_iters = samples * ITERS
    plan = Plan(jobs, LC_FP32, device=local)
    out = plan.empty()
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        plan.generate(out=out, stream=stream)
    torch.cuda.synchronize()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches = 0
    iter_ms = []
    barrier()
    with ClockSampler(local) as clk:
        start.record(stream)
        for _ in range(args.steps):
            plan.generate(out=out, stream=stream)
            launches += lc_plan_last_launches(plan.handle)
        end.record(stream)
        barrier()
    total_ms = start.elapsed_time(end)
    # iteration-stage time of each step (events on the library's stream)
    for _ in range(1):
        plan.generate(out=out, stream=stream)
        iter_ms.append(lc_plan_timing(plan.handle)[1])
    t = torch.tensor([total_ms], dtype=torch.float64, device="cuda")
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    max_ms = float(t.item())
    ms_per_step = max_ms / args.steps
    value = world * sample_iters * args.steps / (max_ms / 1000.0)

    # end-to-end through the host entry point: job table in, series out
    e2e = None
    if not args.no_e2e:
        host = torch.empty(samples, dtype=torch.float32).pin_memory()
        jb = _abi.job_array(jobs)
        h2d = len(jobs) * _abi.ctypes.sizeof(_abi.LcJob)
        barrier()
        t0 = time.perf_counter()
        e2e_steps = max(1, min(args.steps, 2))
        for _ in range(e2e_steps):
            h = lc_plan_create(jb, LC_FP32, local)
            lc_generate_host(h, host, None, stream)
            lc_plan_destroy(h)
        barrier()
        dt = time.perf_counter() - t0
        te = torch.tensor([dt], dtype=torch.float64, device="cuda")
        if dist is not None:
            dist.all_reduce(te, op=dist.ReduceOp.MAX)
        e2e = {"value": world * sample_iters * e2e_steps / float(te.item()), "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": samples * 4,
               "what": "lc_plan_create (job table upload) + lc_generate_host (pinned output) + lc_plan_destroy"}

    peak, peak_kind = measured_peaks()
    it_ms = statistics.median(iter_ms)
    alg_bytes = ALG_BYTES_PER_SAMPLE_ITER * sample_iters
    achieved = alg_bytes / (it_ms / 1000.0) / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": None, "kernel": "iteration stage (all E13 iterations of the batch)",
            "peak_kind": peak_kind, "alg_bytes_per_sample_iter": ALG_BYTES_PER_SAMPLE_ITER,
            "iterate_ms": it_ms}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        v, used, dt = cpu_baseline_run(cores, ITERS, cores)
        cpu = {"value": v, "unit": UNIT, "cores": used, "kind": "oracle",
               "sample": f"{cores} curves x 2^{LOG2N} samples x {ITERS} iterations (one curve per thread, "
                         f"{dt:.1f} s)"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD if args.curves == NCURVES else
                           f"PROFILING CASE ({args.curves} curves), not the bench workload", "curves_per_gpu": args.curves, "log2n": LOG2N, "iters": ITERS,
                           "l2": "inputs larger than L2 (per-iteration working set > 2.5 GB)",
                           "parallelism": f"curves sharded over {world} GPU(s), no collective"},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    plan.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
