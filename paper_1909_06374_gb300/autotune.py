"""Autotuning sweep of the iteration path per curve length.

Two complete iteration paths exist for FP32 curves of 2^10..2^16 samples: the
fused on-chip kernels (one CTA per curve up to 2^14, clusters of 2 and 4 CTAs
at 2^15 and 2^16) and the multi-kernel path (tile FFT passes + the sample-sort
or radix argsort through HBM).  Which is faster depends on the length and on the GPU.
For every length in the range this sweep runs a uniform batch of about
2^samples samples for `iters` iterations on each path, timed with CUDA events
around the iteration stage (lc_plan_timing), and reports the crossover: the
longest length up to which the fused kernels win at every length.  The
library's auto mode uses the crossover measured on GB300 (2^12); the
environment variable LC_RESIDENT_MAX_LOG2 applies another one (read when a
plan is created).  Results depend on the length, the precision and the path,
so a different crossover changes the bits of the affected lengths (both paths
stay within the same tolerances of the FP64 oracle).

    python -m paper_1909_06374_gb300.autotune [--lengths 10:16] [--samples 26] [--iters 20] [--out FILE]
"""
from __future__ import annotations

import argparse
import json
import os
import sys


def crossover(table, lo=10):
    """Longest log2 length L >= lo such that the fused path is faster at every
    measured length from lo to L; lo - 1 when it loses at lo.  `table` maps L
    to {"resident": throughput, "multi": throughput} (higher is faster)."""
    best = lo - 1
    for L in sorted(table):
        if L < lo:
            continue
        row = table[L]
        if row.get("resident") is None or row["resident"] <= row["multi"]:
            break
        best = L
    return best


def measure(log2n, path, samples=26, iters=20, device=0):
    """sample*iter/s of the iteration stage of a uniform batch on one path."""
    from paper_1909_06374_gb300 import LC_FP32, Plan, lc_plan_timing, workloads
    ncurves = max(1, (1 << samples) >> log2n)
    jobs = workloads.uniform(ncurves=ncurves, log2n=log2n, iters=iters)
    old = os.environ.get("LC_PATH")
    os.environ["LC_PATH"] = path  # read when the plan is created
    try:
        with Plan(jobs, LC_FP32, device=device) as p:
            p.generate()  # warm-up: graph capture, first-touch of the arena
            p.generate()
            _, it_ms = lc_plan_timing(p.handle)
    finally:
        if old is None:
            os.environ.pop("LC_PATH", None)
        else:
            os.environ["LC_PATH"] = old
    return ncurves * (1 << log2n) * iters / (it_ms / 1e3)


def sweep(lengths=range(10, 17), samples=26, iters=20, device=0):
    table = {}
    for L in lengths:
        table[L] = {"resident": measure(L, "resident", samples, iters, device) if 10 <= L <= 16 else None,
                    "multi": measure(L, "multi", samples, iters, device)}
    return table


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--lengths", default="10:16", help="log2 lengths, lo:hi inclusive")
    ap.add_argument("--samples", type=int, default=26, help="log2 of the samples per batch")
    ap.add_argument("--iters", type=int, default=20)
    ap.add_argument("--device", type=int, default=0)
    ap.add_argument("--out", default=None, help="write the table and the crossover as JSON")
    a = ap.parse_args(argv)
    lo, hi = (int(v) for v in a.lengths.split(":"))
    table = sweep(range(lo, hi + 1), a.samples, a.iters, a.device)
    x = crossover(table, lo=max(lo, 10))
    print("| log2 N | fused kernels | multi-kernel path | faster |")
    print("|---|---|---|---|")
    for L, row in sorted(table.items()):
        r = row["resident"]
        faster = "fused" if r is not None and r > row["multi"] else "multi-kernel"
        print(f"| {L} | {'-' if r is None else f'{r:.3g}'} | {row['multi']:.3g} | {faster} |")
    print(f"crossover: LC_RESIDENT_MAX_LOG2={x}")
    if a.out:
        with open(a.out, "w") as f:
            json.dump({"table": {str(k): v for k, v in table.items()}, "resident_max_log2": x,
                       "samples_log2": a.samples, "iters": a.iters}, f, indent=1)
    return 0


if __name__ == "__main__":
    sys.exit(main())
