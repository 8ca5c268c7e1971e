"""Seeded synthetic workloads (job parameter lists) for the light-curve generator.

This module holds no arithmetic of the method: it only draws the per-curve
parameters (lengths, PSD break and slopes, ERDF break and slopes, seeds,
iteration counts, arrival times) that both the CUDA library and the CPU oracle
receive as inputs.  The random numbers that the method itself uses (TK95
Gaussians and ERDF uniforms) are generated inside each side from Philox
counters keyed by (seed, curve_id).

Workloads (all lengths are powers of two, Sec. 3.2.3; dt in days):
  single   1 curve,  N = 2^14, FP64, 100 iterations, seed 1
  uniform  4096 curves, N = 2^16, FP32, 200 iterations, seed = curve_id = 0..4095
  long     8 curves, N = 2^26, dt = 7 d, per-curve f_br and high slope, 50 iterations
  ragged   10000 curves, N log-uniform over 2^10..2^20, per-curve PSD and ERDF, 100 iterations
  serving  Poisson arrivals at 200/s for 60 s, N log-uniform over 2^12..2^24,
           iterations uniform in 20..200

Base PSD (Eq. 3): f_br = 1/300 d^-1, alpha_low = 1, alpha_high = 2.
Base ERDF (sharp broken power law in log10 lambda): [-4, 0], break -1.5,
slopes +0.4 below and -2.5 above (dN/dlog10 lambda ~ lambda^slope).

ERDF shapes printed in the paper (Sec. 2.1.1, Sec. 4.1 Table 2), as job
parameter overrides (ERDF_SHAPES):
  smooth_eq1  Eq. 1 with W17's log lambda* = -1.84, delta 0.47 / 2.53, on the
              range W17 probes, log lambda in [-4, 1]
  table2      Eq. 1 as in the reference setup of Table 2: lambda* = 0.11,
              delta 0.47 / 2.53, log lambda in [-3.75, 0.5]
  lognormal   Eq. 2 with log lambda* = -3.25, sigma = 0.64, on [-4, 1]
"""
from __future__ import annotations

import numpy as np

BASE = dict(dt=1.0, f_br=1.0 / 300.0, alpha_low=1.0, alpha_high=2.0,
            log_lmin=-4.0, log_lmax=0.0, log_lbreak=-1.5, slope_low=0.4, slope_high=-2.5,
            linear_space=0, erdf_kind=0, sigma=0.0, tk_coeffs=0, tk_targets=0)

ERDF_SHAPES = {
    "smooth_eq1": dict(erdf_kind=1, log_lmin=-4.0, log_lmax=1.0, log_lbreak=-1.84,
                       slope_low=-0.47, slope_high=-2.53),
    "table2": dict(erdf_kind=1, log_lmin=-3.75, log_lmax=0.5, log_lbreak=float(np.log10(0.11)),
                   slope_low=-0.47, slope_high=-2.53),
    "lognormal": dict(erdf_kind=2, log_lmin=-4.0, log_lmax=1.0, log_lbreak=-3.25, sigma=0.64,
                      slope_low=0.0, slope_high=0.0),
}


def job(log2n, iters, seed, curve_id, **over):
    j = dict(BASE)
    j.update(log2n=int(log2n), iters=int(iters), seed=int(seed), curve_id=int(curve_id))
    j.update(over)
    return j


def single(iters=100):
    """1 curve of 2^14 samples (computed in FP64)."""
    return [job(14, iters, seed=1, curve_id=0)]


def uniform(ncurves=4096, log2n=16, iters=200):
    """A uniform batch; seed = curve_id = curve index."""
    return [job(log2n, iters, seed=c, curve_id=c) for c in range(ncurves)]


def _loguniform(rng, lo, hi, size=None):
    return np.exp(rng.uniform(np.log(lo), np.log(hi), size))


def long_curves(ncurves=8, log2n=26, iters=50, master_seed=2):
    """Long curves at 7-day cadence; f_br log-uniform in [1e-4, 1e-1] d^-1 and the
    high-frequency slope uniform in [2, 3] (the PSD of Eq. 3 falls as f^-alpha)."""
    rng = np.random.default_rng(master_seed)
    out = []
    for c in range(ncurves):
        out.append(job(log2n, iters, seed=c, curve_id=c, dt=7.0,
                       f_br=float(_loguniform(rng, 1e-4, 1e-1)),
                       alpha_high=float(rng.uniform(2.0, 3.0))))
    return out


def ragged(ncurves=10000, lo=10, hi=20, iters=100, master_seed=3):
    """Curves of uneven length: log2 N uniform over lo..hi (log-uniform N), per-curve
    PSD (f_br, high slope) and ERDF (break in [-2.5, -0.5], high slope in [-3, -1.5])."""
    rng = np.random.default_rng(master_seed)
    out = []
    for c in range(ncurves):
        out.append(job(int(rng.integers(lo, hi + 1)), iters, seed=c, curve_id=c,
                       f_br=float(_loguniform(rng, 1e-4, 1e-1)),
                       alpha_high=float(rng.uniform(2.0, 3.0)),
                       log_lbreak=float(rng.uniform(-2.5, -0.5)),
                       slope_high=float(rng.uniform(-3.0, -1.5))))
    return out


def serving_stream(rate=200.0, duration=60.0, lo=12, hi=24, it_lo=20, it_hi=200,
                   master_seed=4):
    """Poisson request stream: list of (arrival_time_s, job)."""
    rng = np.random.default_rng(master_seed)
    t = 0.0
    out = []
    c = 0
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t >= duration:
            break
        out.append((t, job(int(rng.integers(lo, hi + 1)), int(rng.integers(it_lo, it_hi + 1)),
                           seed=c, curve_id=c,
                           f_br=float(_loguniform(rng, 1e-4, 1e-1)),
                           alpha_high=float(rng.uniform(2.0, 3.0)),
                           log_lbreak=float(rng.uniform(-2.5, -0.5)),
                           slope_high=float(rng.uniform(-3.0, -1.5)))))
        c += 1
    return out


def total_samples(jobs):
    return sum(1 << j["log2n"] for j in jobs)


def sample_iters(jobs):
    return sum((1 << j["log2n"]) * j["iters"] for j in jobs)


def shard_jobs(jobs, world):
    """Split a job list over `world` ranks, balancing the work sum N * iters
    (longest-processing-time greedy).  Curves are independent, so ranks never
    exchange data; every job lands on exactly one rank, in its original order."""
    loads = [0] * world
    owner = [0] * len(jobs)
    order = sorted(range(len(jobs)), key=lambda i: -((1 << jobs[i]["log2n"]) * max(1, jobs[i]["iters"])))
    for i in order:
        r = min(range(world), key=lambda q: loads[q])
        owner[i] = r
        loads[r] += (1 << jobs[i]["log2n"]) * max(1, jobs[i]["iters"])
    return [[jobs[i] for i in range(len(jobs)) if owner[i] == r] for r in range(world)]
