"""Comparison rules between the CUDA path and the FP64 oracle.

Per position (the acceptance rule): the GPU's value at position k must be
the oracle's, unless the oracle's pre-ranking values (x_adj of the last
iteration) at the oracle's rank of k and at the rank the GPU's value implies
differ by less than `tie_rel` times rms(x_adj) (a near tie that FP32 FFT
rounding may legitimately flip).
"""
from __future__ import annotations

import numpy as np


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def position_check(gpu_x, oracle_x, s_sorted, xadj_oracle, tie_rel=1e-5):
    """Returns dict(mismatch, exempt, fail, not_in_draws, n)."""
    g = np.asarray(gpu_x, dtype=np.float64)
    o = np.asarray(oracle_x, dtype=np.float64)
    s = np.asarray(s_sorted, dtype=np.float64)
    xa = np.asarray(xadj_oracle, dtype=np.float64)
    n = g.size
    rms = float(np.sqrt(np.mean(xa ** 2)))
    order = np.argsort(xa, kind="stable")
    rank_or = np.empty(n, dtype=np.int64)
    rank_or[order] = np.arange(n)
    xs = xa[order]
    lo = np.searchsorted(s, g, side="left")
    hi = np.searchsorted(s, g, side="right") - 1
    not_in = lo > hi
    same = (g == o)
    mism = ~same
    r_g = np.clip(rank_or, lo, np.maximum(hi, lo))
    r_g = np.clip(r_g, 0, n - 1)
    gap = np.abs(xs[r_g] - xs[rank_or])
    exempt = mism & ~not_in & (gap < tie_rel * rms)
    fail = mism & ~exempt
    return dict(n=n, mismatch=int(mism.sum()), exempt=int(exempt.sum()), fail=int(fail.sum()),
                not_in_draws=int(not_in.sum()))


def rank_stats(gpu_x, oracle_x):
    """Rank displacement statistics between two permutations of the same values."""
    g = np.asarray(gpu_x, dtype=np.float64)
    o = np.asarray(oracle_x, dtype=np.float64)
    n = g.size
    rg = np.empty(n); rg[np.argsort(g, kind="stable")] = np.arange(n)
    ro = np.empty(n); ro[np.argsort(o, kind="stable")] = np.arange(n)
    d = np.abs(rg - ro)
    rho = float(np.corrcoef(rg, ro)[0, 1]) if n > 1 else 1.0
    return dict(mismatch_frac=float(np.mean(g != o)), median_disp=float(np.median(d)),
                max_disp=float(d.max()), spearman=rho)
