"""The rank-order replacement step (Sec. 2.1 third step, Sec. 3.2.2) on its
own, through the C ABI: out[perm[r]] = s[r] with perm the stable argsort of the
given values, against the oracle's argsort, bit for bit (integer index work).

The values are chosen to hit every branch of both sort paths: the sample sort
of FP32 curves of 2^13..2^20 samples (splitters from a sample of 1024 or 4096
values, buckets, groups of up to 2048, 4096 or 8192 elements ranked in shared
memory, oversize buckets sorted by block radix passes) and the LSD radix
passes of the other lengths and of FP64."""
import numpy as np
import pytest

import oracle
from paper_1909_06374_gb300 import LC_FP32, LC_FP64, Plan, workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _patterns(n, rng):
    """Value patterns of length n (float64; cast to the plan's precision)."""
    i = np.arange(n)
    return {
        "normal": rng.standard_normal(n),
        "lognormal_shifted": np.exp(2.0 * rng.standard_normal(n)) - 3.0,
        "all_equal": np.full(n, 0.25),
        "signed_zeros": np.where(rng.random(n) < 0.5, -0.0, 0.0),
        "spike_30pct": np.where(rng.random(n) < 0.3, 1.0, rng.standard_normal(n)),
        "spike_90pct_zero": np.where(rng.random(n) < 0.9, 0.0, rng.standard_normal(n)),
        "integer_ties": rng.integers(0, 50, n).astype(np.float64),
        "ascending": i.astype(np.float64),
        "descending": -i.astype(np.float64),
        "tiny": rng.standard_normal(n) * 1e-30,
        "huge_and_denormal": np.where(rng.random(n) < 0.5, rng.standard_normal(n) * 1e30,
                                      rng.standard_normal(n) * 1e-42),
        "two_clusters": np.where(rng.random(n) < 0.5, 1e6, -1e6) + rng.standard_normal(n),
    }


def _check(prec, log2ns, seed):
    rng = np.random.default_rng(seed)
    jobs = [workloads.job(l, 1, seed=100 + c, curve_id=c) for c, l in enumerate(log2ns)]
    dt = np.float32 if prec == LC_FP32 else np.float64
    with Plan(jobs, prec) as p:
        p.setup()
        s = p.buffer(2).cpu().numpy()
        pats = {}
        for c, j in enumerate(jobs):
            for name, v in _patterns(1 << j["log2n"], rng).items():
                pats.setdefault(name, []).append(v.astype(dt))
        for name, parts in pats.items():
            xa = np.concatenate(parts)
            got = p.rank_replace(torch.tensor(xa, device="cuda")).cpu().numpy()
            for c in range(len(jobs)):
                seg = slice(p.offsets[c], p.offsets[c + 1])
                perm = oracle.argsort(xa[seg].astype(np.float64))  # stable; -0 == +0
                want = np.empty_like(s[seg])
                want[perm] = s[seg]
                assert np.array_equal(got[seg], want), (name, prec, jobs[c]["log2n"])


def test_rank_replace_fp32_sample_sort_lengths():
    _check(LC_FP32, [13, 14, 15, 16, 17], seed=1)


def test_rank_replace_fp32_long_sample_sort_lengths():
    _check(LC_FP32, [18, 19, 20], seed=5)


def test_rank_replace_fp32_radix_lengths():
    _check(LC_FP32, [4, 9, 12, 21], seed=2)


def test_rank_replace_fp64():
    _check(LC_FP64, [9, 13, 16], seed=3)


def test_rank_replace_radix_override_agrees(monkeypatch):
    """LC_SORT=radix keeps the LSD passes at every length: the same output."""
    rng = np.random.default_rng(4)
    jobs = [workloads.job(16, 1, seed=7, curve_id=0), workloads.job(15, 1, seed=8, curve_id=1),
            workloads.job(19, 1, seed=9, curve_id=2)]
    xa = torch.tensor(np.concatenate([rng.standard_normal(1 << 16), np.exp(rng.standard_normal(1 << 15)),
                                      rng.standard_normal(1 << 19) ** 3]),
                      dtype=torch.float32, device="cuda")
    with Plan(jobs, LC_FP32) as p:
        p.setup()
        a = p.rank_replace(xa).cpu().numpy()
    monkeypatch.setenv("LC_SORT", "radix")
    with Plan(jobs, LC_FP32) as q:
        q.setup()
        b = q.rank_replace(xa).cpu().numpy()
    assert np.array_equal(a, b)
