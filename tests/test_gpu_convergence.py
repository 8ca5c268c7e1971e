"""Convergence test of Sec. 3.2.2 (Eq. 4) on the CUDA path, through the C ABI.

delta_i = rms_n log10(x_i / x_{i-1}) is checked three ways: against the
oracle's Eq. 4 applied to the GPU's own consecutive iterates (the reduction
itself, 1e-5 relative: FP32 logs and per-thread FP32 sums of at most 32
squares, FP64 beyond); against the oracle's own iteration (end to end, 1e-3
relative, which leaves room for near-tie rank flips); and through the stopping
rule (strict threshold, per curve, bit-identical to a plain run of that many
iterations).  Every iteration path is covered: the fused single-CTA kernel
(2^10..2^14), the cluster kernel (2^15 under the default table, 2^16 when
forced), the multi-kernel path (2^8, 2^16, 2^17, FP64, and forced at 2^12).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1909_06374_gb300 import LC_FP32, LC_FP64, LcError, Plan, workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEF_TOL = 1e-5    # GPU delta vs Eq. 4 on the GPU's own iterates
E2E_TOL = 1e-3    # GPU delta vs the oracle's own iteration


def _np(t):
    return t.detach().cpu().numpy().astype(np.float64)


def _jobs(log2ns, iters, seed=21):
    return [workloads.job(l, iters, seed=seed + i, curve_id=i) for i, l in enumerate(log2ns)]


CASES = {
    # name: (log2n list, precision, LC_PATH)
    "auto_fp32": ([8, 10, 12, 14, 15, 16, 17], LC_FP32, None),
    "auto_fp64": ([9, 12, 15], LC_FP64, None),
    "forced_multi": ([12, 14], LC_FP32, "multi"),
    "forced_resident": ([16, 15, 13], LC_FP32, "resident"),
}


def _env(monkeypatch, path):
    if path:
        monkeypatch.setenv("LC_PATH", path)
    else:
        monkeypatch.delenv("LC_PATH", raising=False)


@pytest.mark.parametrize("name", list(CASES))
def test_delta_is_eq4_of_consecutive_iterates(name, monkeypatch):
    log2ns, prec, path = CASES[name]
    _env(monkeypatch, path)
    jobs = _jobs(log2ns, 3)
    with Plan(jobs, prec) as p:
        p.set_convergence(None, history=4)
        p.setup()
        for step in range(3):
            prev = _np(p.get_state())
            p.iterate(1)
            cur = _np(p.get_state())
            d, run = p.convergence()
            assert np.all(run == 1), (name, step, run)
            assert np.all(np.isnan(d[:, 1:]))
            for c in range(len(jobs)):
                seg = slice(p.offsets[c], p.offsets[c + 1])
                want = oracle.delta(prev[seg], cur[seg])
                got = d[c, 0]
                assert want > 0
                assert abs(got - want) <= DEF_TOL * want, (name, step, c, got, want)


@pytest.mark.parametrize("name", list(CASES))
def test_delta_sequence_matches_oracle_iteration(name, monkeypatch):
    """Both sides iterate from the draws; the GPU's delta_1..delta_K follow the
    oracle's, and turning the test on does not change the series."""
    log2ns, prec, path = CASES[name]
    _env(monkeypatch, path)
    K = 5
    jobs = _jobs(log2ns, K)
    po = 0 if prec == LC_FP32 else 1
    with Plan(jobs, prec) as p:
        plain = _np(p.generate())
        p.set_convergence(None, history=K + 2)
        with_test = _np(p.generate())
        d, run = p.convergence()
    assert np.array_equal(plain, with_test), name
    assert np.all(run == K)
    assert np.all(np.isnan(d[:, K:]))
    for c, j in enumerate(jobs):
        r = oracle.generate(dict(j, iters=0), prec=po, want=("x", "A", "s"))
        _, want, n_run = oracle.iterate_conv(r["A"], r["s"], r["x"], K, 0.0)
        assert n_run == K
        np.testing.assert_allclose(d[c, :K], want, rtol=E2E_TOL, err_msg=f"{name} curve {c}")


def _first_new_minimum(d):
    for i in range(1, d.size):
        if d[i] < d[:i].min():
            return i
    return None


@pytest.mark.parametrize("name", list(CASES))
def test_threshold_stops_each_curve_at_its_first_crossing(name, monkeypatch):
    log2ns, prec, path = CASES[name]
    _env(monkeypatch, path)
    K = 8
    jobs = _jobs(log2ns, K)
    with Plan(jobs, prec) as p:
        p.set_convergence(None, history=K)
        p.generate()
        D, _ = p.convergence()
    # curve 0 never stops (threshold 0); the others stop after their first new minimum
    thr = np.zeros(len(jobs))
    stop_at = np.full(len(jobs), K)
    for c in range(1, len(jobs)):
        k = _first_new_minimum(D[c])
        if k is not None:
            thr[c] = float(np.nextafter(D[c, k], np.inf))
            stop_at[c] = k + 1
    with Plan(jobs, prec) as p:
        p.set_convergence(thr, history=K)
        x = _np(p.generate())
        d, run = p.convergence()
    assert np.array_equal(run, stop_at.astype(np.uint32)), (run, stop_at)
    for c in range(len(jobs)):
        assert np.array_equal(d[c, :stop_at[c]], D[c, :stop_at[c]]), (name, c)
        assert np.all(np.isnan(d[c, stop_at[c]:]))
    # the stopped series are the plain series of that many iterations
    short = [dict(j, iters=int(stop_at[c])) for c, j in enumerate(jobs)]
    with Plan(short, prec) as q:
        ref = _np(q.generate())
    assert np.array_equal(x, ref), name
    # an infinite threshold stops every curve after one iteration
    with Plan(jobs, prec) as p:
        p.set_convergence(np.full(len(jobs), math.inf), history=2)
        p.generate()
        d1, run1 = p.convergence()
    assert np.all(run1 == 1) and np.array_equal(d1[:, 0], D[:, 0])


@pytest.mark.parametrize("path", [None, "multi"])
def test_fixed_point_stops_with_delta_exactly_zero(path, monkeypatch):
    """At 2^10 the E13 map reaches a fixed point within a few hundred
    iterations: a tiny positive threshold stops the run at the first exact
    zero, and one more iteration from there changes nothing."""
    _env(monkeypatch, path)
    K = 1000
    jobs = [workloads.job(10, K, seed=5, curve_id=1)]
    with Plan(jobs, LC_FP32) as p:
        p.set_convergence(np.array([1e-300]), history=K)
        x = _np(p.generate())
        d, run = p.convergence()
        n = int(run[0])
        assert n < K, "no fixed point reached"
        assert d[0, n - 1] == 0.0 and np.all(d[0, :n - 1] > 0)
        p.iterate(1)
        d2, run2 = p.convergence()
        assert run2[0] == 1 and d2[0, 0] == 0.0
        assert np.array_equal(_np(p.get_state()), x)


def test_convergence_argument_errors():
    jobs = _jobs([10, 12], 2)
    with Plan(jobs, LC_FP32) as p:
        with pytest.raises(LcError):
            p.history = 2
            p.convergence()  # before set_convergence
        with pytest.raises(LcError):
            p.set_convergence(np.array([0.1, np.nan]), history=2)
        with pytest.raises(LcError):
            p.set_convergence(None, history=0)
        with pytest.raises(LcError):
            p.set_convergence(None, history=(1 << 16) + 1)
    deep = [workloads.job(10, 2, seed=1, curve_id=0, log_lmin=-40.0, log_lbreak=-20.0)]
    with Plan(deep, LC_FP32) as p:
        with pytest.raises(LcError):
            p.set_convergence(None, history=2)
    with Plan(deep, LC_FP64) as p:
        p.set_convergence(None, history=2)
        p.generate()
        d, run = p.convergence()
        assert run[0] == 2 and np.all(np.isfinite(d[0]))
