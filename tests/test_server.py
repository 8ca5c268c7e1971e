"""Continuous-batching server: every result equals the same job run alone
(bit for bit) and, one iteration from the setup state, the FP64 oracle per
position; admission respects the slots of the HBM budget; a retired job's slot
is reused while its cohort still runs; cohorts overlap on the device; errors
come back as status codes."""
import time

import numpy as np
import pytest

from paper_1909_06374_gb300 import (LC_FP32, LcError, Plan, _abi, lc_plan_footprint, lc_poll, lc_server_create,
                                    lc_server_destroy, lc_server_stats, lc_server_trace, lc_submit, workloads)

# bytes of the server's planes per sample of capacity (FP32), and the share
# of the budget they take
PLANE_BYTES = 40
PLANE_SHARE = 0.875


def _budget_for(samples):
    """A budget whose planes hold `samples` (a power of two) but not twice as many."""
    return int(1.5 * samples * PLANE_BYTES / PLANE_SHARE)


def _has_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def test_server_create_without_device_is_an_error():
    if _has_gpu():
        pytest.skip("a GPU is present")
    with pytest.raises(LcError) as e:
        lc_server_create(0, 1 << 30, LC_FP32)
    assert e.value.status == _abi.LC_ERR_INVALID


def _mixed_jobs(n, seed):
    rng = np.random.default_rng(seed)
    jobs = []
    for c in range(n):
        jobs.append(workloads.job(int(rng.integers(6, 15)), int(rng.integers(0, 30)), seed=100 + c,
                                  curve_id=c, f_br=float(10 ** rng.uniform(-4, -1)),
                                  alpha_high=float(rng.uniform(2, 3)), log_lbreak=float(rng.uniform(-2.5, -0.5)),
                                  slope_high=float(rng.uniform(-3, -1.5))))
    # the tabulated ERDF shapes (Eq. 1 smooth, Eq. 2 log-normal) run in the same cohorts
    shapes = list(workloads.ERDF_SHAPES.values())
    for c in range(0, n, 5):
        jobs[c] = workloads.job(jobs[c]["log2n"], jobs[c]["iters"], seed=jobs[c]["seed"], curve_id=c,
                                **shapes[(c // 5) % len(shapes)])
    return jobs


def _drain(server, tickets, jobs, timeout=120.0):
    out, lat = {}, {}
    t0 = time.time()
    while len(out) < len(tickets):
        assert time.time() - t0 < timeout, "server did not finish in time"
        for t, j in zip(tickets, jobs):
            if t in out:
                continue
            buf = np.empty(1 << j["log2n"], dtype=np.float32)
            st, ns = lc_poll(server, t, buf)
            if st == _abi.LC_OK:
                out[t], lat[t] = buf, ns
        time.sleep(0.002)
    return out, lat


@pytest.mark.gpu
def test_results_equal_the_job_alone():
    jobs = _mixed_jobs(16, 1)
    server = lc_server_create(0, 0, LC_FP32)
    try:
        tickets = []
        for j in jobs:
            tickets.append(lc_submit(server, j))
            time.sleep(0.003)  # staggered arrivals: later jobs join while earlier ones run
        out, lat = _drain(server, tickets, jobs)
    finally:
        lc_server_destroy(server)
    for t, j in zip(tickets, jobs):
        with Plan([j], LC_FP32) as p:
            alone = p.generate().cpu().numpy()
        assert np.array_equal(out[t], alone), j
        assert lat[t] > 0


@pytest.mark.gpu
def test_long_jobs_equal_the_job_alone():
    """Jobs of 2^15..2^20 samples (the sample-sort argsort, with every sample
    size and finish-group capacity) and shorter ones in the same cohorts: each
    result equals the job run alone in a plan of its own, bit for bit."""
    rng = np.random.default_rng(7)
    lengths = [15, 20, 9, 18, 13, 19, 17, 11, 16, 20]
    jobs = [workloads.job(n, int(rng.integers(2, 6)), seed=300 + c, curve_id=c,
                          f_br=float(10 ** rng.uniform(-4, -1)), alpha_high=float(rng.uniform(2, 3)))
            for c, n in enumerate(lengths)]
    server = lc_server_create(0, 0, LC_FP32)
    try:
        tickets = []
        for j in jobs:
            tickets.append(lc_submit(server, j))
            time.sleep(0.002)
        out, _ = _drain(server, tickets, jobs)
    finally:
        lc_server_destroy(server)
    for t, j in zip(tickets, jobs):
        with Plan([j], LC_FP32) as p:
            alone = p.generate().cpu().numpy()
        assert np.array_equal(out[t], alone), j["log2n"]


@pytest.mark.gpu
def test_admission_respects_the_budget():
    jobs = [workloads.job(14, 40, seed=c, curve_id=c) for c in range(6)]
    # planes of 2^15 samples: two slots of 2^14
    server = lc_server_create(0, _budget_for(1 << 15), LC_FP32)
    peak_active = 0
    try:
        assert lc_server_trace(server)["capacity"] == 1 << 15
        tickets = [lc_submit(server, j) for j in jobs]
        t0 = time.time()
        while True:
            fin, act, wait = lc_server_stats(server)
            peak_active = max(peak_active, act)
            if fin + act + wait == len(jobs) and wait == 0 and act == 0:
                break
            assert time.time() - t0 < 120
            time.sleep(0.001)
        out, _ = _drain(server, tickets, jobs)
        assert lc_server_trace(server)["free_samples"] == 1 << 15  # every slot returned
    finally:
        lc_server_destroy(server)
    assert 1 <= peak_active <= 2
    assert len(out) == len(jobs)


@pytest.mark.gpu
def test_retired_slot_is_reused_while_its_cohort_runs():
    """Two slots: a long job and a short one start together; a third job,
    waiting for a slot, takes the short job's slot when that retires and
    finishes long before the long job of the first cohort."""
    long_j = workloads.job(14, 400, seed=1, curve_id=1)
    short_j = workloads.job(14, 8, seed=2, curve_id=2)
    third = workloads.job(14, 8, seed=3, curve_id=3)
    server = lc_server_create(0, _budget_for(1 << 15), LC_FP32)
    try:
        ta = lc_submit(server, long_j)
        tb = lc_submit(server, short_j)
        tc = lc_submit(server, third)
        order = []
        t0 = time.time()
        bufs = {t: np.empty(1 << 14, dtype=np.float32) for t in (ta, tb, tc)}
        while len(order) < 3:
            assert time.time() - t0 < 120
            for t in (ta, tb, tc):
                if t in order:
                    continue
                st, _ = lc_poll(server, t, bufs[t])
                if st == _abi.LC_OK:
                    order.append(t)
            time.sleep(0.0005)
    finally:
        lc_server_destroy(server)
    assert order.index(tc) < order.index(ta), order
    with Plan([third], LC_FP32) as p:
        assert np.array_equal(bufs[tc], p.generate().cpu().numpy())


@pytest.mark.gpu
def test_cohorts_overlap_on_the_device():
    """A second cohort admitted while the first runs executes at the same time
    on the device (CUDA events around every chunk on the cohorts' streams)."""
    first = [workloads.job(20, 120, seed=c, curve_id=c) for c in range(4)]
    second = [workloads.job(20, 120, seed=10 + c, curve_id=10 + c) for c in range(4)]
    server = lc_server_create(0, 0, LC_FP32)
    try:
        tickets = [lc_submit(server, j) for j in first]
        time.sleep(0.05)  # the first cohort is running
        tickets += [lc_submit(server, j) for j in second]
        _drain(server, tickets, first + second, timeout=300)
        tr = lc_server_trace(server)
    finally:
        lc_server_destroy(server)
    assert tr["busy_ms"] > 0 and tr["overlap_ms"] > 0.1 * tr["busy_ms"], tr


@pytest.mark.gpu
def test_server_result_one_step_against_the_oracle():
    """One iteration from the setup state (the draws in draw order), through
    the server, per position against the FP64 oracle."""
    import oracle
    from tests.parity import position_check
    jobs = [workloads.job(12, 1, seed=5, curve_id=5), workloads.job(16, 1, seed=6, curve_id=6, f_br=0.01),
            workloads.job(13, 1, seed=7, curve_id=7, **workloads.ERDF_SHAPES["lognormal"])]
    server = lc_server_create(0, 0, LC_FP32)
    try:
        tickets = [lc_submit(server, j) for j in jobs]
        out, _ = _drain(server, tickets, jobs)
    finally:
        lc_server_destroy(server)
    for t, j in zip(tickets, jobs):
        r = oracle.generate(dict(j, iters=0), prec=0, want=("x", "A", "s"))
        x1, xa, _ = oracle.iterate(r["A"], r["s"], r["x"], 1, want_adj=True)
        res = position_check(out[t], x1, r["s"], xa)
        assert res["fail"] == 0 and res["not_in_draws"] == 0, (j["log2n"], res)


@pytest.mark.gpu
def test_plan_footprint_is_the_workspace():
    from paper_1909_06374_gb300 import lc_plan_workspace_bytes
    for log2n in range(12, 21):
        jobs = [workloads.job(log2n, 2, seed=1, curve_id=0), workloads.job(max(9, log2n - 3), 2, seed=2, curve_id=1)]
        with Plan(jobs, LC_FP32) as p:
            assert lc_plan_workspace_bytes(p.handle) == lc_plan_footprint(jobs), log2n


def test_plan_footprint_on_the_host():
    """No device is needed; more samples, more bytes; bad jobs are rejected."""
    a = lc_plan_footprint([workloads.job(12, 1, 0, 0)])
    b = lc_plan_footprint([workloads.job(16, 1, 0, 0)])
    c = lc_plan_footprint(workloads.uniform(ncurves=4, log2n=16, iters=1))
    assert 0 < a < b < c
    assert c > 4 * (1 << 16) * 4 * 7  # state, FFT, draws, amplitudes and sort buffers at least
    with pytest.raises(LcError) as e:
        lc_plan_footprint([workloads.job(3, 1, 0, 0)])
    assert e.value.status == _abi.LC_ERR_INVALID


@pytest.mark.gpu
def test_server_error_codes():
    server = lc_server_create(0, 1 << 28, LC_FP32)
    try:
        with pytest.raises(LcError) as e:
            lc_submit(server, workloads.job(3, 1, 0, 0))
        assert e.value.status == _abi.LC_ERR_INVALID
        with pytest.raises(LcError) as e:
            lc_submit(server, workloads.job(27, 1, 0, 0))  # longer than the planes of this budget
        assert e.value.status == _abi.LC_ERR_INVALID
        with pytest.raises(LcError) as e:  # a budget without a single slot
            lc_server_create(0, 100, LC_FP32)
        assert e.value.status == _abi.LC_ERR_INVALID
        with pytest.raises(LcError) as e:
            lc_poll(server, 987654321)
        assert e.value.status == _abi.LC_ERR_UNKNOWN_TICKET
        j = workloads.job(10, 2, 1, 1)
        t = lc_submit(server, j)
        out, _ = _drain(server, [t], [j])
        with pytest.raises(LcError) as e:  # collected already
            lc_poll(server, t)
        assert e.value.status == _abi.LC_ERR_UNKNOWN_TICKET
    finally:
        lc_server_destroy(server)


@pytest.mark.gpu
def test_destroy_with_jobs_in_flight():
    server = lc_server_create(0, 0, LC_FP32)
    for j in _mixed_jobs(8, 2):
        lc_submit(server, dict(j, iters=200))
    time.sleep(0.05)
    lc_server_destroy(server)
