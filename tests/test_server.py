"""Continuous-batching server: every result equals the same job run alone
(bit for bit), admission respects the HBM budget, and errors come back as
status codes."""
import time

import numpy as np
import pytest

from paper_1909_06374_gb300 import (LC_FP32, LcError, Plan, _abi, lc_poll, lc_server_create,
                                    lc_server_destroy, lc_server_stats, lc_submit, workloads)


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
def test_admission_respects_the_budget():
    jobs = [workloads.job(14, 40, seed=c, curve_id=c) for c in range(6)]
    # a budget that holds about two of these jobs at a time
    from paper_1909_06374_gb300 import lc_plan_workspace_bytes
    with Plan(jobs[:1], LC_FP32) as p:
        one = lc_plan_workspace_bytes(p.handle)
    server = lc_server_create(0, int(3.0 * one), LC_FP32)
    peak_active = 0
    try:
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
    finally:
        lc_server_destroy(server)
    assert 1 <= peak_active <= 2
    assert len(out) == len(jobs)


@pytest.mark.gpu
def test_server_error_codes():
    server = lc_server_create(0, 1 << 28, LC_FP32)
    try:
        with pytest.raises(LcError) as e:
            lc_submit(server, workloads.job(3, 1, 0, 0))
        assert e.value.status == _abi.LC_ERR_INVALID
        with pytest.raises(LcError) as e:
            lc_submit(server, workloads.job(27, 1, 0, 0))  # larger than the budget
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
