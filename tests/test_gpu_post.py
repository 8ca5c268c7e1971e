"""Periodogram (App. A, Eq. A2 / A4) and structure function (Eq. A6) on the GPU,
through the C ABI, against the FP64 oracle applied to the same series.

Bars: FP32 periodogram within 2e-5 relative L2 per curve (the FP32 FFT, as
for the TK95 stage), FP64 within 1e-12; structure function within 1e-5 (runs
of 64 FP32 squares) and 1e-12 in FP64; Parseval and Eq. A5 hold on the GPU
output at full size."""
import numpy as np
import pytest

import oracle
from paper_1909_06374_gb300 import LC_FP32, LC_FP64, LcError, Plan, workloads
from tests.parity import rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _jobs():
    # the radix-pass FFT (2^4, 2^10), the tile FFT (2^13, 2^17), dt != 1
    return [workloads.job(4, 2, seed=1, curve_id=0), workloads.job(10, 3, seed=2, curve_id=1, dt=0.25),
            workloads.job(13, 3, seed=3, curve_id=2, **workloads.ERDF_SHAPES["lognormal"]),
            workloads.job(17, 2, seed=4, curve_id=3, dt=7.0)]


@pytest.mark.parametrize("prec", [LC_FP32, LC_FP64])
@pytest.mark.parametrize("rms", [False, True])
def test_periodogram_matches_oracle(prec, rms):
    jobs = _jobs()
    tol = 2e-5 if prec == LC_FP32 else 1e-12
    with Plan(jobs, prec) as p:
        x = p.generate()
        P = p.periodogram(x, rms=rms).cpu().numpy()
        xs = x.cpu().numpy().astype(np.float64)
    offh = 0
    for c, j in enumerate(jobs):
        n = 1 << j["log2n"]
        want = oracle.periodogram(xs[p.offsets[c]:p.offsets[c + 1]], dt=j["dt"], rms=rms)
        got = P[offh:offh + n // 2 + 1]
        offh += n // 2 + 1
        assert rel_l2(got, want) <= tol, (c, rel_l2(got, want))
        assert got[0] == pytest.approx(want[0], rel=1e-6 if prec == LC_FP32 else 1e-13)


@pytest.mark.parametrize("prec", [LC_FP32, LC_FP64])
def test_structure_function_matches_oracle(prec):
    jobs = _jobs()
    lags = [1, 2, 3, 5, 8, 15]  # the shortest curve has N = 16
    tol = 1e-5 if prec == LC_FP32 else 1e-12
    with Plan(jobs, prec) as p:
        x = p.generate()
        sf = p.structure_function(x, lags).cpu().numpy()
        xs = x.cpu().numpy().astype(np.float64)
    for c in range(len(jobs)):
        want = oracle.structure_function(xs[p.offsets[c]:p.offsets[c + 1]], lags)
        np.testing.assert_allclose(sf[c], want, rtol=tol)
    jobs2 = [workloads.job(16, 1, seed=9, curve_id=9)]
    lags2 = np.unique(np.logspace(0, 15.9, 40, base=2).astype(np.uint32))
    with Plan(jobs2, prec) as p:
        x = p.generate()
        sf = p.structure_function(x, lags2).cpu().numpy()[0]
        want = oracle.structure_function(x.cpu().numpy().astype(np.float64), lags2)
    np.testing.assert_allclose(sf, want, rtol=tol)


def test_full_size_identities_and_sampled_curves():
    """The uniform workload's size (4096 x 2^16, a few iterations): Parseval
    and Eq. A5 on every curve of the GPU output; sampled curves against the
    oracle."""
    jobs = workloads.uniform(ncurves=4096, log2n=16, iters=2)
    n = 1 << 16
    lags = [1, 10, 100, 1000, 10000]
    with Plan(jobs, LC_FP32) as p:
        x = p.generate()
        P = p.periodogram(x).cpu().numpy().reshape(4096, n // 2 + 1)
        Pr = p.periodogram(x, rms=True).cpu().numpy().reshape(4096, n // 2 + 1)
        sf = p.structure_function(x, lags).cpu().numpy()
        xs = x.cpu().numpy().astype(np.float64).reshape(4096, n)
    lhs = P[:, 0] + P[:, -1] + 2 * P[:, 1:-1].sum(axis=1)
    np.testing.assert_allclose(lhs, 2.0 / n * np.sum(xs ** 2, axis=1), rtol=2e-5)
    integral = (Pr[:, 1:-1].sum(axis=1) + 0.5 * Pr[:, -1]) / n
    np.testing.assert_allclose(integral, xs.var(axis=1) / xs.mean(axis=1) ** 2, rtol=2e-4)
    for c in (0, 1234, 4095):
        assert rel_l2(P[c], oracle.periodogram(xs[c])) <= 2e-5
        np.testing.assert_allclose(sf[c], oracle.structure_function(xs[c], lags), rtol=1e-5)


def test_estimator_argument_errors():
    jobs = [workloads.job(6, 1, seed=1, curve_id=0), workloads.job(10, 1, seed=2, curve_id=1)]
    with Plan(jobs, LC_FP32) as p:
        x = p.generate()
        for bad in ([0], [64], [1, 2, 70]):
            with pytest.raises(LcError):
                p.structure_function(x, bad)
        with pytest.raises(LcError):
            p.structure_function(x, [])
        sf = p.structure_function(x, [63])
        assert torch.isfinite(sf).all()
