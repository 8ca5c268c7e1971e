"""The allocation-free entry point (for callers that cannot call cudaMalloc:
hosts whose device memory belongs to another allocator, or loops that must not
allocate after start-up) against the ordinary batch entry point, through the C
ABI, on consecutive calls that reuse its static device array."""
import ctypes

import numpy as np
import pytest

from paper_1909_06374_gb300 import LC_FP32, Plan, _abi, workloads

torch = pytest.importorskip("torch")


@pytest.mark.gpu
def test_noalloc_matches_lc_generate_on_consecutive_calls():
    lib = _abi.load()
    jobs = [workloads.job(12, 10, seed=7, curve_id=3),
            workloads.job(16, 4, seed=8, curve_id=4, f_br=0.01, alpha_high=2.6),
            workloads.job(9, 6, seed=9, curve_id=5, log_lbreak=-2.0, slope_high=-1.8),
            workloads.job(13, 5, seed=10, curve_id=6, **workloads.ERDF_SHAPES["lognormal"]),
            workloads.job(16, 2, seed=11, curve_id=7, **workloads.ERDF_SHAPES["table2"])]
    stream = torch.cuda.current_stream()
    for j in jobs:
        n = 1 << j["log2n"]
        out = torch.full((n,), float("nan"), dtype=torch.float32, device="cuda")
        job = _abi.make_job(j)
        st = lib.lc_generate_noalloc(ctypes.byref(job), ctypes.c_void_p(out.data_ptr()),
                                     ctypes.c_void_p(stream.cuda_stream))
        assert st == _abi.LC_OK, _abi.last_error()
        got = out.cpu().numpy()
        with Plan([j], LC_FP32) as p:
            ref = p.generate().cpu().numpy()
        # same kernels on the same job: identical bits (the suite's bar for
        # determinism; stricter than the one-step parity tolerance)
        assert np.array_equal(got, ref), j


@pytest.mark.gpu
def test_noalloc_rejects_curves_beyond_its_array():
    lib = _abi.load()
    out = torch.empty(1 << 17, dtype=torch.float32, device="cuda")
    job = _abi.make_job(workloads.job(17, 1, seed=1, curve_id=1))
    st = lib.lc_generate_noalloc(ctypes.byref(job), ctypes.c_void_p(out.data_ptr()), None)
    assert st == _abi.LC_ERR_INVALID
    assert "16" in _abi.last_error()
