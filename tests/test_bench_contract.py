"""bench.py on the host: the reference arm's JSON line (the FP64 oracle on the
host cores) and the bounded CPU-oracle samples of the other workloads."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1909_06374_gb300 import workloads  # noqa: E402


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == bench.UNIT
    assert line["metric"] == bench.METRIC and line["higher_is_better"] is True
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_cpu_baseline_samples_are_bounded_pieces_of_their_workloads():
    for w, full in (("single", workloads.single()), ("long", workloads.long_curves()),
                    ("ragged", workloads.ragged())):
        jobs, prec, desc = bench.cpu_baseline_sample(w, 16)
        assert 1 <= len(jobs) <= 16 and desc
        assert prec == (1 if w == "single" else 0)
        assert workloads.sample_iters(jobs) <= 2 ** 27  # seconds of CPU work, not minutes
        for j, f in zip(jobs, full):
            # the workload's own parameters (the long curves at a shorter length)
            for key in ("f_br", "alpha_high", "log_lbreak", "slope_high", "seed", "curve_id", "dt"):
                assert j[key] == f[key], (w, key)


def test_scheduled_bytes_per_sample_iteration():
    """The bytes the scheduled kernels move per sample-iteration: the headline
    (2^16, FP32: three FFT kernels of 8 B + 2 B of amplitudes, sample sort
    34 B) 60 B; the long curves (2^26: five FFT kernels, radix argsort 76 B)
    118 B; the FP64 single curve (2^14: three FFT kernels of 16 B + 4 B, 256 B
    of radix passes) 308 B; the ragged batch between its fused and its
    multi-kernel curves' figures, undefined when the fused samples match no
    crossover of the path table."""
    import bench
    jobs, _, _, _ = bench.rank_jobs("uniform", 0, 1)
    assert bench.scheduled_bytes_per_sample_iter(jobs, 4, 0) == 60.0
    jobs, _, _, _ = bench.rank_jobs("long", 0, 1)
    assert bench.scheduled_bytes_per_sample_iter(jobs, 4, 0) == 118.0
    jobs, _, _, _ = bench.rank_jobs("single", 0, 1)
    assert bench.scheduled_bytes_per_sample_iter(jobs, 8, 0) == 308.0
    jobs, _, _, _ = bench.rank_jobs("ragged", 0, 1)
    for top in (12, 14):  # the built-in crossover and LC_RESIDENT_MAX_LOG2=14
        fused = sum(1 << j["log2n"] for j in jobs if 10 <= j["log2n"] <= top)
        v = bench.scheduled_bytes_per_sample_iter(jobs, 4, fused)
        assert 14.0 / 100 < v < 118.0
    assert bench.scheduled_bytes_per_sample_iter(jobs, 4, fused + 1) is None
