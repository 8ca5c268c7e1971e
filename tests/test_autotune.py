"""The autotuning sweep of the iteration path (paper_1909_06374_gb300.autotune):
its crossover rule on the host, and on a GPU the sweep itself and the
LC_RESIDENT_MAX_LOG2 override of the auto mode's per-length table."""
import numpy as np
import pytest

from paper_1909_06374_gb300 import autotune


def test_crossover_is_the_longest_length_of_an_unbroken_fused_lead():
    t = {10: {"resident": 3.0, "multi": 1.0}, 11: {"resident": 3.0, "multi": 2.0},
         12: {"resident": 2.0, "multi": 2.5}, 13: {"resident": 4.0, "multi": 1.0}}
    assert autotune.crossover(t) == 11          # a later fused win does not count
    assert autotune.crossover({10: {"resident": 1.0, "multi": 2.0}}) == 9
    assert autotune.crossover({10: {"resident": 2.0, "multi": 1.0}, 11: {"resident": None, "multi": 1.0}}) == 10
    assert autotune.crossover({}) == 9
    ties = {10: {"resident": 1.0, "multi": 1.0}}
    assert autotune.crossover(ties) == 9        # a tie keeps the multi-kernel path


@pytest.mark.gpu
def test_sweep_runs_both_paths():
    table = autotune.sweep(range(10, 12), samples=14, iters=2)
    assert set(table) == {10, 11}
    for row in table.values():
        assert row["resident"] > 0 and row["multi"] > 0
    assert 9 <= autotune.crossover(table) <= 11


@pytest.mark.gpu
@pytest.mark.parametrize("env,fused", [(None, True), ("9", False), ("12", True), ("11", False)])
def test_resident_max_log2_moves_the_crossover(env, fused, monkeypatch):
    """A 2^12 curve runs on the fused kernel under the built-in table (crossover
    2^12) and with LC_RESIDENT_MAX_LOG2 >= 12, on the multi-kernel path below;
    the one-iteration profile shows which kernels ran."""
    torch = pytest.importorskip("torch")
    from paper_1909_06374_gb300 import LC_FP32, Plan, lc_plan_profile, workloads
    monkeypatch.delenv("LC_PATH", raising=False)
    if env is None:
        monkeypatch.delenv("LC_RESIDENT_MAX_LOG2", raising=False)
    else:
        monkeypatch.setenv("LC_RESIDENT_MAX_LOG2", env)
    with Plan([workloads.job(12, 1, seed=1, curve_id=0)], LC_FP32) as p:
        p.generate()
        prof = lc_plan_profile(p.handle)
    assert (prof["fused_elements"] == 1 << 12) == fused
    assert (prof["sorted_elements"] == 1 << 12) == (not fused)
