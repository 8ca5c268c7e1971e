"""CUDA path against the FP64 oracle, through the C ABI.

Bars (the acceptance rules): ERDF draws and their multiset bit-exact; TK95
stage within 2e-5 relative L2; one iteration from the same state equal per
position except near ties (1e-5 rms of the oracle's pre-ranking series);
FP64 runs equal end to end except near ties; runs deterministic."""
import numpy as np
import pytest

import oracle
from paper_1909_06374_gb300 import LC_FP32, LC_FP64, Plan, workloads
from tests.parity import position_check, rank_stats, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TK_TOL = 2e-5


def _np(t):
    return t.detach().cpu().numpy().astype(np.float64)


def small_ragged(n=6, lo=4, hi=14, iters=4, seed=11):
    rng = np.random.default_rng(seed)
    jobs = workloads.ragged(ncurves=n, lo=lo, hi=hi, iters=iters, master_seed=seed)
    # cover the smallest and a mid size explicitly
    jobs[0]["log2n"] = lo
    jobs[1]["log2n"] = hi
    jobs[2]["log2n"] = 12
    del rng
    return jobs


JOBSETS = {
    "uniform_2^12": lambda: workloads.uniform(ncurves=8, log2n=12, iters=3),
    "ragged_2^4..2^14": lambda: small_ragged(),
    "long_2^20": lambda: workloads.long_curves(ncurves=2, log2n=20, iters=2),
    "linear_space": lambda: [workloads.job(11, 2, seed=5, curve_id=9, linear_space=1)],
    # the tabulated ERDF shapes (Eq. 1 smooth, Eq. 2 log-normal), mixed with a
    # sharp curve, on the fused (2^12) and multi-kernel (2^9, 2^17) paths
    "erdf_shapes": lambda: [
        workloads.job(12, 3, seed=21, curve_id=0, **workloads.ERDF_SHAPES["smooth_eq1"]),
        workloads.job(12, 3, seed=22, curve_id=1, **workloads.ERDF_SHAPES["lognormal"]),
        workloads.job(12, 3, seed=23, curve_id=2),
        workloads.job(9, 3, seed=24, curve_id=3, **workloads.ERDF_SHAPES["table2"]),
        workloads.job(17, 2, seed=25, curve_id=4, linear_space=1, **workloads.ERDF_SHAPES["lognormal"]),
        workloads.job(10, 3, seed=26, curve_id=5, linear_space=1, **workloads.ERDF_SHAPES["table2"]),
    ],
    # zero ERDF slopes below / above the break (the linear pieces of the
    # inverse CDF), directly and through linear_space (slope -1 + 1 = 0)
    "zero_slopes": lambda: [
        workloads.job(12, 3, seed=41, curve_id=0, slope_low=0.0),
        workloads.job(11, 3, seed=42, curve_id=1, slope_high=0.0),
        workloads.job(9, 3, seed=43, curve_id=2, slope_low=-1.0, linear_space=1),
        workloads.job(13, 2, seed=44, curve_id=3, slope_low=0.0, slope_high=0.0),
    ],
    # PSD variants: fixed-amplitude TK coefficients, PSD target amplitudes, a
    # single power law (equal slopes), on both iteration paths
    "psd_variants": lambda: [
        workloads.job(12, 3, seed=31, curve_id=0, tk_coeffs=1),
        workloads.job(12, 3, seed=32, curve_id=1, tk_targets=1),
        workloads.job(11, 3, seed=33, curve_id=2, tk_coeffs=1, tk_targets=1, alpha_low=1.5, alpha_high=1.5),
        workloads.job(17, 2, seed=34, curve_id=3, tk_coeffs=1, tk_targets=1),
        workloads.job(8, 3, seed=35, curve_id=4, alpha_low=2.2, alpha_high=2.2),
    ],
}


@pytest.mark.parametrize("name", list(JOBSETS))
@pytest.mark.parametrize("prec", [LC_FP32, LC_FP64])
def test_draws_bit_exact_and_sorted(name, prec):
    jobs = JOBSETS[name]()
    with Plan(jobs, prec) as p:
        p.setup()
        x0 = _np(p.buffer(0))
        s = _np(p.buffer(2))
    po = 0 if prec == LC_FP32 else 1
    for c, j in enumerate(jobs):
        n = 1 << j["log2n"]
        erdf = oracle.job_params(j)[4:]
        d = oracle.erdf_draws(erdf, n, j["seed"], j["curve_id"], prec=po, linear_space=j.get("linear_space", 0),
                              kind=j.get("erdf_kind", 0))
        seg = slice(p.offsets[c], p.offsets[c + 1])
        assert np.array_equal(x0[seg], d), (name, c)
        assert np.array_equal(s[seg], np.sort(d)), (name, c)


@pytest.mark.parametrize("name", list(JOBSETS))
@pytest.mark.parametrize("prec", [LC_FP32, LC_FP64])
def test_tk_stage_and_amplitudes(name, prec):
    jobs = JOBSETS[name]()
    with Plan(jobs, prec) as p:
        tk = p.empty()
        p.setup(out_tk=tk)
        tk = _np(tk)
        A = _np(p.buffer(1))
    offh = 0
    for c, j in enumerate(jobs):
        n = 1 << j["log2n"]
        par = oracle.job_params(j)
        x_tk, A_or, _ = oracle.tk_series(j["log2n"], par[0], par[1:4], j["seed"], j["curve_id"],
                                         coeffs=j.get("tk_coeffs", 0), targets=j.get("tk_targets", 0))
        err = rel_l2(tk[p.offsets[c]:p.offsets[c + 1]], x_tk)
        assert err <= (TK_TOL if prec == LC_FP32 else 1e-12), (name, c, err)
        a = A[offh:offh + n // 2 + 1]
        offh += n // 2 + 1
        assert a[0] == 0.0
        assert rel_l2(a, A_or) <= (2e-7 if prec == LC_FP32 else 1e-13), (name, c)


@pytest.mark.parametrize("name", list(JOBSETS))
@pytest.mark.parametrize("prec", [LC_FP32, LC_FP64])
@pytest.mark.parametrize("k", [0, 2])
def test_one_iteration_from_the_same_state(name, prec, k):
    """The oracle runs k iterations from its own setup; both sides then take one
    iteration from that state (each with its own amplitudes and draws)."""
    jobs = JOBSETS[name]()
    po = 0 if prec == LC_FP32 else 1
    states, expect = [], []
    for j in jobs:
        r = oracle.generate(dict(j, iters=0), prec=po, want=("x", "A", "s"))
        xk, _, _ = oracle.iterate(r["A"], r["s"], r["x"], k)
        x1, xa, _ = oracle.iterate(r["A"], r["s"], xk, 1, want_adj=True)
        states.append(xk)
        expect.append((x1, r["s"], xa))
    with Plan(jobs, prec) as p:
        p.setup()
        st = torch.tensor(np.concatenate(states), dtype=p.dtype, device="cuda")
        p.set_state(st)
        p.iterate(1)
        got = _np(p.get_state())
    for c, (x1, s, xa) in enumerate(expect):
        g = got[p.offsets[c]:p.offsets[c + 1]]
        r = position_check(g, x1, s, xa)
        assert r["not_in_draws"] == 0 and r["fail"] == 0, (name, c, r)


def test_fp64_single_curve_end_to_end():
    """The single-curve FP64 workload at full size (2^14 samples, 100 iterations)."""
    jobs = workloads.single()
    j = jobs[0]
    with Plan(jobs, LC_FP64) as p:
        g = _np(p.generate())
    r = oracle.generate(dict(j, iters=0), prec=1, want=("x", "A", "s"))
    x99, _, _ = oracle.iterate(r["A"], r["s"], r["x"], 99)
    x100, xa, _ = oracle.iterate(r["A"], r["s"], x99, 1, want_adj=True)
    assert np.array_equal(np.sort(g), r["s"])
    res = position_check(g, x100, r["s"], xa)
    stats = rank_stats(g, x100)
    print("fp64 single curve:", res, stats)
    assert res["fail"] == 0, (res, stats)


@pytest.mark.parametrize("prec", [LC_FP32, LC_FP64])
def test_end_to_end_multiset_and_rank_statistics(prec):
    jobs = small_ragged(n=5, lo=10, hi=13, iters=20, seed=4)
    po = 0 if prec == LC_FP32 else 1
    with Plan(jobs, prec) as p:
        g = _np(p.generate())
    for c, j in enumerate(jobs):
        r = oracle.generate(j, prec=po, want=("x", "s"))
        seg = g[p.offsets[c]:p.offsets[c + 1]]
        assert np.array_equal(np.sort(seg), r["s"])
        st = rank_stats(seg, r["x"])
        print(f"prec={prec} curve {c} N=2^{j['log2n']}: {st}")
        assert st["spearman"] > 0.99


def test_deterministic_and_independent_of_batch_mix():
    jobs = small_ragged(n=6, lo=8, hi=14, iters=5, seed=21)
    with Plan(jobs, LC_FP32) as p:
        a = _np(p.generate())
        b = _np(p.generate())
    assert np.array_equal(a, b)
    alone_job = jobs[3]
    with Plan([alone_job], LC_FP32) as q:
        alone = _np(q.generate())
    assert np.array_equal(alone, a[p.offsets[3]:p.offsets[4]])


def test_iterate_equals_generate():
    jobs = workloads.uniform(ncurves=3, log2n=11, iters=6)
    with Plan(jobs, LC_FP32) as p:
        full = _np(p.generate())
        p.setup()
        p.iterate(2)
        p.iterate(4)
        split = _np(p.get_state())
    assert np.array_equal(full, split)


def test_zero_iterations_returns_draw_order():
    jobs = [workloads.job(12, 0, seed=3, curve_id=1)]
    with Plan(jobs, LC_FP32) as p:
        g = _np(p.generate())
    d = oracle.erdf_draws(oracle.job_params(jobs[0])[4:], 1 << 12, 3, 1, prec=0)
    assert np.array_equal(g, d)


def test_host_entry_point_matches_device():
    from paper_1909_06374_gb300 import lc_generate_host
    jobs = small_ragged(n=4, lo=9, hi=12, iters=3, seed=8)
    with Plan(jobs, LC_FP32) as p:
        dev = _np(p.generate())
        tk_dev = p.empty()
        p.setup(out_tk=tk_dev)
        host = torch.empty(p.total, dtype=torch.float32).pin_memory()
        host_tk = torch.empty(p.total, dtype=torch.float32).pin_memory()
        lc_generate_host(p.handle, host, host_tk)
        assert np.array_equal(host.numpy().astype(np.float64), dev)
        assert np.array_equal(host_tk.numpy(), tk_dev.cpu().numpy())


def test_uniform_full_size_sampled():
    """4096 curves x 2^16, 200 iterations (the benchmark launch): the multiset of
    64 sampled curves is the oracle's draw multiset, bit for bit, and one more
    iteration from the oracle's state matches per position on 2 curves."""
    jobs = workloads.uniform()
    rng = np.random.default_rng(0)
    sample = sorted(rng.choice(len(jobs), 64, replace=False).tolist())
    step = sample[:2]
    with Plan(jobs, LC_FP32) as p:
        g = p.generate()
        gn = g.cpu().numpy()
        for c in sample:
            j = jobs[c]
            d = oracle.erdf_draws(oracle.job_params(j)[4:], 1 << 16, j["seed"], j["curve_id"], prec=0)
            assert np.array_equal(np.sort(gn[p.offsets[c]:p.offsets[c + 1]].astype(np.float64)), np.sort(d))
        # one-step check on sampled curves inside the full batch
        st = g.clone()
        expect = {}
        for c in step:
            j = jobs[c]
            r = oracle.generate(dict(j, iters=0), prec=0, want=("x", "A", "s"))
            xk, _, _ = oracle.iterate(r["A"], r["s"], r["x"], 1)
            x1, xa, _ = oracle.iterate(r["A"], r["s"], xk, 1, want_adj=True)
            st[p.offsets[c]:p.offsets[c + 1]] = torch.tensor(xk, dtype=torch.float32, device="cuda")
            expect[c] = (x1, r["s"], xa)
        p.set_state(st)
        p.iterate(1)
        got = p.get_state().cpu().numpy()
    for c, (x1, s, xa) in expect.items():
        r = position_check(got[p.offsets[c]:p.offsets[c + 1]], x1, s, xa)
        assert r["fail"] == 0 and r["not_in_draws"] == 0, (c, r)


def _one_step_in_batch(p, jobs, gpu_state, picks, prec=0):
    """Replace the state of the picked curves by the oracle's state after one
    oracle iteration, run one GPU iteration on the whole batch, and compare
    the picked curves with the oracle's next iteration per position."""
    st = gpu_state.clone()
    expect = {}
    for c in picks:
        j = jobs[c]
        r = oracle.generate(dict(j, iters=0), prec=prec, want=("x", "A", "s"))
        xk, _, _ = oracle.iterate(r["A"], r["s"], r["x"], 1)
        x1, xa, _ = oracle.iterate(r["A"], r["s"], xk, 1, want_adj=True)
        st[p.offsets[c]:p.offsets[c + 1]] = torch.tensor(xk, dtype=p.dtype, device="cuda")
        expect[c] = (x1, r["s"], xa)
    p.set_state(st)
    p.iterate(1)
    got = p.get_state().cpu().numpy()
    for c, (x1, s, xa) in expect.items():
        r = position_check(got[p.offsets[c]:p.offsets[c + 1]], x1, s, xa)
        assert r["fail"] == 0 and r["not_in_draws"] == 0, (c, jobs[c]["log2n"], r)


def test_ragged_full_size_sampled():
    """10000 curves, N log-uniform over 2^10..2^20, 100 iterations (the ragged
    workload as benchmarked): draw multisets of 40 sampled curves bit-exact, and
    one iteration from the oracle's state per position on curves of both paths
    (the one-CTA fused kernel up to 2^14, the multi-kernel path above)."""
    jobs = workloads.ragged()
    rng = np.random.default_rng(1)
    sample = sorted(rng.choice(len(jobs), 40, replace=False).tolist())
    by_len = {}
    for c, j in enumerate(jobs):
        by_len.setdefault(j["log2n"], c)
    picks = [by_len[l] for l in (10, 14, 15, 16, 17)]
    with Plan(jobs, LC_FP32) as p:
        g = p.generate()
        gn = g.cpu().numpy()
        for c in sample:
            j = jobs[c]
            d = oracle.erdf_draws(oracle.job_params(j)[4:], 1 << j["log2n"], j["seed"], j["curve_id"], prec=0)
            seg = gn[p.offsets[c]:p.offsets[c + 1]].astype(np.float64)
            assert np.array_equal(np.sort(seg), np.sort(d)), c
        _one_step_in_batch(p, jobs, g, picks)


def test_long_full_size_sampled():
    """8 curves of 2^26 samples, 50 iterations: the draw multiset of two curves
    is the oracle's, bit for bit (one iteration at 2^20 is checked per position
    in test_one_iteration_from_the_same_state)."""
    jobs = workloads.long_curves()
    with Plan(jobs, LC_FP32) as p:
        g = p.generate()
        for c in (0, 5):
            j = jobs[c]
            d = oracle.erdf_draws(oracle.job_params(j)[4:], 1 << j["log2n"], j["seed"], j["curve_id"], prec=0)
            seg = g[p.offsets[c]:p.offsets[c + 1]].cpu().numpy().astype(np.float64)
            assert np.array_equal(np.sort(seg), np.sort(d)), c


def test_maximum_length_2_27():
    """One curve of the largest length the boundary accepts (2^27 samples, three
    tile passes per transform with three twiddle levels, 65536 sort tiles per
    pass): 4096 sampled draws equal the oracle's Philox + inverse-CDF draw at
    that index, bit for bit; the TK95 series has mean 0 and rms 1 (the
    normalisation); after two iterations the series is a permutation of the
    sorted draws, bit for bit (checked with torch's sort, not the library's)."""
    n = 1 << 27
    j = workloads.job(27, 2, seed=7, curve_id=3)
    erdf = oracle.job_params(j)[4:]
    rng = np.random.default_rng(5)
    ks = np.unique(np.concatenate([[0, 1, n - 2, n - 1], rng.integers(0, n, 4092)]))
    blocks = ks >> 1
    ctr = np.stack([blocks & 0xffffffff, blocks >> 32, np.full_like(blocks, j["curve_id"]), np.ones_like(blocks)], 1)
    key = np.tile(np.array([j["seed"] & 0xffffffff, j["seed"] >> 32], dtype=np.uint64), (len(ks), 1))
    w = oracle.philox(ctr.astype(np.uint32), key.astype(np.uint32))
    U = np.array([oracle.u01(int(r[2 * (k & 1)]), int(r[2 * (k & 1) + 1])) for r, k in zip(w, ks)])
    want = oracle.erdf_icdf(erdf[:5], U).astype(np.float32)
    with Plan([j], LC_FP32) as p:
        tk = p.empty()
        p.setup(out_tk=tk)
        x0 = p.buffer(0)
        s = p.buffer(2)
        assert np.array_equal(x0[torch.as_tensor(ks, device=x0.device)].cpu().numpy(), want)
        assert torch.equal(torch.sort(x0).values, s)
        tkd = tk.double()
        assert abs(float(tkd.mean())) < 1e-4 and abs(float(tkd.square().mean().sqrt()) - 1.0) < 1e-4
        x2 = p.generate()
        assert torch.equal(torch.sort(x2).values, s)
        assert not torch.equal(x2, x0)


@pytest.mark.parametrize("path,log2n", [("resident", 16), ("resident", 15), ("multi", 12), ("multi", 13),
                                        ("multi", 14)])
def test_forced_paths_one_step(path, log2n, monkeypatch):
    """The per-length table picks one iteration path; every complete path stays
    correct: LC_PATH=resident runs 2^16 curves on the 4-CTA and 2^15 curves on
    the 2-CTA cluster kernel, LC_PATH=multi runs 2^12 curves (radix-pass FFT,
    radix argsort) and 2^13, 2^14 curves (tile FFT, sample sort) on the
    multi-kernel path."""
    monkeypatch.setenv("LC_PATH", path)
    jobs = workloads.uniform(ncurves=3, log2n=log2n, iters=2)
    states, expect = [], []
    for j in jobs:
        r = oracle.generate(dict(j, iters=0), prec=0, want=("x", "A", "s"))
        xk, _, _ = oracle.iterate(r["A"], r["s"], r["x"], 1)
        x1, xa, _ = oracle.iterate(r["A"], r["s"], xk, 1, want_adj=True)
        states.append(xk)
        expect.append((x1, r["s"], xa))
    with Plan(jobs, LC_FP32) as p:
        p.setup()
        p.set_state(torch.tensor(np.concatenate(states), dtype=torch.float32, device="cuda"))
        p.iterate(1)
        got = _np(p.get_state())
    for c, (x1, s, xa) in enumerate(expect):
        r = position_check(got[p.offsets[c]:p.offsets[c + 1]], x1, s, xa)
        assert r["fail"] == 0 and r["not_in_draws"] == 0, (path, c, r)


def test_profile_runs_one_iteration_with_timed_groups():
    """lc_plan_profile advances the state by exactly one iteration (the same
    bits as lc_iterate(1) from that state) and times the kernel groups that
    ran: fused kernels for the 2^12 curve, transforms / sort for the rest."""
    from paper_1909_06374_gb300 import lc_plan_profile
    jobs = [workloads.job(12, 2, seed=1, curve_id=0), workloads.job(17, 2, seed=2, curve_id=1),
            workloads.job(9, 2, seed=3, curve_id=2)]
    with Plan(jobs, LC_FP32) as p:
        p.generate()
        start = p.get_state()
        prof = lc_plan_profile(p.handle)
        after = _np(p.get_state())
        p.set_state(start)
        p.iterate(1)
        want = _np(p.get_state())
    assert np.array_equal(after, want)
    assert prof["resident"] > 0 and prof["fft"] > 0 and prof["sort_scatter"] > 0 and prof["sort_hist_scan"] > 0
    assert prof["convergence"] == 0
    # the 2^9 class: four FP32 radix passes; the 2^17 class: the sample sort (one span)
    assert prof["scatter_launches"] == 4 + 1
    assert prof["sorted_elements"] == (1 << 17) + (1 << 9) and prof["fused_elements"] == 1 << 12
    assert prof["bucket_elements"] == 1 << 17


def test_classes_sharing_tile_kernels_one_step():
    """Curves of 2^18, 2^16 and 2^17 samples in one plan: the 2^18 and 2^17
    classes run the fused forward-last / spectral / inverse-first kernel of
    radix 2^8, the 2^16 and 2^17 classes the radix-2^8 tile pass, each with a
    different shared-memory size (the twiddle tables grow with the length).
    Every launch of the captured iteration graph must get the size it asks
    for.  One iteration from the oracle's state, per position, on all three
    (the oracle's states after one of its iterations)."""
    jobs = [workloads.job(18, 3, seed=51, curve_id=0, f_br=0.01),
            workloads.job(16, 3, seed=52, curve_id=1),
            workloads.job(17, 3, seed=53, curve_id=2, alpha_high=2.7)]
    states, expect = [], []
    for j in jobs:
        r = oracle.generate(dict(j, iters=0), prec=0, want=("x", "A", "s"))
        xk, _, _ = oracle.iterate(r["A"], r["s"], r["x"], 1)
        x1, xa, _ = oracle.iterate(r["A"], r["s"], xk, 1, want_adj=True)
        states.append(xk)
        expect.append((x1, r["s"], xa))
    with Plan(jobs, LC_FP32) as p:
        p.generate()  # the iteration graph is captured and replayed first
        p.set_state(torch.tensor(np.concatenate(states), dtype=torch.float32, device="cuda"))
        p.iterate(1)
        got = _np(p.get_state())
    for c, (x1, s, xa) in enumerate(expect):
        r = position_check(got[p.offsets[c]:p.offsets[c + 1]], x1, s, xa)
        assert r["fail"] == 0 and r["not_in_draws"] == 0, (jobs[c]["log2n"], r)


def test_stage_launches_shared_by_classes(monkeypatch):
    """Curves of 2^13 .. 2^19, 2^21 and 2^22 samples on the multi-kernel path
    share the launches of each iteration stage.  Transforms: one launch per
    (stage, kernel form, radix) -- the first forward tile pass over the radices
    2^6..2^9, the second one of the 2^21 and 2^22 curves (radix 2^7), the
    fused spectral kernels over 2^6..2^9, and the inverse passes alike: 4 + 1 +
    4 + 1 + 4 = 14.  Sample sort of 2^13..2^19: the sample kernel per sample
    size (1024 values up to 2^17, 4096 above), histogram, scan and scatter
    once, the finish and its tail (the groups beyond the launched slots) per
    group capacity (2048 up to 2^18, 4096 at 2^19): 9.  Radix argsort of 2^21
    and 2^22: four passes of histogram, tile scan, chunk scan and scatter: 16.
    With the iteration counter, 40 launches per iteration, against 99 with one
    launch per class and kernel.  Every curve's
    result is the same, bit for bit, as that curve's run alone."""
    from paper_1909_06374_gb300 import lc_plan_last_launches
    monkeypatch.setenv("LC_PATH", "multi")
    lengths = list(range(13, 20)) + [21, 22]
    jobs = [workloads.job(n, 3, seed=60 + n, curve_id=n, f_br=0.02 if n % 2 else 0.004) for n in lengths]
    with Plan(jobs, LC_FP32) as p:
        mixed = _np(p.generate())
        p.iterate(1)  # queues the iteration budgets' reset and one iteration
        per_iter = lc_plan_last_launches(p.handle) - 1
    assert per_iter == 40, per_iter
    for c, j in enumerate(jobs):
        with Plan([j], LC_FP32) as q:
            alone = _np(q.generate())
        assert np.array_equal(alone, mixed[p.offsets[c]:p.offsets[c + 1]]), j["log2n"]
