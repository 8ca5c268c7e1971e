"""Host model of the sample-sort argsort's decomposition (no GPU).

The CUDA kernels rank every element exactly inside its group of buckets, so
the stable argsort follows from three facts that this model checks on the
CPU with numpy, for the sample sizes and group capacities the library uses
per length (1024 values and groups of 2048 up to 2^17, 4096 values and groups
of N/128 from 2^18 on):
  - the bucket of a value (the number of splitters not above it) is monotone
    in the value, so rank = the group's first bucket base + the rank inside
    the group by (value, position) is the stable argsort;
  - the greedy groups (each as long as the capacity allows, a larger bucket
    alone) never need more than gmax = 2 N / cap + 1 work-item slots;
  - a group can be empty (empty buckets before an oversize one) while later
    groups are not, which is why the finish's tail walks up to the curve's
    group count rather than stopping at the first empty item.
It also reproduces the group counts that set how many finish blocks are
launched per curve: on continuous values, 35 groups on average at 2^16 (of
65 slots) and about 178 from 2^18 on (of 257)."""
import numpy as np
import pytest

BUCKETS = 256


def sample_size(log2n):
    return 4096 if log2n >= 18 else 1024


def capacity(log2n):
    return 2048 if log2n <= 18 else 2048 << (log2n - 18)


def order_key(x32):
    """Order-preserving unsigned key of float32 values (-0 taken as +0)."""
    x = np.where(x32 == 0, np.float32(0), x32).astype(np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    return np.where(u >> 31, 0xFFFFFFFF - u, u | 0x80000000).astype(np.uint64)


def splitters(x32, S):
    n = x32.size
    stride = n // S
    smp = np.sort(x32[np.arange(S) * stride + stride // 2])
    return smp[(S // BUCKETS) * (np.arange(BUCKETS - 1) + 1)]


def buckets_of(x32, spl):
    # the number of splitters <= v, compared as floats (-0 == +0)
    return np.searchsorted(spl, x32, side="right")


def greedy_groups(base, cap):
    """Groups of consecutive buckets: the group starting at bucket s ends
    before the last e with base[e] - base[s] <= cap (at least s + 1)."""
    groups, b = [], 0
    while b < BUCKETS:
        e = np.searchsorted(base, base[b] + cap, side="right") - 1
        e = max(e, b + 1)
        groups.append((b, int(min(e, BUCKETS))))
        b = int(min(e, BUCKETS))
    return groups


def model_argsort(x32, log2n):
    spl = splitters(x32, sample_size(log2n))
    b = buckets_of(x32, spl)
    cnt = np.bincount(b, minlength=BUCKETS)
    base = np.concatenate([[0], np.cumsum(cnt)])
    groups = greedy_groups(base, capacity(log2n))
    key = (order_key(x32) << np.uint64(32)) | np.arange(x32.size, dtype=np.uint64)
    rank = np.empty(x32.size, dtype=np.int64)
    for b0, b1 in groups:
        members = np.nonzero((b >= b0) & (b < b1))[0]
        rank[members[np.argsort(key[members])]] = base[b0] + np.arange(members.size)
    perm = np.empty_like(rank)
    perm[rank] = np.arange(x32.size)
    return perm, groups, base


def patterns(n, rng):
    return {
        "normal": rng.standard_normal(n),
        "integer_ties": rng.integers(0, 50, n).astype(np.float64),
        "signed_zeros": np.where(rng.random(n) < 0.5, -0.0, 0.0),
        "spike_30pct": np.where(rng.random(n) < 0.3, 1.0, rng.standard_normal(n)),
        "two_clusters": np.where(rng.random(n) < 0.5, 1e6, -1e6) + rng.standard_normal(n),
    }


@pytest.mark.parametrize("log2n", [13, 16, 18, 20])
def test_decomposition_is_the_stable_argsort(log2n):
    rng = np.random.default_rng(log2n)
    n = 1 << log2n
    gmax = 2 * n // capacity(log2n) + 1
    for name, v in patterns(n, rng).items():
        x = v.astype(np.float32)
        perm, groups, _ = model_argsort(x, log2n)
        want = np.argsort(order_key(x), kind="stable")
        assert np.array_equal(perm, want), (name, log2n)
        assert len(groups) <= gmax, (name, log2n, len(groups))


def test_empty_groups_precede_later_groups_with_integer_ties():
    rng = np.random.default_rng(3)
    x = rng.integers(0, 50, 1 << 17).astype(np.float32)
    _, groups, base = model_argsort(x, 17)
    sizes = [int(base[b1] - base[b0]) for b0, b1 in groups]
    first_empty = next(i for i, s in enumerate(sizes) if s == 0)
    assert any(s > 0 for s in sizes[first_empty:]), sizes


def test_group_counts_on_continuous_values():
    rng = np.random.default_rng(5)
    counts = {}
    for log2n, trials in ((16, 60), (18, 12)):
        n = 1 << log2n
        g = [len(model_argsort(rng.standard_normal(n).astype(np.float32), log2n)[1]) for _ in range(trials)]
        counts[log2n] = (np.mean(g), max(g))
    assert 33 <= counts[16][0] <= 37 and counts[16][1] <= 38  # 38 finish blocks launched per 2^16 curve
    assert 170 <= counts[18][0] <= 186 and counts[18][1] <= 189  # 189 from 2^18 on
