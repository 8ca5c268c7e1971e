"""Multi-rank path on CPU (gloo, world size 2): the job list is sharded with no
overlap and balanced work, and the step time is the max over ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1909_06374_gb300 import workloads  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    jobs = workloads.ragged(ncurves=300, lo=10, hi=20, iters=100, master_seed=3)
    mine = workloads.shard_jobs(jobs, world)[rank]
    ids = torch.zeros(len(jobs), dtype=torch.int64)
    for j in mine:
        ids[j["curve_id"]] += 1
    dist.all_reduce(ids)
    work = torch.tensor([float(sum((1 << j["log2n"]) * j["iters"] for j in mine))], dtype=torch.float64)
    works = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(works, work)
    t = torch.tensor([10.0 + rank], dtype=torch.float64)  # per-rank step time
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        q.put((ids.tolist(), [w.item() for w in works], t.item()))
    dist.destroy_process_group()


def test_sharding_over_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    ids, works, tmax = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(v == 1 for v in ids)  # every curve on exactly one rank
    assert max(works) / min(works) < 1.05  # balanced
    assert tmax == 11.0  # the step time is the slowest rank's


def test_shard_preserves_order_and_covers():
    jobs = workloads.ragged(ncurves=50, lo=10, hi=16, iters=10, master_seed=1)
    shards = workloads.shard_jobs(jobs, 3)
    seen = sorted(j["curve_id"] for s in shards for j in s)
    assert seen == list(range(50))
    for s in shards:
        ids = [j["curve_id"] for j in s]
        assert ids == sorted(ids)
