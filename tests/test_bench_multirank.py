"""bench.py's multi-rank branch on CPU (gloo, world size 2), with the generator
step replaced by a stub: each rank takes its share of every workload (uniform:
its own batch with curve ids offset by rank; long and ragged: disjoint shards
that cover the job list; single: rank 0 only), the timed loop runs exactly the
requested steps between barriers, the step time is the max over ranks, and the
whole-job value is the work of all ranks over that time -- the same on both
ranks.  The GPU form of this branch (NCCL) is not measured on hardware here."""
import os
import socket
import sys
import time

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    from paper_1909_06374_gb300 import workloads
    dist.init_process_group("gloo", rank=rank, world_size=world)
    out = {}
    for w, kw in (("uniform", dict(curves=8, log2n=10)), ("ragged", {}), ("long", {}), ("single", {})):
        jobs, prec, dtype, desc = bench.rank_jobs(w, rank, world, **kw)
        si = workloads.sample_iters(jobs)
        calls = []

        def step():  # stand-in for one generator run: work-proportional host time
            calls.append(1)
            time.sleep(0.002 + 1e-12 * si)

        steps = 3
        ms = bench.timed_steps(step, steps, dist.barrier, bench.HostClock())
        max_ms = bench.reduce_over_ranks(ms, dist, "max")
        total = bench.reduce_over_ranks(si, dist, "sum")
        out[w] = dict(ids=[(j["curve_id"], j["seed"]) for j in jobs], ms=ms, max_ms=max_ms, total=total,
                      value=bench.throughput(total, steps, max_ms), calls=len(calls), prec=prec, si=si)
    q.put((rank, out))
    dist.destroy_process_group()


def test_bench_branch_over_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    sys.path.insert(0, ROOT)
    from paper_1909_06374_gb300 import workloads
    for w in ("uniform", "ragged", "long", "single"):
        a, b = res[0][w], res[1][w]
        assert a["calls"] == b["calls"] == 3  # exactly the requested steps
        assert a["max_ms"] == b["max_ms"] == max(a["ms"], b["ms"])
        assert a["total"] == b["total"] == a["si"] + b["si"]
        assert a["value"] == b["value"] == a["total"] * 3 / (a["max_ms"] / 1000.0)
        ids_a, ids_b = set(a["ids"]), set(b["ids"])
        assert not ids_a & ids_b  # no curve generated twice
    # weak scaling: rank r's uniform batch is curves 8r .. 8r+7
    assert sorted(res[0]["uniform"]["ids"]) == [(c, c) for c in range(8)]
    assert sorted(res[1]["uniform"]["ids"]) == [(c, c) for c in range(8, 16)]
    # sharded workloads: the two shards are the whole job list
    for w, full in (("ragged", workloads.ragged()), ("long", workloads.long_curves())):
        got = sorted(res[0][w]["ids"] + res[1][w]["ids"])
        assert got == sorted((j["curve_id"], j["seed"]) for j in full)
    assert len(res[0]["single"]["ids"]) == 1 and res[1]["single"]["ids"] == []
    assert res[0]["single"]["prec"] == 1
