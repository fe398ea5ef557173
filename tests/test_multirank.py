"""The N > 1 path of bench.py on CPU: two gloo ranks run the same per-rank
workload (independent problems, weak scaling); the timing barrier and the
max-over-ranks reduction are the only cross-rank steps, and the whole-job
value counts every rank's units."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench._PG = dist
    r, w, loc = bench.dist_env()
    assert (r, w, loc) == (rank, world, rank)
    bench.barrier(w)
    # each rank reports its own elapsed time; the job time is the slowest rank
    t = bench.max_over_ranks(10.0 + rank, w)
    # units processed per rank (same workload on every rank)
    per_rank_bytes = 1000.0
    value = w * per_rank_bytes / t
    out[rank] = (t, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_barrier_and_max_timing():
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0][0] == out[1][0] == 11.0
    assert out[0][1] == pytest.approx(2 * 1000.0 / 11.0)


def test_request_trace_is_seeded_and_shardable():
    """Serving replicas: a seeded trace split round-robin over ranks covers
    every request exactly once."""
    from synth_inputs import requests
    tr = requests.trace(50, seed=3, rate_per_s=10.0)
    assert tr == requests.trace(50, seed=3, rate_per_s=10.0)
    world = 3
    shards = [[q["id"] for q in tr if q["id"] % world == r] for r in range(world)]
    assert sorted(sum(shards, [])) == list(range(50))
    assert all(32 <= q["n"] <= 2048 if q["ndim"] == 2 else 32 <= q["n"] <= 256 for q in tr)
