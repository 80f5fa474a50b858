"""Replica aggregation of the benchmark on CPU ranks (gloo, world size 2).

Every rank solves its own system; the job's time is the slowest rank's, and
the throughput counts the solves of all ranks over that time."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, _ = bench.dist_env()
    my_ms = [1500.0, 2500.0][rank]
    tmax = bench.barrier_max(my_ms, w)
    agg = bench.aggregate([tmax], steps=3, world=w)
    q.put((r, w, tmax, agg))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_max_time_and_total_throughput():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, (r, w, tmax, agg) in enumerate(out):
        assert r == rank and w == 2
        assert tmax == pytest.approx(2500.0)
        # 2 ranks x 3 solves in 2.5 s
        assert agg["value"] == pytest.approx(6 / 2.5)
        assert agg["ms_per_step"] == pytest.approx(2500.0 / 3)
