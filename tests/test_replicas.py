"""The multi-GPU form of the bench is replicas only: each rank solves its own seeded geometries
and the job's time is the maximum over the ranks.  Its host-side logic runs here as two gloo ranks
on the CPU (no GPU): distinct geometry seeds per rank, max-over-ranks timing, whole-job
throughput."""
import os
import socket
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    seeds = bench.geometry_seeds(rank, 4)
    elapsed = 1.5 + rank          # the ranks finish at different times
    tmax = bench.max_over_ranks(elapsed, dist, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, seeds, tmax, bench.job_throughput(world, 3, tmax)))


def test_replicas_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    s0, s1 = set(out[0][1]), set(out[1][1])
    assert not (s0 & s1)                                   # no geometry solved twice
    assert out[0][2] == out[1][2] == 2.5                   # max over ranks, seen by every rank
    assert out[0][3] == out[1][3] == pytest.approx(2 * 3 / 2.5)


def test_single_rank_is_local():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(4.0) == 4.0
    assert bench.geometry_seeds(0, 2) == [1000, 1001]
