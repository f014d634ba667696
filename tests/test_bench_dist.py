"""The N > 1 path of bench.py on CPU: two gloo ranks (world_size 2) take the
maximum of their times and report the whole-job rate (every rank runs its own
replica of the workload; nothing else is exchanged)."""
import os
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_time = [2.5, 4.0][rank]              # seconds for 10 steps of 6 solutions
    t = bench.max_over_ranks(local_time, world)
    v = bench.job_throughput(world, 6 * 10, t)
    q.put((rank, t, v))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation():
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, v in out:
        assert t == 4.0                         # the slowest rank's time, on every rank
        assert v == pytest.approx(2 * 60 / 4.0)  # both replicas' solutions in that time


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, 1) == 3.25
    assert bench.job_throughput(1, 12, 3.0) == 4.0
