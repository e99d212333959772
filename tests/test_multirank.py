"""The N > 1 path of bench.py on CPU: ranks work on independent batches (no
data-path collective) and only the timing is reduced (max over ranks) along
with the total work (sum over ranks).  world_size 2 with the gloo backend."""
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [10.0, 17.5][rank]
    mpix = [3.0, 5.0][rank]
    q.put((rank, bench.reduce_rank_metrics(ms, mpix, dist)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_reduce_time_and_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out[0] == out[1] == (17.5, 8.0)


def test_ranks_get_independent_batches():
    sys.path.insert(0, ROOT)
    import bench
    a = bench.problems_for_rank(0, count=3)
    b = bench.problems_for_rank(1, count=3)
    assert any((x.g.shape != y.g.shape) or abs(x.delta - y.delta) > 0 for x, y in zip(a, b))


def test_single_rank_passthrough():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_rank_metrics(4.0, 2.0, None) == (4.0, 2.0)
