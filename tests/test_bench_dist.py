"""The multi-rank (replica) path of bench.py on CPU: two gloo ranks take the maximum of
their timings and report the whole-job rate."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_q):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms = 100.0 + 50.0 * rank                 # rank 1 is the slow one
    m = bench.max_over_ranks(ms)
    rate = bench.aggregate_rate(1000.0, world, m * 1e-3)
    dist.barrier()
    dist.destroy_process_group()
    out_q.put((rank, m, rate))


def test_two_gloo_ranks_take_the_slowest_time():
    import torch.multiprocessing as mp

    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, rate in res:
        assert m == 150.0
        assert rate == pytest.approx(2 * 1000.0 / 0.150)


def test_single_process_is_unchanged():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.aggregate_rate(10.0, 1, 2.0) == 5.0
