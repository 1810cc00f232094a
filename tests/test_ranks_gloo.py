"""Multi-rank host logic of bench.py with two gloo ranks on the CPU: the
barrier, the max over ranks of the elapsed time and the whole-job rate."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(WORLD_SIZE=str(world), RANK=str(rank), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    from paper_2205_15000_b300 import ranks
    dist = ranks.init("gloo")
    ranks.barrier(dist)
    mine = 1.0 + rank  # rank 1 is the slow one
    slow = ranks.max_over_ranks(dist, mine)
    rate = ranks.throughput(100.0, world, slow)
    q.put((rank, slow, rate, ranks.env_ranks()))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, slow, rate, env in res:
        assert slow == 2.0
        assert rate == pytest.approx(100.0)  # 2 ranks x 100 units / 2 s
        assert env == (2, rank, rank)


def test_single_rank_needs_no_process_group():
    from paper_2205_15000_b300 import ranks
    assert ranks.init() is None
    assert ranks.max_over_ranks(None, 3.5) == 3.5
    assert ranks.throughput(10.0, 1, 2.0) == 5.0
