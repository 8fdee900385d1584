"""The multi-replica path of bench.py on two CPU processes (gloo): the
whole-job time is the maximum over ranks and the work is the sum."""
import multiprocessing as mp
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        q.put((rank, bench.combine_ranks(1.5 + rank, 100.0 * (rank + 1), "cpu")))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_max_time_and_summed_work():
    pytest.importorskip("torch")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out[0] == out[1] == (2.5, 300.0)


def test_single_process_is_the_identity():
    import bench
    assert bench.combine_ranks(2.0, 7.0, "cpu") == (2.0, 7.0)
