"""The multi-process (one replica per rank) host logic of bench.py, on CPU
with the gloo backend and two ranks: the step time is the maximum over the
ranks, every rank sees it, and the reduction does not depend on the order
in which ranks arrive."""
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


def _rank(rank, world, port, q):
    import time
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        if rank == 1:
            time.sleep(0.2)  # arrive late
        local = 0.5 + rank  # rank 1 is the slow replica
        got = bench.max_over_ranks(local)
        dist.barrier()
        q.put((rank, got))
    finally:
        dist.destroy_process_group()


def test_step_time_is_max_over_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        if p.is_alive():
            p.terminate()
            pytest.fail("a rank did not finish")
        assert p.exitcode == 0
    res = dict(q.get(timeout=10) for _ in range(world))
    assert res == {0: 1.5, 1: 1.5}
