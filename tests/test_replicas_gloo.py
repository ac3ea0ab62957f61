"""The multi-GPU mode is replicas only: each rank factors its own matrix and
the only collective reduces the step time to the slowest rank's.  That host
logic of bench.py runs here as two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(100.0 + 10.0 * rank, world, "cpu")
        rate = bench.job_rate(1e12, ms, world)
        dist.barrier()
        q.put((rank, ms, rate))
    finally:
        dist.destroy_process_group()


def test_single_rank_passthrough():
    assert bench.max_over_ranks(12.5, 1, "cpu") == 12.5
    assert bench.job_rate(2e12, 1000.0, 1) == pytest.approx(2000.0)


def test_two_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [110.0, 110.0]
    # both replicas' work over the slowest replica's time
    assert out[0][2] == pytest.approx(2 * 1e12 / 0.110 / 1e9)
