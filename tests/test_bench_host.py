"""Host logic of bench.py: multi-rank timing (max over ranks, gloo on CPU,
world size 2) and the whole-job rate of replicated runs."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    out[rank] = bench.max_over_ranks(10.0 + 5.0 * rank, torch.device("cpu"), world)
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert out[0] == 15.0 and out[1] == 15.0


def test_job_rate_weak_scaling():
    import bench
    one = bench.job_rate(8192 * 8192, 64, 1, 2.0)
    assert abs(one - 8192 * 8192 * 64 / 2e-3 / 1e9) < 1e-9
    assert abs(bench.job_rate(8192 * 8192, 64, 4, 2.0) - 4 * one) < 1e-6
    assert bench.max_over_ranks(3.5, None, 1) == 3.5
