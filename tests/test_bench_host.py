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


def test_reference_arm_json_line():
    """The reference arm (the FP64 oracle on the host cores) runs without a
    GPU and prints one JSON line with the keys the benchmark contract asks
    for, on the main arm's metric and workload."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1"], capture_output=True, text=True, timeout=600, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["metric"].startswith("GStencil/s") and line["unit"] == "GStencil/s"
    assert line["higher_is_better"] is True and line["steps"] == 1 and line["warmup"] >= 3
    assert line["value"] > 0 and line["config"]["workload"].startswith("2d5p 8192x8192")
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
