"""The multi-rank pieces of bench.py (barrier, max over ranks, whole-job rate) on two gloo
ranks on the CPU: the same calls the benchmark makes between replicas on several GPUs."""
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
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench.barrier(world)
    t = 1.0 + 0.5 * rank  # the slower replica decides the step time
    t_max = bench.max_over_ranks(t, world)
    out[rank] = (t_max, bench.whole_job_rate(1e9, t_max, world))
    bench.barrier(world)
    dist.destroy_process_group()


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as manager:
        out = manager.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
        assert all(p.exitcode == 0 for p in procs)
        for r in range(world):
            t_max, rate = out[r]
            assert t_max == 1.5
            assert abs(rate - world * 1e9 / 1.5 / 1e9) < 1e-12


def test_single_rank_helpers():
    import bench
    assert bench.max_over_ranks(3.0, 1) == 3.0
    bench.barrier(1)
    assert bench.whole_job_rate(2e9, 2.0, 1) == 1.0

