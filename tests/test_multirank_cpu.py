"""Host logic of the N > 1 benchmark path on CPU with world-size-2 gloo ranks:
the job time is the largest rank time (barrier + max reduction), the job
throughput counts every rank's solves, and the reference arm runs on rank 0
only.  No GPU: the reduction is the same torch.distributed call bench.py
makes with NCCL."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import sys
    import torch
    import torch.distributed as dist
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            init_method=f"tcp://127.0.0.1:{port}")
    dist.barrier()
    t = bench.max_over_ranks(1.0 + 0.5 * rank, dist, torch.device("cpu"))
    out.put((rank, t, bench.job_throughput(world, 4, t)))
    dist.destroy_process_group()


def test_job_time_is_the_max_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [1.5, 1.5]       # both ranks see the slowest time
    assert all(abs(r[2] - 2 * 4 / 1.5) < 1e-12 for r in res)


def test_single_process_keeps_its_time():
    import bench
    assert bench.max_over_ranks(2.5, None, None) == 2.5
    assert bench.job_throughput(1, 5, 2.5) == 2.0


def test_reference_arm_runs_on_rank_zero_only(capsys):
    import bench

    class Args:
        n, p, steps, warmup, cpu_seconds = 64, 2, 1, 0, 0.1
    bench.run_reference(Args(), rank=1, world=2)   # returns at once, prints nothing
    assert capsys.readouterr().out == ""
