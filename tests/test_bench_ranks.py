"""Host logic of the multi-GPU bench (every rank runs an independent replica):
the step time is the maximum over ranks and the job's throughput counts every
rank's units; under torchrun only rank 0 runs the oracle reference arm.  Run as
two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, local_ms, q):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(local_ms[rank], world, device="cpu")
        q.put((rank, t, bench.job_throughput(1000, t, world)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_throughput_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    local_ms = [2.0, 5.0]
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, local_ms, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, thr in out:
        assert t == 5.0                       # every rank sees the slowest rank's time
        assert thr == pytest.approx(2 * 1000 / 5e-3)   # both ranks' units in that time


def test_single_rank_is_identity():
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.job_throughput(10, 2.0, 1) == pytest.approx(5000.0)


def test_reference_arm_runs_on_rank_zero_only():
    class A:
        steps, warmup = 1, 3
    assert bench.run_reference(A(), rank=1, world=2) is None
