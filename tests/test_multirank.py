"""The bench's multi-rank host logic on CPU with two gloo ranks (127.0.0.1): the elapsed time is
the maximum over ranks and reaches every rank, the whole-job rate counts every rank's solves, and
the reference arm runs on rank 0 only.  No GPU is used."""

import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(times[rank], world, "cpu")
        out[rank] = (ms, bench.whole_job_rate(5, world, ms))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        times = [120.0, 150.0]
        mp.start_processes(_rank_main, args=(2, _free_port(), times, out), nprocs=2, join=True,
                           start_method="spawn")
        res = dict(out)
    assert res[0][0] == 150.0 and res[1][0] == 150.0
    assert res[0][1] == pytest.approx(2 * 5 / 0.150)


def test_single_rank_keeps_local_time():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(42.0, 1, "cpu") == 42.0
    assert bench.whole_job_rate(10, 1, 500.0) == pytest.approx(20.0)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        steps, warmup, ref_n, gpus = 1, 0, 9, 2

    bench.run_reference(Args, rank=1, world=2)
    assert capsys.readouterr().out == ""
