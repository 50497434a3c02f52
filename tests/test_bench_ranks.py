"""The multi-rank (replicas) path of bench.py on CPU: two gloo ranks agree on the slowest rank's
time, the whole-job rate counts every rank's units, and the reference arm prints from rank 0
only."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    got = bench.max_over_ranks(10.0 + 5.0 * rank)
    out[rank] = got
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert dict(out) == {0: 15.0, 1: 15.0}


def test_whole_job_rate_and_single_process_defaults():
    import bench

    assert bench.max_over_ranks(3.5) == 3.5  # no process group: unchanged
    assert bench.whole_job_rate(131584, 1, 10.0) == pytest.approx(13.1584)
    assert bench.whole_job_rate(131584, 4, 10.0) == pytest.approx(4 * 13.1584)


def test_reference_arm_prints_only_on_rank_zero(capsys):
    import argparse

    import bench

    args = argparse.Namespace(gpus=2, steps=1, warmup=0, impl="reference")
    bench.run_reference(args, world=2, rank=1)
    assert capsys.readouterr().out == ""
