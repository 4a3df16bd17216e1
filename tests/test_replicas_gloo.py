"""Multi-process path of bench.py on CPU: world size 2 over gloo.

With N GPUs every rank solves its own copy of the workload (the batch
dimension is independent, so there is no collective on the data path); the
only exchange is the whole-job timing: the slowest rank's time (max) and all
ranks' work (sum). This runs that reduction as two gloo ranks on the host.
"""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t_local = [0.5, 0.8][rank]      # rank 1 is the slower one
    work_local = [1000.0, 3000.0][rank]
    t, w = bench.reduce_over_ranks(dist, t_local, work_local, torch.device("cpu"))
    out[rank] = (t, w)
    dist.barrier()
    dist.destroy_process_group()


def test_whole_job_value_is_total_work_over_slowest_rank():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        t, w = out[r]
        assert t == 0.8
        assert w == 4000.0
    assert out[0][1] / out[0][0] == 5000.0


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks(None, 0.25, 7.0, None) == (0.25, 7.0)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    """Under torchrun the oracle arm runs on rank 0 only; other ranks exit without work."""
    sys.path.insert(0, ROOT)
    import argparse

    import bench
    args = argparse.Namespace(steps=1, warmup=0, ref_iters=1)
    assert bench.reference_arm(args, rank=1, world=2) is None
    assert capsys.readouterr().out == ""
