"""The multi-rank bookkeeping of bench.py on CPU (gloo, world size 2): every
rank is an independent replica; the job time is the slowest rank's and the
job rate counts every rank's cell-updates. The reference arm runs on rank 0
only."""
import argparse
import io
import os
import sys
from contextlib import redirect_stdout

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t_local = 1.0 + rank  # rank 1 is the slower replica
    t = bench.slowest(t_local, world, "cpu")
    out[rank] = (t, bench.job_rate(world, 3e9, t))
    dist.barrier()
    dist.destroy_process_group()


def test_slowest_rank_sets_the_job_time():
    world = 2
    port = 29500 + os.getpid() % 1000
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(world, port, out), nprocs=world, start_method="spawn")
        res = dict(out)
    assert res[0] == res[1] == (2.0, pytest.approx(2 * 3e9 / 2.0 / 1e9))


def test_single_rank_is_the_identity():
    assert bench.slowest(0.25, 1, "cpu") == 0.25
    assert bench.job_rate(1, 5e9, 0.5) == pytest.approx(10.0)


def test_reference_arm_runs_on_rank_zero_only():
    args = argparse.Namespace(grid=8, time_steps=2, workload="inclusions256", warmup=0, steps=1,
                              gpus=2, operator="pointwise")
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(args, rank=1, world=2)
    assert buf.getvalue() == ""
