"""The multi-rank side of bench.py on CPU: two gloo ranks agree on the
slowest rank's time, the whole-job value counts every rank's units, and the
reference arm runs on rank 0 only."""
import contextlib
import io
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(10.0 * (rank + 1), dist, "cpu")
        out[rank] = (ms, bench.job_value(world, 1000, ms))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    # both ranks see the slower rank's 20 ms; 2 x 1000 units in 20 ms
    assert res[0] == res[1] == (20.0, pytest.approx(1e5))


def test_single_process_keeps_its_time():
    assert bench.max_over_ranks(12.5, None, "cpu") == 12.5
    assert bench.job_value(1, 64153844, 416.0) == pytest.approx(64153844 / 0.416)


def test_reference_arm_only_on_rank_zero():
    class Args:
        workload, scale, steps, warmup, gpus = "er2000", 22, 1, 0, 2
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(Args, rank=1, world=2)
    assert buf.getvalue() == ""
