"""The bench's multi-process path on the CPU (gloo, world size 2): every rank
gets the slowest rank's time, the whole-job value counts every rank's
entries, and only rank 0 of the reference arm does any work. (With GPUs the
same code runs one rank per GPU over NCCL.)"""
import io
import contextlib
import os
import socket
import sys

import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    r, w, local = bench.dist_env()
    ms = bench.combine_ranks(10.0 + 5.0 * rank, world, torch.device("cpu"))
    value = bench.aggregate_value(world, 1_000_000, 4, ms)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, r, w, local, ms, value))


def test_two_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(k, 2, port, q)) for k in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, r, w, local, ms, value in out:
        assert (r, w, local) == (rank, 2, rank)
        assert ms == 15.0  # the slower rank's
        assert value == pytest.approx(2 * 1_000_000 * 4 / 0.015 / 1e9)


def test_reference_arm_other_ranks_do_nothing():
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        pass

    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        assert bench.run_reference(Args(), rank=1, world=2) == 0
    assert buf.getvalue() == ""
