"""bench.py's multi-GPU arm runs independent replicas (the operator pair needs no exchange):
the host logic that combines them -- max of the step time over ranks, whole-job throughput --
checked with two gloo ranks on the CPU."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    value, ms_max = bench.replica_throughput(100.0 + 50.0 * rank, 1e9, world, "cpu")
    out[rank] = (value, ms_max)
    dist.destroy_process_group()


def test_replica_throughput_two_gloo_ranks():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        value, ms_max = out[r]
        assert ms_max == 150.0                                # the slower replica's time
        assert value == pytest.approx(2 * 2.0 * 1e9 / 0.150)  # both replicas' samples / that time


def test_replica_throughput_single_rank():
    import bench
    value, ms_max = bench.replica_throughput(200.0, 5e8, 1, "cpu")
    assert ms_max == 200.0 and value == pytest.approx(2.0 * 5e8 / 0.2)
